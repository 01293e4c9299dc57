// Plane-wave set of one k-point (Sec. 2): all integer n with |(n + k) . B| <= K_max.
// Host code, compiled with -ffp-contract=off so that |k+G|^2 is evaluated
// exactly as written (the order below is part of the interface).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "flapw_internal.h"

namespace flapw {

// b_i = 2 pi (a_j x a_k) / det, det = a_1 . (a_2 x a_3).
void reciprocal(const double lat[9], double rec[9], double* det_out) {
  auto cross = [](const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  double c[3][3];
  cross(lat + 3, lat + 6, c[0]);
  cross(lat + 6, lat + 0, c[1]);
  cross(lat + 0, lat + 3, c[2]);
  double det = lat[0] * c[0][0] + lat[1] * c[0][1] + lat[2] * c[0][2];
  double f = 6.283185307179586 / det;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) rec[3 * i + j] = f * c[i][j];
  if (det_out) *det_out = det;
}

namespace {
struct Cand {
  int64_t key;
  int n[3];
  bool operator<(const Cand& o) const {
    if (key != o.key) return key < o.key;
    if (n[0] != o.n[0]) return n[0] < o.n[0];
    if (n[1] != o.n[1]) return n[1] < o.n[1];
    return n[2] < o.n[2];
  }
};
}  // namespace

// Returns N_G and fills n3 (3 ints per plane wave) in ascending |k+G|^2
// quantised to 2^-40 K_max^2, ties by (n1, n2, n3).
int enumerate_g(const double lat[9], const double k[3], double kmax, std::vector<int>* n3) {
  double rec[9], det;
  reciprocal(lat, rec, &det);
  if (!(std::fabs(det) > 0) || !(kmax > 0)) return -1;
  int lim[3];
  for (int i = 0; i < 3; ++i) {
    const double* a = lat + 3 * i;
    double alen = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    lim[i] = static_cast<int>(std::ceil(kmax * alen / 6.283185307179586)) + 2;
  }
  const double kk = kmax * kmax;
  std::vector<Cand> out;
  for (int i = -lim[0]; i <= lim[0]; ++i) {
    const double q1 = i + k[0];
    for (int j = -lim[1]; j <= lim[1]; ++j) {
      const double q2 = j + k[1];
      for (int l = -lim[2]; l <= lim[2]; ++l) {
        const double q3 = l + k[2];
        double K[3];
        for (int c = 0; c < 3; ++c) K[c] = q1 * rec[c] + q2 * rec[3 + c] + q3 * rec[6 + c];
        const double K2 = K[0] * K[0] + K[1] * K[1] + K[2] * K[2];
        if (K2 <= kk) out.push_back(Cand{std::llround(K2 / kk * 1099511627776.0), {i, j, l}});
      }
    }
  }
  std::sort(out.begin(), out.end());
  n3->resize(out.size() * 3);
  for (size_t g = 0; g < out.size(); ++g)
    for (int c = 0; c < 3; ++c) (*n3)[3 * g + c] = out[g].n[c];
  return static_cast<int>(out.size());
}

}  // namespace flapw
