// Matching coefficients A, B (Sec. 2, Eq. (basis)).
//
//   A^{a,G}_{lm} = 4 pi/sqrt(Omega) e^{i K.tau_a} i^l conj(Y_lm(K_hat)) a_l(|K|)
//   B^{a,G}_{lm} = same with b_l,     K = k + G,
//   a u(R) + b udot(R) = j_l(|K|R),  a u'(R) + b udot'(R) = |K| j_l'(|K|R),
//
// i.e. continuity of value and slope with the plane wave at the sphere.  The
// work splits in two kernels:
//   ab_prep     one thread per (plane wave, job), a job being one order m of
//               Y_lm (normalised associated-Legendre recurrence over l), the
//               radial matching of one type (j_l by Miller's downward
//               recurrence, or the stable upward one when x > l_max, then the
//               2x2 solve per l), or the phases of kPhaseAtoms atoms with an
//               exact FP64 reduction of the argument (n + k).tau to
//               [-1/2, 1/2] turns.
//   ab_assemble one thread per (G, L, atom): A = phase * Yc * a_l, B likewise,
//               16-byte stores coalesced along G.  The kernel is bound by the
//               32 bytes it stores per (atom, L, G); its loads (Yc shared by
//               all atoms, the phase by all L) mostly hit L2.
#include <cmath>

#include "flapw_internal.h"

namespace flapw {
namespace {

constexpr int kMaxL1 = kMaxLmax + 2;  // j_0 .. j_{lmax+1}
constexpr int kPhaseAtoms = 8;        // atom phases per ab_prep job

// Spherical Bessel j_0..j_L at x >= 0 into j[0..L].
__device__ void sph_bessel_all(int L, double x, double* j) {
  if (x < 1e-3) {
    // ascending series, three terms: relative error < x^6 / 48
    double xl = 1.0, dfac = 1.0;
    for (int l = 0; l <= L; ++l) {
      if (l > 0) {
        xl *= x;
        dfac *= (2 * l + 1);
      }
      const double x2 = x * x;
      j[l] = xl / dfac * (1.0 - x2 / (2.0 * (2 * l + 3)) + x2 * x2 / (8.0 * (2 * l + 3) * (2 * l + 5)));
    }
    return;
  }
  double s, c;
  sincos(x, &s, &c);
  if (x > L) {
    // upward recurrence is stable for x > l
    j[0] = s / x;
    if (L >= 1) j[1] = s / (x * x) - c / x;
    for (int l = 1; l < L; ++l) j[l + 1] = (2 * l + 1) / x * j[l] - j[l - 1];
    return;
  }
  // Miller: recur downward from N well above max(L, x), normalise with
  // sum_l (2l+1) j_l^2 = 1.
  const int N = (L > (int)x ? L : (int)x) + 25;
  double fp1 = 0.0, f = 1e-100, norm = 0.0;
  for (int l = N; l >= 1; --l) {
    if (l <= L) j[l] = f;
    norm += (2 * l + 1) * f * f;
    const double fm1 = (2 * l + 1) / x * f - fp1;
    fp1 = f;
    f = fm1;
  }
  j[0] = f;
  norm += f * f;
  const double sc = 1.0 / sqrt(norm);
  // fix the sign with j_0 = sin x / x where it is not small, else with j_1
  double ref = s / x, got = f;
  if (fabs(ref) < 0.1 && L >= 1) {
    ref = s / (x * x) - c / x;
    got = j[1];
  }
  const double sg = ((ref >= 0) == (got >= 0)) ? sc : -sc;
  for (int l = 0; l <= L; ++l) j[l] *= sg;
}

// Fractional part of n . tau in [-1/2, 1/2] turns, each product reduced with
// its exact rounding error (fma), plus k . tau precomputed in FP64.
__device__ double phase_turns(const int* n, const double* tau, double ktau) {
  double f = 0.0, e = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double nd = (double)n[i];
    const double p = nd * tau[i];
    e += fma(nd, tau[i], -p);
    f += p - rint(p);
  }
  f += e + ktau;
  return f - rint(f);
}

// grid: (ceil(G / 128), lmax + 1 + n_types + ceil(n_atoms / kPhaseAtoms)).
__global__ void __launch_bounds__(128) ab_prep_kernel(Geom geo, GData gd, const double* radial,
                                                      const double* coef, double2* Yc, double* al,
                                                      double* bl, double2* ph) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= geo.g_total) return;
  const int64_t G = geo.g_total;
  const int k = gd.gk[gi];
  const int n[3] = {gd.n3[3 * gi], gd.n3[3 * gi + 1], gd.n3[3 * gi + 2]};
  const int lmax = geo.lmax;
  const int job = blockIdx.y;
  if (job > lmax + geo.n_types) {
    // atom phases e^{2 pi i (n + k).tau}
    const int a0 = (job - lmax - 1 - geo.n_types) * kPhaseAtoms;
    const int a1 = min(geo.n_atoms, a0 + kPhaseAtoms);
    for (int a = a0; a < a1; ++a) {
      const double f = phase_turns(n, geo.pos + 3 * a, geo.ktau[(int64_t)k * geo.n_atoms + a]);
      double s, c;
      sincospi(2.0 * f, &s, &c);
      ph[(int64_t)a * G + gi] = make_double2(c, s);
    }
    return;
  }
  const double q0 = n[0] + geo.kfrac[3 * k], q1 = n[1] + geo.kfrac[3 * k + 1],
               q2 = n[2] + geo.kfrac[3 * k + 2];
  double K[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) K[c] = q0 * geo.rec[c] + q1 * geo.rec[3 + c] + q2 * geo.rec[6 + c];
  const double rho2 = K[0] * K[0] + K[1] * K[1];
  const double kabs = sqrt(rho2 + K[2] * K[2]);
  if (job > lmax) {
    // radial matching of one type, per l
    const int t = job - lmax - 1;
    double j[kMaxL1];
    const double R = geo.radius[t];
    const double x = kabs * R;
    sph_bessel_all(lmax + 1, x, j);
    for (int l = 0; l <= lmax; ++l) {
      double dj = 0.0;
      if (kabs > 0) {
        const double jd = (l == 0) ? -j[1] : j[l - 1] - (l + 1) / x * j[l];
        dj = kabs * jd;
      }
      const double* rd = radial + ((int64_t)t * (lmax + 1) + l) * 4;
      const double u = rd[0], up = rd[1], ud = rd[2], udp = rd[3];
      const double D = u * udp - up * ud;
      const int64_t o = ((int64_t)t * (lmax + 1) + l) * G + gi;
      al[o] = (j[l] * udp - dj * ud) / D;
      bl[o] = (u * dj - up * j[l]) / D;
    }
    return;
  }
  // Yc[L] = pref * i^l * conj(Y_lm) for m = job: normalised Legendre recurrence over l
  double ct = 1.0, st = 0.0, ep_re = 1.0, ep_im = 0.0;
  if (kabs > 0) {
    ct = K[2] / kabs;
    const double rho = sqrt(rho2);
    st = rho / kabs;
    if (rho > 0) {
      ep_re = K[0] / rho;
      ep_im = K[1] / rho;
    }
  }
  const int m = job;
  double pmm = 0.28209479177387814;  // 1/sqrt(4 pi)
  double em_re = 1.0, em_im = 0.0;   // e^{i m phi}
  for (int mm = 1; mm <= m; ++mm) {
    pmm *= -coef[2 * (mm * (mm + 1) / 2 + mm)] * st;
    const double r = em_re * ep_re - em_im * ep_im;
    em_im = em_re * ep_im + em_im * ep_re;
    em_re = r;
  }
  double p2 = 0.0, p1 = 0.0;
  for (int l = m; l <= lmax; ++l) {
    double p;
    if (l == m) {
      p = pmm;
    } else if (l == m + 1) {
      p = coef[2 * (l * (l + 1) / 2 + m)] * ct * pmm;
    } else {
      const int ci = 2 * (l * (l + 1) / 2 + m);
      p = coef[ci] * (ct * p1 - coef[ci + 1] * p2);
    }
    p2 = p1;
    p1 = p;
    // i^l
    double il_re = 0.0, il_im = 0.0;
    switch (l & 3) {
      case 0: il_re = 1.0; break;
      case 1: il_im = 1.0; break;
      case 2: il_re = -1.0; break;
      default: il_im = -1.0; break;
    }
    const double a = geo.pref * p;
    // conj(Y_lm) = P e^{-i m phi}
    const double y_re = a * em_re, y_im = -a * em_im;
    Yc[(int64_t)(l * l + l + m) * G + gi] =
        make_double2(il_re * y_re - il_im * y_im, il_re * y_im + il_im * y_re);
    if (m > 0) {
      // conj(Y_{l,-m}) = (-1)^m Y_lm = (-1)^m P e^{i m phi}
      const double sg = (m & 1) ? -a : a;
      const double z_re = sg * em_re, z_im = sg * em_im;
      Yc[(int64_t)(l * l + l - m) * G + gi] =
          make_double2(il_re * z_re - il_im * z_im, il_re * z_im + il_im * z_re);
    }
  }
}

// gtiles: (k, g0) pairs, 128 plane waves each.  grid: (tiles, N_L, atoms).
__global__ void __launch_bounds__(128) ab_assemble_kernel(Geom geo, const int* gtiles,
                                                          const int64_t* goff, const double2* Yc,
                                                          const double* al, const double* bl,
                                                          const double2* ph, double2* A,
                                                          double2* B) {
  const int k = gtiles[2 * blockIdx.x], g0 = gtiles[2 * blockIdx.x + 1];
  const int L = blockIdx.y, a = blockIdx.z;
  const int g = g0 + threadIdx.x;
  const int64_t ng = goff[k + 1] - goff[k];
  if (g >= ng) return;
  const int64_t G = geo.g_total;
  const int64_t gi = goff[k] + g;
  const int t = geo.type[a];
  const int nl = geo.n_L;
  int l = 0;  // L = l^2 + l + m
  while ((l + 1) * (l + 1) <= L) ++l;
  const double2 p = ph[(int64_t)a * G + gi];
  const double2 y = Yc[(int64_t)L * G + gi];
  const int64_t ro = ((int64_t)t * (geo.lmax + 1) + l) * G + gi;
  const double ra = al[ro], rb = bl[ro];
  const double w_re = p.x * y.x - p.y * y.y, w_im = p.x * y.y + p.y * y.x;
  const int64_t o = (int64_t)nl * geo.n_atoms * goff[k] + ((int64_t)a * nl + L) * ng + g;
  A[o] = make_double2(w_re * ra, w_im * ra);
  B[o] = make_double2(w_re * rb, w_im * rb);
}

}  // namespace

cudaError_t launch_ab_prep(const Geom& geo, const GData& gd, const double* radial,
                           const double* ylm_coef, double2* Yc, double* al, double* bl,
                           double2* ph, cudaStream_t st) {
  if (geo.g_total == 0) return cudaSuccess;
  const unsigned jobs = (unsigned)(geo.lmax + 1 + geo.n_types + (geo.n_atoms + kPhaseAtoms - 1) / kPhaseAtoms);
  dim3 grid((unsigned)((geo.g_total + 127) / 128), jobs);
  ab_prep_kernel<<<grid, 128, 0, st>>>(geo, gd, radial, ylm_coef, Yc, al, bl, ph);
  return cudaGetLastError();
}

cudaError_t launch_ab_assemble_tiles(const Geom& geo, const int* gtiles, int n_gtiles,
                                     const int64_t* goff, const double2* Yc, const double* al,
                                     const double* bl, const double2* ph, double2* A, double2* B,
                                     cudaStream_t st) {
  if (n_gtiles == 0 || geo.n_atoms == 0) return cudaSuccess;
  dim3 grid(n_gtiles, geo.n_L, geo.n_atoms);
  ab_assemble_kernel<<<grid, 128, 0, st>>>(geo, gtiles, goff, Yc, al, bl, ph, A, B);
  return cudaGetLastError();
}

}  // namespace flapw
