/*
 * CPU oracle for the FLAPW muffin-tin Hamiltonian / overlap build.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code with the CUDA path and is deliberately plain and slow: every quantity
 * is computed from its textbook definition with straight loops.
 *
 * What it follows:
 *   - Plane-wave set {G : |k+G| <= K_max} (Sec. 2, the expansion of psi_{k,nu}).
 *   - LAPW basis inside sphere a (Sec. 2, Eq. (basis)):
 *       phi_G(r) = sum_lm [A^{a,G}_lm u_l(r) + B^{a,G}_lm udot_l(r)] Y_lm(r_hat)
 *     with A, B fixed by continuity of value and slope with the plane wave
 *     Omega^{-1/2} exp(i (k+G).r) at the sphere boundary (Sec. 2, after
 *     Eq. (basis)).  The paper prints no formula; the coefficients follow
 *     from the Rayleigh expansion
 *       exp(i K.r) = 4 pi sum_lm i^l j_l(K r) Y*_lm(K_hat) Y_lm(r_hat)
 *     and a 2x2 Cramer solve per (type, l) against u, u', udot, udot' at R.
 *   - Overlap S (Eq. (def_overlap)) and Hamiltonian H (Eq. (def_hamilton)),
 *     equivalently Eqs. (h) and (s):
 *       S_{G'G} = sum_a sum_L conj(A_{L}^{a,G'}) A_L^{a,G}
 *                             + ||udot_l||^2 conj(B_L^{a,G'}) B_L^{a,G}
 *       H_{G'G} = sum_a sum_{L',L} conj(X_{L'}^{a,G'}) T^{[XY]}_{L'L;a} Y_L^{a,G}
 *     summed over the four blocks XY in {AA, AB, BA, BB}.  Row G', column G.
 *
 * Precision: special functions, phases and A/B in long double, stored as
 * double; the H/S sums in double (FP64), one column at a time.
 *
 * Readings taken where the paper is silent (also listed in the design notes):
 *   - G order: ascending |k+G|^2 quantised to 2^-40 of K_max^2, ties broken by
 *     (n1, n2, n3) lexicographically.
 *   - Y_lm complex, orthonormal, Condon-Shortley phase; L = l*l + l + m.
 *   - K = 0 takes K_hat = z.
 *   - U in Eq. (s) is diag(||udot_l||), so S carries ||udot_l||^2.
 *   - T rows/cols ordered [A-part L=0..N_L-1, B-part L=0..N_L-1], row-major.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double real_t;
typedef long double _Complex cplx_t;

static const real_t PI_L = 3.141592653589793238462643383279502884L;

/* ------------------------------------------------------------------ */
/* lattice                                                             */
/* ------------------------------------------------------------------ */

/* Reciprocal vectors b_i = 2 pi (a_j x a_k) / (a_1 . (a_2 x a_3)), in double.
 * Rows of `lat` are a_1, a_2, a_3; rows of `rec` are b_1, b_2, b_3. */
static void recip_double(const double lat[9], double rec[9]) {
  const double *a1 = lat, *a2 = lat + 3, *a3 = lat + 6;
  double c23[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2],
                   a2[0] * a3[1] - a2[1] * a3[0]};
  double c31[3] = {a3[1] * a1[2] - a3[2] * a1[1], a3[2] * a1[0] - a3[0] * a1[2],
                   a3[0] * a1[1] - a3[1] * a1[0]};
  double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2],
                   a1[0] * a2[1] - a1[1] * a2[0]};
  double det = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
  double f = 6.283185307179586 / det;
  for (int j = 0; j < 3; ++j) {
    rec[j] = f * c23[j];
    rec[3 + j] = f * c31[j];
    rec[6 + j] = f * c12[j];
  }
}

static void recip_long(const double lat[9], real_t rec[9], real_t* volume) {
  real_t a[9];
  for (int i = 0; i < 9; ++i) a[i] = lat[i];
  real_t *a1 = a, *a2 = a + 3, *a3 = a + 6;
  real_t c23[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2],
                   a2[0] * a3[1] - a2[1] * a3[0]};
  real_t c31[3] = {a3[1] * a1[2] - a3[2] * a1[1], a3[2] * a1[0] - a3[0] * a1[2],
                   a3[0] * a1[1] - a3[1] * a1[0]};
  real_t c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2],
                   a1[0] * a2[1] - a1[1] * a2[0]};
  real_t det = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
  real_t f = 2 * PI_L / det;
  for (int j = 0; j < 3; ++j) {
    rec[j] = f * c23[j];
    rec[3 + j] = f * c31[j];
    rec[6 + j] = f * c12[j];
  }
  *volume = fabsl(det);
}

/* ------------------------------------------------------------------ */
/* plane-wave set                                                      */
/* ------------------------------------------------------------------ */

typedef struct {
  long long key;
  int n[3];
} gentry_t;

static int gentry_cmp(const void* pa, const void* pb) {
  const gentry_t* a = (const gentry_t*)pa;
  const gentry_t* b = (const gentry_t*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  for (int i = 0; i < 3; ++i)
    if (a->n[i] != b->n[i]) return a->n[i] < b->n[i] ? -1 : 1;
  return 0;
}

/* All integer n with |(n + k) . B| <= kmax, sorted as described in the header.
 * Writes up to max_g triples into n3 (may be NULL) and returns the count. */
int oracle_gvectors(const double lat[9], const double k[3], double kmax, int max_g, int* n3) {
  double rec[9];
  recip_double(lat, rec);
  int nmax[3];
  for (int i = 0; i < 3; ++i) {
    double alen = sqrt(lat[3 * i] * lat[3 * i] + lat[3 * i + 1] * lat[3 * i + 1] +
                       lat[3 * i + 2] * lat[3 * i + 2]);
    nmax[i] = (int)ceil(kmax * alen / 6.283185307179586) + 2;
  }
  double kmax2 = kmax * kmax;
  size_t cap = (size_t)(2 * nmax[0] + 1) * (2 * nmax[1] + 1) * (2 * nmax[2] + 1);
  gentry_t* list = (gentry_t*)malloc(cap * sizeof(gentry_t));
  if (!list) return -1;
  int count = 0;
  for (int n1 = -nmax[0]; n1 <= nmax[0]; ++n1)
    for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2)
      for (int n3i = -nmax[2]; n3i <= nmax[2]; ++n3i) {
        double q1 = n1 + k[0], q2 = n2 + k[1], q3 = n3i + k[2];
        double K[3];
        for (int j = 0; j < 3; ++j) K[j] = q1 * rec[j] + q2 * rec[3 + j] + q3 * rec[6 + j];
        double K2 = K[0] * K[0] + K[1] * K[1] + K[2] * K[2];
        if (K2 <= kmax2) {
          list[count].key = llround(K2 / kmax2 * 1099511627776.0);
          list[count].n[0] = n1;
          list[count].n[1] = n2;
          list[count].n[2] = n3i;
          ++count;
        }
      }
  qsort(list, (size_t)count, sizeof(gentry_t), gentry_cmp);
  if (n3) {
    int m = count < max_g ? count : max_g;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < 3; ++j) n3[3 * i + j] = list[i].n[j];
  }
  free(list);
  return count;
}

/* ------------------------------------------------------------------ */
/* spherical Bessel functions (Abramowitz & Stegun 10.1.2, 10.1.8)      */
/* ------------------------------------------------------------------ */

static real_t factl(int n) {
  real_t f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

/* Ascending series: j_l(x) = x^l/(2l+1)!! sum_n (-x^2/2)^n / (n! prod_{i=1..n}(2l+2i+1)). */
static real_t jl_series(int l, real_t x) {
  real_t pref = 1;
  for (int i = 1; i <= l; ++i) pref *= x / (2 * i + 1);
  real_t term = 1, sum = 1, h = -x * x / 2;
  for (int n = 1; n < 400; ++n) {
    term *= h / ((real_t)n * (real_t)(2 * l + 2 * n + 1));
    sum += term;
    if (fabsl(term) <= 1e-30L * fabsl(sum)) break;
  }
  return pref * sum;
}

/* Finite trigonometric form: j_l(x) = [P sin(x - l pi/2) + Q cos(x - l pi/2)] / x. */
static real_t jl_trig(int l, real_t x) {
  real_t P = 0, Q = 0, t2 = 2 * x;
  for (int k = 0; 2 * k <= l; ++k) {
    real_t c = factl(l + 2 * k) / (factl(2 * k) * factl(l - 2 * k)) / powl(t2, 2 * k);
    P += (k % 2 ? -c : c);
  }
  for (int k = 0; 2 * k + 1 <= l; ++k) {
    real_t c = factl(l + 2 * k + 1) / (factl(2 * k + 1) * factl(l - 2 * k - 1)) / powl(t2, 2 * k + 1);
    Q += (k % 2 ? -c : c);
  }
  real_t arg = x - l * PI_L / 2;
  return (P * sinl(arg) + Q * cosl(arg)) / x;
}

static real_t jl(int l, real_t x) {
  if (x == 0) return l == 0 ? 1 : 0;
  if (x < l + 1 || x < 2) return jl_series(l, x);
  return jl_trig(l, x);
}

/* d/dx j_l(x) = j_{l-1}(x) - (l+1)/x j_l(x);  j_0' = -j_1. */
static real_t jl_deriv(int l, real_t x) {
  if (x == 0) return l == 1 ? (real_t)1 / 3 : 0;
  if (l == 0) return -jl(1, x);
  return jl(l - 1, x) - (l + 1) / x * jl(l, x);
}

void oracle_sph_bessel(int l, double x, double* j, double* dj) {
  *j = (double)jl(l, x);
  *dj = (double)jl_deriv(l, x);
}

/* ------------------------------------------------------------------ */
/* spherical harmonics                                                 */
/* ------------------------------------------------------------------ */

/* Y_lm(theta, phi) for all l <= lmax, |m| <= l, at index L = l*l + l + m.
 * P_l^m with the Condon-Shortley phase by the standard recurrences
 *   P_m^m = (-1)^m (2m-1)!! sin^m(theta),  P_{m+1}^m = (2m+1) cos(theta) P_m^m,
 *   (l-m) P_l^m = (2l-1) cos(theta) P_{l-1}^m - (l+m-1) P_{l-2}^m,
 * Y_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m e^{i m phi},
 * Y_{l,-m} = (-1)^m conj(Y_lm). */
static void ylm_all(int lmax, real_t theta, real_t phi, cplx_t* Y) {
  real_t x = cosl(theta), sx = sinl(theta);
  for (int m = 0; m <= lmax; ++m) {
    real_t pmm = 1;
    for (int i = 1; i <= m; ++i) pmm *= -(2 * i - 1) * sx;
    real_t plm2 = 0, plm1 = 0;
    for (int l = m; l <= lmax; ++l) {
      real_t p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = x * (2 * m + 1) * pmm;
      else p = ((2 * l - 1) * x * plm1 - (l + m - 1) * plm2) / (l - m);
      plm2 = plm1;
      plm1 = p;
      real_t norm = sqrtl((2 * l + 1) / (4 * PI_L) * factl(l - m) / factl(l + m));
      cplx_t e = cosl(m * phi) + I * sinl(m * phi);
      cplx_t y = norm * p * e;
      Y[l * l + l + m] = y;
      if (m > 0) Y[l * l + l - m] = ((m % 2) ? -1 : 1) * conjl(y);
    }
  }
}

void oracle_ylm(int lmax, double theta, double phi, double* out) {
  int nl = (lmax + 1) * (lmax + 1);
  cplx_t* Y = (cplx_t*)malloc(sizeof(cplx_t) * nl);
  ylm_all(lmax, theta, phi, Y);
  for (int i = 0; i < nl; ++i) {
    out[2 * i] = (double)creall(Y[i]);
    out[2 * i + 1] = (double)cimagl(Y[i]);
  }
  free(Y);
}

/* ------------------------------------------------------------------ */
/* matching coefficients A, B for one plane wave                       */
/* ------------------------------------------------------------------ */

typedef struct {
  const double* lat;
  int n_atoms;
  const double* pos;
  const int* type;
  int n_types;
  const double* radius;
  int lmax;
  const double* k;
  const double* radial; /* [n_types][lmax+1][4] */
  real_t rec[9];
  real_t volume;
} ab_ctx_t;

static void ab_ctx_init(ab_ctx_t* c, const double* lat, int n_atoms, const double* pos,
                        const int* type, int n_types, const double* radius, int lmax,
                        const double* k, const double* radial) {
  c->lat = lat;
  c->n_atoms = n_atoms;
  c->pos = pos;
  c->type = type;
  c->n_types = n_types;
  c->radius = radius;
  c->lmax = lmax;
  c->k = k;
  c->radial = radial;
  recip_long(lat, c->rec, &c->volume);
}

/* A[a][L], B[a][L] for the plane wave with integer index n (Sec. 2, Eq. (basis)):
 *   f   = 4 pi / sqrt(Omega) * exp(2 pi i (n+k).tau_a) * i^l * conj(Y_lm(K_hat))
 *   A u(R) + B udot(R)   = f j_l(K R)
 *   A u'(R) + B udot'(R) = f K j_l'(K R)                                   */
static void ab_one(const ab_ctx_t* c, const int n[3], cplx_t* A, cplx_t* B) {
  int nl = (c->lmax + 1) * (c->lmax + 1);
  real_t q[3] = {n[0] + (real_t)c->k[0], n[1] + (real_t)c->k[1], n[2] + (real_t)c->k[2]};
  real_t K[3];
  for (int j = 0; j < 3; ++j) K[j] = q[0] * c->rec[j] + q[1] * c->rec[3 + j] + q[2] * c->rec[6 + j];
  real_t kabs = sqrtl(K[0] * K[0] + K[1] * K[1] + K[2] * K[2]);
  real_t theta = 0, phi = 0;
  if (kabs > 0) {
    theta = atan2l(sqrtl(K[0] * K[0] + K[1] * K[1]), K[2]);
    phi = atan2l(K[1], K[0]);
  }
  cplx_t* Y = (cplx_t*)malloc(sizeof(cplx_t) * nl);
  ylm_all(c->lmax, theta, phi, Y);
  real_t* al = (real_t*)malloc(sizeof(real_t) * c->n_types * (c->lmax + 1));
  real_t* bl = (real_t*)malloc(sizeof(real_t) * c->n_types * (c->lmax + 1));
  for (int t = 0; t < c->n_types; ++t) {
    real_t R = c->radius[t];
    for (int l = 0; l <= c->lmax; ++l) {
      const double* rd = c->radial + ((size_t)t * (c->lmax + 1) + l) * 4;
      real_t u = rd[0], up = rd[1], ud = rd[2], udp = rd[3];
      real_t j = jl(l, kabs * R), dj = kabs * jl_deriv(l, kabs * R);
      real_t D = u * udp - up * ud;
      al[t * (c->lmax + 1) + l] = (j * udp - dj * ud) / D;
      bl[t * (c->lmax + 1) + l] = (u * dj - up * j) / D;
    }
  }
  real_t pref = 4 * PI_L / sqrtl(c->volume);
  for (int a = 0; a < c->n_atoms; ++a) {
    int t = c->type[a];
    real_t arg = q[0] * c->pos[3 * a] + q[1] * c->pos[3 * a + 1] + q[2] * c->pos[3 * a + 2];
    arg -= floorl(arg);
    cplx_t phase = cosl(2 * PI_L * arg) + I * sinl(2 * PI_L * arg);
    for (int l = 0; l <= c->lmax; ++l) {
      cplx_t il = (l % 4 == 0) ? 1 : (l % 4 == 1) ? I : (l % 4 == 2) ? -1 : -I;
      for (int m = -l; m <= l; ++m) {
        int L = l * l + l + m;
        cplx_t f = pref * phase * il * conjl(Y[L]);
        A[(size_t)a * nl + L] = f * al[t * (c->lmax + 1) + l];
        B[(size_t)a * nl + L] = f * bl[t * (c->lmax + 1) + l];
      }
    }
  }
  free(Y);
  free(al);
  free(bl);
}

/* A, B for the plane waves n3[g_idx[i]], i < n_sel.
 * Output layout [n_atoms][N_L][n_sel] complex interleaved (re, im). */
int oracle_build_ab(const double lat[9], int n_atoms, const double* pos, const int* type,
                    int n_types, const double* radius, int lmax, const double k[3],
                    const double* radial, const int* n3, int n_sel, const int* g_idx,
                    double* A_out, double* B_out) {
  ab_ctx_t c;
  ab_ctx_init(&c, lat, n_atoms, pos, type, n_types, radius, lmax, k, radial);
  int nl = (lmax + 1) * (lmax + 1);
#pragma omp parallel
  {
    cplx_t* A = (cplx_t*)malloc(sizeof(cplx_t) * n_atoms * nl);
    cplx_t* B = (cplx_t*)malloc(sizeof(cplx_t) * n_atoms * nl);
#pragma omp for schedule(dynamic, 4)
    for (int i = 0; i < n_sel; ++i) {
      ab_one(&c, n3 + 3 * g_idx[i], A, B);
      for (int a = 0; a < n_atoms; ++a)
        for (int L = 0; L < nl; ++L) {
          size_t o = (((size_t)a * nl + L) * n_sel + i) * 2;
          A_out[o] = (double)creall(A[(size_t)a * nl + L]);
          A_out[o + 1] = (double)cimagl(A[(size_t)a * nl + L]);
          B_out[o] = (double)creall(B[(size_t)a * nl + L]);
          B_out[o + 1] = (double)cimagl(B[(size_t)a * nl + L]);
        }
    }
    free(A);
    free(B);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* H and S, column by column                                           */
/* ------------------------------------------------------------------ */

/* Columns cols[c] of H and S (Eqs. (def_hamilton), (def_overlap)).
 * Output H_out[c][G'] = H_{G', cols[c]} for all G' < n_g, complex interleaved.
 * T is [n_slots][2N_L][2N_L] complex row-major; U is [n_types][lmax+1].
 * For each column G: y_a = T_{slot(a)} [A_a; B_a](G) and
 * s_a = [A_a(G); ||udot||^2 B_a(G)]; then for every row G':
 *   H_{G'G} = sum_a [A_a; B_a](G')^H y_a,  S_{G'G} = sum_a [A_a; B_a](G')^H s_a. */
int oracle_hs_columns(const double lat[9], int n_atoms, const double* pos, const int* type,
                      int n_types, const double* radius, int lmax, const double k[3],
                      const double* radial, const double* U, const double* T,
                      const int* atom_slot, int n_g, const int* n3, int n_cols,
                      const int* cols, double* H_out, double* S_out) {
  ab_ctx_t c;
  ab_ctx_init(&c, lat, n_atoms, pos, type, n_types, radius, lmax, k, radial);
  int nl = (lmax + 1) * (lmax + 1);
  int n2 = 2 * nl;
  const double _Complex* Tc = (const double _Complex*)T;
  double _Complex* y = (double _Complex*)malloc(sizeof(double _Complex) * (size_t)n_cols * n_atoms * n2);
  double _Complex* s = (double _Complex*)malloc(sizeof(double _Complex) * (size_t)n_cols * n_atoms * n2);
  if (!y || !s) return -1;
#pragma omp parallel
  {
    cplx_t* A = (cplx_t*)malloc(sizeof(cplx_t) * n_atoms * nl);
    cplx_t* B = (cplx_t*)malloc(sizeof(cplx_t) * n_atoms * nl);
    double _Complex* w = (double _Complex*)malloc(sizeof(double _Complex) * n2);
#pragma omp for schedule(dynamic, 1)
    for (int ci = 0; ci < n_cols; ++ci) {
      ab_one(&c, n3 + 3 * cols[ci], A, B);
      for (int a = 0; a < n_atoms; ++a) {
        int t = type[a];
        const double _Complex* Ta = Tc + (size_t)atom_slot[a] * n2 * n2;
        for (int L = 0; L < nl; ++L) {
          w[L] = (double _Complex)A[(size_t)a * nl + L];
          w[nl + L] = (double _Complex)B[(size_t)a * nl + L];
        }
        double _Complex* ya = y + ((size_t)ci * n_atoms + a) * n2;
        double _Complex* sa = s + ((size_t)ci * n_atoms + a) * n2;
        for (int i = 0; i < n2; ++i) {
          double _Complex acc = 0;
          for (int j = 0; j < n2; ++j) acc += Ta[(size_t)i * n2 + j] * w[j];
          ya[i] = acc;
        }
        for (int l = 0; l <= lmax; ++l) {
          double u2 = U[t * (lmax + 1) + l] * U[t * (lmax + 1) + l];
          for (int m = -l; m <= l; ++m) {
            int L = l * l + l + m;
            sa[L] = w[L];
            sa[nl + L] = u2 * w[nl + L];
          }
        }
      }
    }
#pragma omp for schedule(dynamic, 8)
    for (int gp = 0; gp < n_g; ++gp) {
      ab_one(&c, n3 + 3 * gp, A, B);
      for (int ci = 0; ci < n_cols; ++ci) {
        double _Complex h = 0, sv = 0;
        for (int a = 0; a < n_atoms; ++a) {
          const double _Complex* ya = y + ((size_t)ci * n_atoms + a) * n2;
          const double _Complex* sa = s + ((size_t)ci * n_atoms + a) * n2;
          for (int L = 0; L < nl; ++L) {
            double _Complex ca = conj((double _Complex)A[(size_t)a * nl + L]);
            double _Complex cb = conj((double _Complex)B[(size_t)a * nl + L]);
            h += ca * ya[L] + cb * ya[nl + L];
            sv += ca * sa[L] + cb * sa[nl + L];
          }
        }
        size_t o = ((size_t)ci * n_g + gp) * 2;
        H_out[o] = creal(h);
        H_out[o + 1] = cimag(h);
        S_out[o] = creal(sv);
        S_out[o + 1] = cimag(sv);
      }
    }
    free(A);
    free(B);
    free(w);
  }
  free(y);
  free(s);
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
