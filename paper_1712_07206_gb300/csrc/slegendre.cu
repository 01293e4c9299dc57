// Overlap matrix by the addition theorem (an alternative to the S contraction
// for the library's own matching coefficients).
//
// With A_{aLG} = e^{iK.tau_a} Yc_L(K) a_{t,l}(|K|), Yc_L = (4 pi / sqrt(Omega))
// i^l conj(Y_lm(Khat)) (the Rayleigh matching of Sec. 2), the sum over m in
// S_{G'G} = sum_a sum_L conj(A_{aLG'}) A_{aLG} + U_{tl}^2 conj(B_{aLG'}) B_{aLG}
// (Eq. (def_overlap)) collapses by sum_m Y_lm(u) conj(Y_lm(v)) = (2l+1)/(4 pi)
// P_l(u.v):
//     S_{G'G} = (4 pi / Omega) sum_t rho_t(G', G) sum_l (2l+1) P_l(Khat'.Khat)
//               [a_l(K') a_l(K) + U_l^2 b_l(K') b_l(K)],
//     rho_t(G', G) = sum_{atoms a of type t} conj(e^{iK'.tau_a}) e^{iK.tau_a}.
// It removes the factor N_L of the contraction: one of the compressions of A
// and B by mathematical identities that the Conclusions point to.  Per
// element it costs N_A complex multiply-adds for the structure factors and
// (l_max + 1) per type for the Legendre sum, against 8 N_A N_L for the
// contraction.
//
// The Legendre recurrence P_{l+1} = ((2l+1) x P_l - l P_{l-1}) / (l+1) and the
// phase sums need more than FP32: the FP64 path evaluates them in FP64, the
// emulated path in double-float arithmetic on the FP32 pipes (dfloat.cuh; a
// pre-pass splits the inputs into FP32 pairs), which GB300 issues 64 times
// faster than FP64.  CTA tile: 64 x 64 of the lower triangle (the FP64
// contraction's tile list), 256 threads with a 4 x 4 block each; per type the
// atoms' phases stream through shared memory 8 at a time.
#include "dfloat.cuh"
#include "flapw_internal.h"

namespace flapw {
namespace {

constexpr int kT = 64;
constexpr int kChunkAtoms = 8;  // keeps the static shared memory under 48 KB
constexpr int kL1 = kMaxLmax + 1;

// Khat of every plane wave (z for K = 0), the K of ab_prep.
__global__ void __launch_bounds__(128) khat_kernel(Geom geo, GData gd, double* khat) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= geo.g_total) return;
  const int k = gd.gk[gi];
  const double q0 = gd.n3[3 * gi] + geo.kfrac[3 * k], q1 = gd.n3[3 * gi + 1] + geo.kfrac[3 * k + 1],
               q2 = gd.n3[3 * gi + 2] + geo.kfrac[3 * k + 2];
  double K[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) K[c] = q0 * geo.rec[c] + q1 * geo.rec[3 + c] + q2 * geo.rec[6 + c];
  const double kabs = sqrt(K[0] * K[0] + K[1] * K[1] + K[2] * K[2]);
  double* o = khat + 3 * gi;
  if (kabs > 0) {
    o[0] = K[0] / kabs;
    o[1] = K[1] / kabs;
    o[2] = K[2] / kabs;
  } else {
    o[0] = 0.0;
    o[1] = 0.0;
    o[2] = 1.0;
  }
}

__global__ void __launch_bounds__(256) slegendre_kernel(SLegArgs a, const F64Tile* __restrict__ tiles) {
  __shared__ double kh[2][kT][3];          // [0] rows G', [1] columns G
  __shared__ double rad[4][kL1][kT];        // a_l rows, U^2 b_l rows, a_l cols, b_l cols
  __shared__ double2 phs[2][kChunkAtoms][kT];
  __shared__ double rec_ab[kL1][2];  // P_{l+1} = alpha_l x P_l - beta_l P_{l-1}
  const F64Tile T = tiles[blockIdx.x];
  const Prob P = a.probs[T.prob];
  const int64_t ng = P.n_g;
  const int64_t g0 = P.row_base - a.s_row0;  // global plane wave of the problem's first row
  const int r0 = T.ib * kT, c0 = T.jb * kT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int L1 = a.lmax + 1;
  const int64_t G = a.g_total;
  if (tid < kL1) {
    rec_ab[tid][0] = (double)(2 * tid + 1) / (double)(tid + 1);
    rec_ab[tid][1] = (double)tid / (double)(tid + 1);
  }
  for (int i = tid; i < 2 * kT * 3; i += 256) {
    const int w = i / (kT * 3), e = i % (kT * 3), g = e / 3, c = e % 3;
    const int64_t gl = (w == 0 ? r0 : c0) + g;
    kh[w][g][c] = (gl < ng) ? a.khat[3 * (g0 + gl) + c] : 0.0;
  }
  double2 S[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) S[i][j] = make_double2(0.0, 0.0);

  for (int t = 0; t < a.n_types; ++t) {
    __syncthreads();
    for (int i = tid; i < 4 * L1 * kT; i += 256) {
      const int w = i / (L1 * kT), e = i % (L1 * kT), l = e / kT, g = e % kT;
      const int64_t gl = ((w < 2) ? r0 : c0) + g;
      double v = 0.0;
      if (gl < ng) {
        // rows carry the factor 2l + 1, and U^2 on b_l
        const int64_t ro = ((int64_t)t * L1 + l) * G + g0 + gl;
        const double u = a.U[t * L1 + l];
        if (w == 0) v = (2 * l + 1) * a.al[ro];
        else if (w == 1) v = (2 * l + 1) * u * u * a.bl[ro];
        else if (w == 2) v = a.al[ro];
        else v = a.bl[ro];
      }
      rad[w][l][g] = v;
    }
    // rho_t for this thread's 4 x 4 block
    double2 rho[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) rho[i][j] = make_double2(0.0, 0.0);
    const int a0 = a.type_start[t], a1 = a.type_start[t + 1];
    for (int ab = a0; ab < a1; ab += kChunkAtoms) {
      const int na = min(kChunkAtoms, a1 - ab);
      __syncthreads();
      for (int i = tid; i < 2 * kChunkAtoms * kT; i += 256) {
        const int w = i / (kChunkAtoms * kT), e = i % (kChunkAtoms * kT), q = e / kT, g = e % kT;
        const int64_t gl = (w == 0 ? r0 : c0) + g;
        double2 v = make_double2(0.0, 0.0);
        if (q < na && gl < ng) v = a.ph[(int64_t)a.type_atoms[ab + q] * G + g0 + gl];
        phs[w][q][g] = v;
      }
      __syncthreads();
      for (int q = 0; q < na; ++q) {
        double2 pr[4], pc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          pr[i] = phs[0][q][ty * 4 + i];
          pc[i] = phs[1][q][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {  // conj(pr) pc
            rho[i][j].x = fma(pr[i].x, pc[j].x, fma(pr[i].y, pc[j].y, rho[i][j].x));
            rho[i][j].y = fma(pr[i].x, pc[j].y, fma(-pr[i].y, pc[j].x, rho[i][j].y));
          }
      }
    }
    __syncthreads();
    // Legendre sum of type t, times rho_t
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ri = ty * 4 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cj = tx * 4 + j;
        const double x = kh[0][ri][0] * kh[1][cj][0] + kh[0][ri][1] * kh[1][cj][1] + kh[0][ri][2] * kh[1][cj][2];
        double pm = 1.0, p = x;  // P_{l-1}, P_l from l = 1
        double Lt = fma(rad[0][0][ri], rad[2][0][cj], rad[1][0][ri] * rad[3][0][cj]);
        for (int l = 1; l < L1; ++l) {
          Lt = fma(p, fma(rad[0][l][ri], rad[2][l][cj], rad[1][l][ri] * rad[3][l][cj]), Lt);
          const double pn = fma(rec_ab[l][0] * x, p, -rec_ab[l][1] * pm);
          pm = p;
          p = pn;
        }
        S[i][j].x = fma(rho[i][j].x, Lt, S[i][j].x);
        S[i][j].y = fma(rho[i][j].y, Lt, S[i][j].y);
      }
    }
  }
  // lower triangle of the problem, scaled by 4 pi / Omega
  double* outd = reinterpret_cast<double*>(P.out);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = r0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = c0 + tx * 4 + j;
      if (gr < ng && gc <= gr) {
        const int64_t o = (P.layout == FLAPW_LAYOUT_LOWER_PACKED) ? gc * ng - gc * (gc - 1) / 2 + (gr - gc)
                                                                   : gc * P.ld + gr;
        outd[2 * o] = a.scale * S[i][j].x;
        outd[2 * o + 1] = a.scale * S[i][j].y;
      }
    }
  }
}

// Double-float copies of the Legendre kernels' inputs for plane wave gi:
// rows (2l+1) a_l and (2l+1) U^2 b_l (U = null: (2l+1) b_l, for H), columns
// a_l and b_l ([4][t][l][G]), phases ([atom][G] as Re, Im pairs) and Khat
// ([G][3]).
__device__ void split_inputs(int64_t gi, int64_t G, int L1, int n_types, int n_atoms, const double* U,
                             const double* al_, const double* bl_, const double2* ph_, const double* khat,
                             float2* rad) {
  const int64_t nr = (int64_t)n_types * L1 * G;
  float2* ph = rad + 4 * nr;
  float2* kh = ph + 2 * (int64_t)n_atoms * G;
  for (int t = 0; t < n_types; ++t)
    for (int l = 0; l < L1; ++l) {
      const int64_t ro = ((int64_t)t * L1 + l) * G + gi;
      const double u = U ? U[t * L1 + l] : 1.0, al = al_[ro], bl = bl_[ro];
      rad[ro] = dfl::split((2 * l + 1) * al);
      rad[nr + ro] = dfl::split((2 * l + 1) * u * u * bl);
      rad[2 * nr + ro] = dfl::split(al);
      rad[3 * nr + ro] = dfl::split(bl);
    }
  for (int at = 0; at < n_atoms; ++at) {
    const double2 v = ph_[(int64_t)at * G + gi];
    ph[2 * ((int64_t)at * G + gi)] = dfl::split(v.x);
    ph[2 * ((int64_t)at * G + gi) + 1] = dfl::split(v.y);
  }
  for (int c = 0; c < 3; ++c) kh[3 * gi + c] = dfl::split(khat[3 * gi + c]);
}

// One thread per plane wave.
__global__ void __launch_bounds__(128) slegendre_split_kernel(SLegArgs a) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.g_total) return;
  split_inputs(gi, a.g_total, a.lmax + 1, a.n_types, a.n_atoms, a.U, a.al, a.bl, a.ph, a.khat, a.dfw);
}

__global__ void __launch_bounds__(128) hlegendre_split_kernel(HLegArgs a) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.g_total) return;
  split_inputs(gi, a.g_total, a.lmax + 1, a.n_types, a.n_atoms, nullptr, a.al, a.bl, a.ph, a.khat, a.dfw);
}

// slegendre_kernel in double-float: 512 threads of 2 x 4 elements (the double-float
// accumulators of 4 x 4 per thread allowed one CTA of 8 warps per SM).
constexpr int kDfRows = 2, kDfCols = 4;
constexpr int kDfThreads = (kT / kDfRows) * (kT / kDfCols);
__global__ void __launch_bounds__(kDfThreads) slegendre_df_kernel(SLegArgs a, const F64Tile* __restrict__ tiles) {
  using dfl::df;
  __shared__ float2 kh[2][kT][3];
  __shared__ float2 rad[4][kL1][kT];
  __shared__ float4 phs[2][kChunkAtoms][kT];
  __shared__ float2 rec_ab[kL1][2];
  const F64Tile T = tiles[blockIdx.x];
  const Prob P = a.probs[T.prob];
  const int64_t ng = P.n_g;
  const int64_t g0 = P.row_base - a.s_row0;
  const int r0 = T.ib * kT, c0 = T.jb * kT;
  const int tid = threadIdx.x, ty = tid / (kT / kDfCols), tx = tid % (kT / kDfCols);
  const int L1 = a.lmax + 1;
  const int64_t G = a.g_total;
  const int64_t nr = (int64_t)a.n_types * L1 * G;
  const float2* radg = a.dfw;
  const float4* phg = reinterpret_cast<const float4*>(a.dfw + 4 * nr);
  const float2* khg = a.dfw + 4 * nr + 2 * (int64_t)a.n_atoms * G;
  const float2 zero2 = make_float2(0.f, 0.f);
  if (tid < kL1) {
    rec_ab[tid][0] = dfl::split((double)(2 * tid + 1) / (double)(tid + 1));
    rec_ab[tid][1] = dfl::split((double)tid / (double)(tid + 1));
  }
  for (int i = tid; i < 2 * kT * 3; i += kDfThreads) {
    const int w = i / (kT * 3), e = i % (kT * 3), g = e / 3, c = e % 3;
    const int64_t gl = (w == 0 ? r0 : c0) + g;
    kh[w][g][c] = (gl < ng) ? khg[3 * (g0 + gl) + c] : zero2;
  }
  df Sr[kDfRows][kDfCols], Si[kDfRows][kDfCols];
#pragma unroll
  for (int i = 0; i < kDfRows; ++i)
#pragma unroll
    for (int j = 0; j < kDfCols; ++j) Sr[i][j] = Si[i][j] = df{0.f, 0.f};

  for (int t = 0; t < a.n_types; ++t) {
    __syncthreads();
    for (int i = tid; i < 4 * L1 * kT; i += kDfThreads) {
      const int w = i / (L1 * kT), e = i % (L1 * kT), l = e / kT, g = e % kT;
      const int64_t gl = ((w < 2) ? r0 : c0) + g;
      rad[w][l][g] = (gl < ng) ? radg[w * nr + ((int64_t)t * L1 + l) * G + g0 + gl] : zero2;
    }
    df rr[kDfRows][kDfCols], ri[kDfRows][kDfCols];  // rho_t
#pragma unroll
    for (int i = 0; i < kDfRows; ++i)
#pragma unroll
      for (int j = 0; j < kDfCols; ++j) rr[i][j] = ri[i][j] = df{0.f, 0.f};
    const int a0 = a.type_start[t], a1 = a.type_start[t + 1];
    for (int ab = a0; ab < a1; ab += kChunkAtoms) {
      const int na = min(kChunkAtoms, a1 - ab);
      __syncthreads();
      for (int i = tid; i < 2 * kChunkAtoms * kT; i += kDfThreads) {
        const int w = i / (kChunkAtoms * kT), e = i % (kChunkAtoms * kT), q = e / kT, g = e % kT;
        const int64_t gl = (w == 0 ? r0 : c0) + g;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < na && gl < ng) v = phg[(int64_t)a.type_atoms[ab + q] * G + g0 + gl];
        phs[w][q][g] = v;
      }
      __syncthreads();
      for (int q = 0; q < na; ++q) {
        float4 pr[kDfRows], pc[kDfCols];
#pragma unroll
        for (int i = 0; i < kDfRows; ++i) pr[i] = phs[0][q][ty * kDfRows + i];
#pragma unroll
        for (int j = 0; j < kDfCols; ++j) pc[j] = phs[1][q][tx * kDfCols + j];
#pragma unroll
        for (int i = 0; i < kDfRows; ++i) {
          const df ar{pr[i].x, pr[i].y}, ai{pr[i].z, pr[i].w};
#pragma unroll
          for (int j = 0; j < kDfCols; ++j) {  // conj(pr) pc
            const df br{pc[j].x, pc[j].y}, bi{pc[j].z, pc[j].w};
            rr[i][j] = dfl::fma(ar, br, dfl::fma(ai, bi, rr[i][j]));
            ri[i][j] = dfl::fma(ar, bi, dfl::fma(dfl::neg(ai), br, ri[i][j]));
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kDfRows; ++i) {
      const int rw = ty * kDfRows + i;
#pragma unroll
      for (int j = 0; j < kDfCols; ++j) {
        const int cl = tx * kDfCols + j;
        const df x = dfl::fma(dfl::make(kh[0][rw][0]), dfl::make(kh[1][cl][0]),
                              dfl::fma(dfl::make(kh[0][rw][1]), dfl::make(kh[1][cl][1]),
                                       dfl::mul(dfl::make(kh[0][rw][2]), dfl::make(kh[1][cl][2]))));
        df pm{1.f, 0.f}, p = x;
        df Lt = dfl::fma(dfl::make(rad[0][0][rw]), dfl::make(rad[2][0][cl]),
                         dfl::mul(dfl::make(rad[1][0][rw]), dfl::make(rad[3][0][cl])));
        for (int l = 1; l < L1; ++l) {
          const df c = dfl::fma(dfl::make(rad[0][l][rw]), dfl::make(rad[2][l][cl]),
                                dfl::mul(dfl::make(rad[1][l][rw]), dfl::make(rad[3][l][cl])));
          Lt = dfl::fma(p, c, Lt);
          const df pn = dfl::fma(dfl::mul(dfl::make(rec_ab[l][0]), x), p,
                                 dfl::neg(dfl::mul(dfl::make(rec_ab[l][1]), pm)));
          pm = p;
          p = pn;
        }
        Sr[i][j] = dfl::fma(rr[i][j], Lt, Sr[i][j]);
        Si[i][j] = dfl::fma(ri[i][j], Lt, Si[i][j]);
      }
    }
  }
  double* outd = reinterpret_cast<double*>(P.out);
#pragma unroll
  for (int i = 0; i < kDfRows; ++i) {
    const int64_t gr = r0 + ty * kDfRows + i;
#pragma unroll
    for (int j = 0; j < kDfCols; ++j) {
      const int64_t gc = c0 + tx * kDfCols + j;
      if (gr < ng && gc <= gr) {
        const int64_t o = (P.layout == FLAPW_LAYOUT_LOWER_PACKED) ? gc * ng - gc * (gc - 1) / 2 + (gr - gc)
                                                                   : gc * P.ld + gr;
        outd[2 * o] = a.scale * dfl::to_double(Sr[i][j]);
        outd[2 * o + 1] = a.scale * dfl::to_double(Si[i][j]);
      }
    }
  }
}

// The spherical part of H by the addition theorem (FLAPW_H_SPHERICAL): for
// T^{XY}_{L'L} = t^{XY}_l delta_{L'L} per slot, Eq. (def_hamilton) with the
// library's matching coefficients collapses like S:
//   H_{G'G} = (4 pi / Omega) sum_c rho_c(G', G) sum_l (2l+1) P_l(Khat'.Khat)
//             [t^AA a'a + t^BB b'b + Re t^BA (a'b + b'a) + i Im t^BA (b'a - a'b)]_l
// with a' = a_l(K'), a = a_l(K) (b likewise) of the combination's type, t of
// its slot (t^AB = conj t^BA: T is Hermitian), rho_c the phase sum over the
// atoms of the (slot, type) combination c.  FP64 on the FP64 path, double-float
// (hlegendre_df_kernel) on the emulated path.  add: the result
// is added to the lower triangle already in P.out (the contraction of the
// rest of T), otherwise written.
__global__ void __launch_bounds__(256) hlegendre_kernel(HLegArgs a, const F64Tile* __restrict__ tiles,
                                                        int add) {
  __shared__ double kh[2][kT][3];
  __shared__ double rad[4][kL1][kT];  // (2l+1) a_l, (2l+1) b_l rows; a_l, b_l columns
  __shared__ double2 phs[2][kChunkAtoms][kT];
  __shared__ double coef[kL1][4];     // t^AA, t^BB, Re t^BA, Im t^BA of the slot
  __shared__ double rec_ab[kL1][2];
  const F64Tile T = tiles[blockIdx.x];
  const Prob P = a.probs[T.prob];
  const int64_t ng = P.n_g;
  const int64_t g0 = P.row_base - a.h_row0;  // global plane wave of the problem's first row
  const int r0 = T.ib * kT, c0 = T.jb * kT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int L1 = a.lmax + 1;
  const int64_t G = a.g_total;
  if (tid < kL1) {
    rec_ab[tid][0] = (double)(2 * tid + 1) / (double)(tid + 1);
    rec_ab[tid][1] = (double)tid / (double)(tid + 1);
  }
  for (int i = tid; i < 2 * kT * 3; i += 256) {
    const int w = i / (kT * 3), e = i % (kT * 3), g = e / 3, c = e % 3;
    const int64_t gl = (w == 0 ? r0 : c0) + g;
    kh[w][g][c] = (gl < ng) ? a.khat[3 * (g0 + gl) + c] : 0.0;
  }
  double2 Hs[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Hs[i][j] = make_double2(0.0, 0.0);

  for (int cb = 0; cb < a.n_combo; ++cb) {
    const int t = a.combo_type[cb], sl = a.combo_slot[cb];
    __syncthreads();
    for (int i = tid; i < 4 * L1 * kT; i += 256) {
      const int w = i / (L1 * kT), e = i % (L1 * kT), l = e / kT, g = e % kT;
      const int64_t gl = ((w < 2) ? r0 : c0) + g;
      double v = 0.0;
      if (gl < ng) {
        const int64_t ro = ((int64_t)t * L1 + l) * G + g0 + gl;
        const double x = (w == 0 || w == 2) ? a.al[ro] : a.bl[ro];
        v = (w < 2) ? (2 * l + 1) * x : x;
      }
      rad[w][l][g] = v;
    }
    if (tid < 4 * L1) coef[tid >> 2][tid & 3] = a.tsph[((int64_t)sl * L1 + (tid >> 2)) * 4 + (tid & 3)];
    double2 rho[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) rho[i][j] = make_double2(0.0, 0.0);
    const int a0 = a.combo_start[cb], a1 = a.combo_start[cb + 1];
    for (int ab = a0; ab < a1; ab += kChunkAtoms) {
      const int na = min(kChunkAtoms, a1 - ab);
      __syncthreads();
      for (int i = tid; i < 2 * kChunkAtoms * kT; i += 256) {
        const int w = i / (kChunkAtoms * kT), e = i % (kChunkAtoms * kT), q = e / kT, g = e % kT;
        const int64_t gl = (w == 0 ? r0 : c0) + g;
        double2 v = make_double2(0.0, 0.0);
        if (q < na && gl < ng) v = a.ph[(int64_t)a.combo_atoms[ab + q] * G + g0 + gl];
        phs[w][q][g] = v;
      }
      __syncthreads();
      for (int q = 0; q < na; ++q) {
        double2 pr[4], pc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          pr[i] = phs[0][q][ty * 4 + i];
          pc[i] = phs[1][q][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {  // conj(pr) pc
            rho[i][j].x = fma(pr[i].x, pc[j].x, fma(pr[i].y, pc[j].y, rho[i][j].x));
            rho[i][j].y = fma(pr[i].x, pc[j].y, fma(-pr[i].y, pc[j].x, rho[i][j].y));
          }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ri = ty * 4 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cj = tx * 4 + j;
        const double x = kh[0][ri][0] * kh[1][cj][0] + kh[0][ri][1] * kh[1][cj][1] + kh[0][ri][2] * kh[1][cj][2];
        double pm = 1.0, p = x;  // P_{l-1}, P_l from l = 1
        double Lr = 0.0, Li = 0.0;
        for (int l = 0; l < L1; ++l) {
          const double pl = (l == 0) ? 1.0 : p;
          const double aa = rad[0][l][ri] * rad[2][l][cj], bb = rad[1][l][ri] * rad[3][l][cj];
          const double ab_ = rad[0][l][ri] * rad[3][l][cj], ba = rad[1][l][ri] * rad[2][l][cj];
          const double wr = fma(coef[l][0], aa, fma(coef[l][1], bb, coef[l][2] * (ab_ + ba)));
          const double wi = coef[l][3] * (ba - ab_);
          Lr = fma(pl, wr, Lr);
          Li = fma(pl, wi, Li);
          if (l >= 1) {
            const double pn = fma(rec_ab[l][0] * x, p, -rec_ab[l][1] * pm);
            pm = p;
            p = pn;
          }
        }
        // rho_c x L_c, complex
        Hs[i][j].x = fma(rho[i][j].x, Lr, fma(-rho[i][j].y, Li, Hs[i][j].x));
        Hs[i][j].y = fma(rho[i][j].x, Li, fma(rho[i][j].y, Lr, Hs[i][j].y));
      }
    }
  }
  double* outd = reinterpret_cast<double*>(P.out);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = r0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = c0 + tx * 4 + j;
      if (gr < ng && gc <= gr) {
        const int64_t o = (P.layout == FLAPW_LAYOUT_LOWER_PACKED) ? gc * ng - gc * (gc - 1) / 2 + (gr - gc)
                                                                   : gc * P.ld + gr;
        const double re = a.scale * Hs[i][j].x, im = a.scale * Hs[i][j].y;
        if (add) {
          outd[2 * o] += re;
          outd[2 * o + 1] += im;
        } else {
          outd[2 * o] = re;
          outd[2 * o + 1] = im;
        }
      }
    }
  }
}

// hlegendre_kernel in double-float (the emulated path): the layout of
// slegendre_df_kernel, 512 threads of 2 x 4 elements, with the complex
// Legendre weight of the (slot, type) combinations.
__global__ void __launch_bounds__(kDfThreads) hlegendre_df_kernel(HLegArgs a, const F64Tile* __restrict__ tiles,
                                                                  int add) {
  using dfl::df;
  __shared__ float2 kh[2][kT][3];
  __shared__ float2 rad[4][kL1][kT];
  __shared__ float4 phs[2][kChunkAtoms][kT];
  __shared__ float2 coef[kL1][4];
  __shared__ float2 rec_ab[kL1][2];
  const F64Tile T = tiles[blockIdx.x];
  const Prob P = a.probs[T.prob];
  const int64_t ng = P.n_g;
  const int64_t g0 = P.row_base - a.h_row0;
  const int r0 = T.ib * kT, c0 = T.jb * kT;
  const int tid = threadIdx.x, ty = tid / (kT / kDfCols), tx = tid % (kT / kDfCols);
  const int L1 = a.lmax + 1;
  const int64_t G = a.g_total;
  const int64_t nr = (int64_t)a.n_types * L1 * G;
  const float2* radg = a.dfw;
  const float4* phg = reinterpret_cast<const float4*>(a.dfw + 4 * nr);
  const float2* khg = a.dfw + 4 * nr + 2 * (int64_t)a.n_atoms * G;
  const float2 zero2 = make_float2(0.f, 0.f);
  if (tid < kL1) {
    rec_ab[tid][0] = dfl::split((double)(2 * tid + 1) / (double)(tid + 1));
    rec_ab[tid][1] = dfl::split((double)tid / (double)(tid + 1));
  }
  for (int i = tid; i < 2 * kT * 3; i += kDfThreads) {
    const int w = i / (kT * 3), e = i % (kT * 3), g = e / 3, c = e % 3;
    const int64_t gl = (w == 0 ? r0 : c0) + g;
    kh[w][g][c] = (gl < ng) ? khg[3 * (g0 + gl) + c] : zero2;
  }
  df Hr[kDfRows][kDfCols], Hi[kDfRows][kDfCols];
#pragma unroll
  for (int i = 0; i < kDfRows; ++i)
#pragma unroll
    for (int j = 0; j < kDfCols; ++j) Hr[i][j] = Hi[i][j] = df{0.f, 0.f};

  for (int cb = 0; cb < a.n_combo; ++cb) {
    const int t = a.combo_type[cb], sl = a.combo_slot[cb];
    __syncthreads();
    for (int i = tid; i < 4 * L1 * kT; i += kDfThreads) {
      const int w = i / (L1 * kT), e = i % (L1 * kT), l = e / kT, g = e % kT;
      const int64_t gl = ((w < 2) ? r0 : c0) + g;
      rad[w][l][g] = (gl < ng) ? radg[w * nr + ((int64_t)t * L1 + l) * G + g0 + gl] : zero2;
    }
    if (tid < 4 * L1) coef[tid >> 2][tid & 3] = dfl::split(a.tsph[((int64_t)sl * L1 + (tid >> 2)) * 4 + (tid & 3)]);
    df rr[kDfRows][kDfCols], ri[kDfRows][kDfCols];  // rho_c
#pragma unroll
    for (int i = 0; i < kDfRows; ++i)
#pragma unroll
      for (int j = 0; j < kDfCols; ++j) rr[i][j] = ri[i][j] = df{0.f, 0.f};
    const int a0 = a.combo_start[cb], a1 = a.combo_start[cb + 1];
    for (int ab = a0; ab < a1; ab += kChunkAtoms) {
      const int na = min(kChunkAtoms, a1 - ab);
      __syncthreads();
      for (int i = tid; i < 2 * kChunkAtoms * kT; i += kDfThreads) {
        const int w = i / (kChunkAtoms * kT), e = i % (kChunkAtoms * kT), q = e / kT, g = e % kT;
        const int64_t gl = (w == 0 ? r0 : c0) + g;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < na && gl < ng) v = phg[(int64_t)a.combo_atoms[ab + q] * G + g0 + gl];
        phs[w][q][g] = v;
      }
      __syncthreads();
      for (int q = 0; q < na; ++q) {
        float4 pr[kDfRows], pc[kDfCols];
#pragma unroll
        for (int i = 0; i < kDfRows; ++i) pr[i] = phs[0][q][ty * kDfRows + i];
#pragma unroll
        for (int j = 0; j < kDfCols; ++j) pc[j] = phs[1][q][tx * kDfCols + j];
#pragma unroll
        for (int i = 0; i < kDfRows; ++i) {
          const df ar{pr[i].x, pr[i].y}, ai{pr[i].z, pr[i].w};
#pragma unroll
          for (int j = 0; j < kDfCols; ++j) {  // conj(pr) pc
            const df br{pc[j].x, pc[j].y}, bi{pc[j].z, pc[j].w};
            rr[i][j] = dfl::fma(ar, br, dfl::fma(ai, bi, rr[i][j]));
            ri[i][j] = dfl::fma(ar, bi, dfl::fma(dfl::neg(ai), br, ri[i][j]));
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kDfRows; ++i) {
      const int rw = ty * kDfRows + i;
#pragma unroll
      for (int j = 0; j < kDfCols; ++j) {
        const int cl = tx * kDfCols + j;
        const df x = dfl::fma(dfl::make(kh[0][rw][0]), dfl::make(kh[1][cl][0]),
                              dfl::fma(dfl::make(kh[0][rw][1]), dfl::make(kh[1][cl][1]),
                                       dfl::mul(dfl::make(kh[0][rw][2]), dfl::make(kh[1][cl][2]))));
        df pm{1.f, 0.f}, p{1.f, 0.f};  // P_{l-1}, P_l
        df Lr{0.f, 0.f}, Li{0.f, 0.f};
        for (int l = 0; l < L1; ++l) {
          if (l == 1) p = x;
          const df ra = dfl::make(rad[0][l][rw]), rb = dfl::make(rad[1][l][rw]);
          const df ca = dfl::make(rad[2][l][cl]), cb_ = dfl::make(rad[3][l][cl]);
          const df ab_ = dfl::mul(ra, cb_), ba = dfl::mul(rb, ca);
          // t^AA a'a + t^BB b'b + Re t^BA (a'b + b'a), and Im t^BA (b'a - a'b)
          const df wr = dfl::fma(dfl::make(coef[l][0]), dfl::mul(ra, ca),
                                 dfl::fma(dfl::make(coef[l][1]), dfl::mul(rb, cb_),
                                          dfl::mul(dfl::make(coef[l][2]), dfl::add(ab_, ba))));
          const df wi = dfl::mul(dfl::make(coef[l][3]), dfl::add(ba, dfl::neg(ab_)));
          Lr = dfl::fma(p, wr, Lr);
          Li = dfl::fma(p, wi, Li);
          if (l >= 1) {
            const df pn = dfl::fma(dfl::mul(dfl::make(rec_ab[l][0]), x), p,
                                   dfl::neg(dfl::mul(dfl::make(rec_ab[l][1]), pm)));
            pm = p;
            p = pn;
          }
        }
        // rho_c x L_c, complex
        Hr[i][j] = dfl::fma(rr[i][j], Lr, dfl::fma(dfl::neg(ri[i][j]), Li, Hr[i][j]));
        Hi[i][j] = dfl::fma(rr[i][j], Li, dfl::fma(ri[i][j], Lr, Hi[i][j]));
      }
    }
  }
  double* outd = reinterpret_cast<double*>(P.out);
#pragma unroll
  for (int i = 0; i < kDfRows; ++i) {
    const int64_t gr = r0 + ty * kDfRows + i;
#pragma unroll
    for (int j = 0; j < kDfCols; ++j) {
      const int64_t gc = c0 + tx * kDfCols + j;
      if (gr < ng && gc <= gr) {
        const int64_t o = (P.layout == FLAPW_LAYOUT_LOWER_PACKED) ? gc * ng - gc * (gc - 1) / 2 + (gr - gc)
                                                                   : gc * P.ld + gr;
        const double re = a.scale * dfl::to_double(Hr[i][j]), im = a.scale * dfl::to_double(Hi[i][j]);
        if (add) {
          outd[2 * o] += re;
          outd[2 * o + 1] += im;
        } else {
          outd[2 * o] = re;
          outd[2 * o + 1] = im;
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_hlegendre(const HLegArgs& a, const F64Tile* tiles, int n_tiles, bool add, cudaStream_t st,
                             bool inputs_ready) {
  if (n_tiles == 0) return cudaSuccess;
  if (a.lmax < 0 || a.lmax > kMaxLmax) return cudaErrorInvalidValue;
  if (a.dfw) {
    if (!inputs_ready) hlegendre_split_kernel<<<(unsigned)((a.g_total + 127) / 128), 128, 0, st>>>(a);
    hlegendre_df_kernel<<<n_tiles, kDfThreads, 0, st>>>(a, tiles, add ? 1 : 0);
  } else {
    hlegendre_kernel<<<n_tiles, 256, 0, st>>>(a, tiles, add ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_khat(const Geom& geo, const GData& gd, double* khat, cudaStream_t st) {
  if (geo.g_total == 0) return cudaSuccess;
  khat_kernel<<<(unsigned)((geo.g_total + 127) / 128), 128, 0, st>>>(geo, gd, khat);
  return cudaGetLastError();
}

size_t slegendre_df_floats2(int n_types, int lmax, int n_atoms, int64_t G) {
  return (size_t)(4 * (int64_t)n_types * (lmax + 1) * G + 2 * (int64_t)n_atoms * G + 3 * G);
}

cudaError_t launch_slegendre(const SLegArgs& a, const F64Tile* tiles, int n_tiles, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  if (a.lmax < 0 || a.lmax > kMaxLmax) return cudaErrorInvalidValue;
  if (a.dfw) {
    slegendre_split_kernel<<<(unsigned)((a.g_total + 127) / 128), 128, 0, st>>>(a);
    slegendre_df_kernel<<<n_tiles, kDfThreads, 0, st>>>(a, tiles);
  } else {
    slegendre_kernel<<<n_tiles, 256, 0, st>>>(a, tiles);
  }
  return cudaGetLastError();
}

}  // namespace flapw
