// Plain FP64 lower-triangle contraction  X = Z^H diag(sigma) Z  (Sec. 3: the
// zherk / zher2k calls of Alg. 1 and Alg. 3 collapse to this one Hermitian
// rank-K update once T is factorised).  The baseline path the emulated one is
// measured against.  Output columns read the operand rows from Prob::col_base,
// so the same kernel also computes Alg. 3's L^H R (L != R, Hermitian result).
//
// 64 x 64 complex output tiles (lower-triangle tiles only), 8 warps, each warp
// 32 x 16 outputs on FP64 tensor cores (mma.sync m8n8k4 f64, DMMA).  With
// Z = Zr + i Zi:  Re X = Zr'^T Zr + Zi'^T Zi,  Im X = Zr'^T Zi - Zi'^T Zr,
// four real MMAs per complex k-step.  Rows with sigma = -1 enter with their
// right-hand copy negated (exact).
#include "flapw_internal.h"

namespace flapw {
namespace {

constexpr int kTM = 64, kTN = 64, kKC = 16;  // tile and K chunk (complex)
constexpr int kLd = 20;                      // padded row (doubles): conflict-free fragments

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256) herk_f64_kernel(const double2* __restrict__ Z, int64_t k_alloc,
                                                       const Prob* __restrict__ probs,
                                                       const F64Tile* __restrict__ tiles) {
  __shared__ double ar[kTM][kLd], ai[kTM][kLd], br[kTN][kLd], bi[kTN][kLd];
  const F64Tile t = tiles[blockIdx.x];
  const Prob P = probs[t.prob];
  const int row0 = t.ib * kTM, col0 = t.jb * kTN;
  const int kp = P.kp, kn = P.kn;
  const int kp_pad = neg_base(kp);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps: 32 rows x 16 cols each
  double cre[4][2][2], cim[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) cre[i][j][0] = cre[i][j][1] = cim[i][j][0] = cim[i][j][1] = 0.0;

  // the two K ranges: [0, kp) with +1, [kp_pad, kp_pad + kn) with -1
  for (int part = 0; part < 2; ++part) {
    const int kbeg = part ? kp_pad : 0;
    const int kend = part ? kp_pad + kn : kp;
    const double sg = part ? -1.0 : 1.0;
    for (int k0 = kbeg; k0 < kend; k0 += kKC) {
      // load 64 rows x 16 complex for each side
      for (int idx = tid; idx < kTM * kKC; idx += 256) {
        const int r = idx / kKC, c = idx % kKC;
        const int kc = k0 + c;
        const int ga = row0 + r, gb = col0 + r;
        double2 za = make_double2(0.0, 0.0), zb = make_double2(0.0, 0.0);
        if (kc < kend) {
          if (ga < P.n_g) za = Z[(int64_t)(P.row_base + ga) * k_alloc + kc];
          if (gb < P.n_g) zb = Z[(int64_t)(P.col_base + gb) * k_alloc + kc];
        }
        ar[r][c] = za.x;
        ai[r][c] = za.y;
        br[r][c] = sg * zb.x;
        bi[r][c] = sg * zb.y;
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < kKC; ks += 4) {
        const int kk = ks + (lane & 3);
        double xr[4], xi[4], yr[2], yi[2];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = wm * 32 + i * 8 + (lane >> 2);
          xr[i] = ar[r][kk];
          xi[i] = ai[r][kk];
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r = wn * 16 + j * 8 + (lane >> 2);
          yr[j] = br[r][kk];
          yi[j] = bi[r][kk];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            dmma(cre[i][j][0], cre[i][j][1], xr[i], yr[j]);
            dmma(cre[i][j][0], cre[i][j][1], xi[i], yi[j]);
            dmma(cim[i][j][0], cim[i][j][1], xr[i], yi[j]);
            dmma(cim[i][j][0], cim[i][j][1], -xi[i], yr[j]);
          }
      }
      __syncthreads();
    }
  }
  // store the lower triangle
  const int64_t ng = P.n_g;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t gr = row0 + wm * 32 + i * 8 + (lane >> 2);
        const int64_t gc = col0 + wn * 16 + j * 8 + 2 * (lane & 3) + h;
        if (gr < ng && gc < ng && gr >= gc) {
          const int64_t o = (P.layout == FLAPW_LAYOUT_LOWER_PACKED)
                                ? gc * ng - gc * (gc - 1) / 2 + (gr - gc)
                                : gc * P.ld + gr;
          P.out[o] = make_double2(cre[i][j][h], cim[i][j][h]);
        }
      }
}

}  // namespace

cudaError_t launch_herk_f64(const double2* Z, int64_t k_alloc, const Prob* probs,
                            const F64Tile* tiles, int n_tiles, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  herk_f64_kernel<<<n_tiles, 256, 0, st>>>(Z, k_alloc, probs, tiles);
  return cudaGetLastError();
}

}  // namespace flapw
