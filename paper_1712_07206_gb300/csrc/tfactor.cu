// Factorisation of each Hermitian T block (Sec. 3, Alg. 1: the Cholesky
// factorisation of T^AA that turns A^H T A into a Hermitian rank-K update).
//
// The full 2N_L x 2N_L block T = [[T^AA, T^AB],[T^BA, T^BB]] is factorised at
// once, so that  H_a = W_a^H T W_a = (C^H W_a)^H diag(sigma) (C^H W_a),
// W_a = [A_a; B_a].  T is generally indefinite (the paper notes that even
// T^AA's Cholesky "may fail"), so instead of plain Cholesky the kernel runs
// the Bunch-Kaufman diagonal-pivoting LDL^H (1x1 and 2x2 pivots) in FP64:
//     P^T T P = L D L^H,
// splits every 2x2 block of D as Q Lambda Q^H, and returns, in pivoted order,
//     M = |Lambda|^{1/2} Q^H L^H,   sigma = sign(Lambda),
// so that C^H = M P^T: the operand rows are M times the W rows gathered by
// the permutation.  M is block upper triangular (zero left of each pivot
// block), which the operand formation exploits.  Each row's place in the
// sigma-grouped operand (sigma = +1 rows first, then -1; zero pivots drop)
// is returned in `outrow`.
//
// Two variants.  tfactor_kernel: one CTA per T slot, the matrix in global
// memory (L2 resident), lower triangle only: n sequential pivot steps, each
// bound by one SM's FP64 rate and by L2 round trips.  Beside the S
// contraction one CTA per slot costs the fewest SMs.  tfactor_dsm_kernel: a
// cluster of kTfCluster CTAs per slot with the rows distributed over their
// shared memory, for the case where the factorisation leads the critical path
// (S by the addition theorem).  Both take the same pivot decisions and do
// the same arithmetic per element.
#include <algorithm>
#include <cmath>

#include "flapw_internal.h"

namespace flapw {
namespace {

constexpr int kMaxN = 2 * kMaxNL;
constexpr int kTfThreads = 512;         // one CTA per slot
constexpr int kTfCluster = 8;           // CTAs per slot in the cluster variant

__device__ __forceinline__ uint32_t tf_cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Barrier of all threads of the cluster (CL > 1) or of the CTA, with
// release/acquire ordering of global and shared memory.
template <int CL>
__device__ __forceinline__ void tf_sync() {
  if (CL > 1)
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
  else
    __syncthreads();
}
// Shared-memory word of CTA `rank` of the cluster at the address of p.
__device__ __forceinline__ double tf_ld_remote(const double* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}
__device__ __forceinline__ int tf_ld_remote(const int* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
  return v;
}

__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }
__device__ __forceinline__ double2 cconj(double2 z) { return make_double2(z.x, -z.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Block-wide argmax of v (ties: smallest index).  Returns through shared.
__device__ void block_argmax(double v, int idx, double* s_val, int* s_idx, double* out_v,
                             int* out_i) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  if (lane == 0) {
    s_val[w] = v;
    s_idx[w] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = s_val[0];
    int bi = s_idx[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
      if (s_val[i] > bv || (s_val[i] == bv && s_idx[i] < bi)) {
        bv = s_val[i];
        bi = s_idx[i];
      }
    *out_v = bv;
    *out_i = bi;
  }
  __syncthreads();
}

// Cluster-wide argmax: each CTA's candidate (cand_v, cand_i, written by its
// thread 0 after block_argmax) is read by every CTA's thread 0 after a cluster
// barrier; ties take the smallest index.  CL = 1: the CTA's own result.
template <int CL>
__device__ void cluster_argmax(const double* cand_v, const int* cand_i, double* out_v, int* out_i) {
  if (CL > 1) {
    tf_sync<CL>();
    if (threadIdx.x < 32) {
      // lane r reads CTA r's candidate: the remote loads overlap
      const int lane = threadIdx.x;
      double bv = -1.0;
      int bi = 1 << 30;
      if (lane < CL) {
        bv = tf_ld_remote(cand_v, (uint32_t)lane);
        bi = tf_ld_remote(cand_i, (uint32_t)lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        *out_v = bv;
        *out_i = bi;
      }
    }
    __syncthreads();
  } else {
    if (threadIdx.x == 0) {
      *out_v = *cand_v;
      *out_i = *cand_i;
    }
    __syncthreads();
  }
}

// One CTA per slot, the matrix in global memory (L2 resident).
__global__ void __launch_bounds__(kTfThreads)
    tfactor_kernel(const double2* T, int n, double2* work, double2* CH, int* perm_out,
                   int* outrow_out, int* npos, int* nneg, int* npiv2, int* err) {
  constexpr int CL = 1;
  const int slot = blockIdx.x;
  const double2* Ts = T + (int64_t)slot * n * n;
  double2* A = work + (int64_t)slot * n * n;
  double2* C = CH + (int64_t)slot * n * n;
  const int tid = threadIdx.x, nt = blockDim.x;

  __shared__ int perm[kMaxN], blk[kMaxN], outrow[kMaxN];
  __shared__ double lam[kMaxN];
  __shared__ double2 qv[kMaxN][2];
  __shared__ double2 col0[kMaxN], col1[kMaxN], lc0[kMaxN], lc1[kMaxN];  // pivot columns, L columns
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double c_colv, c_rowv;  // this CTA's argmax candidates
  __shared__ int c_coli, c_rowi;
  __shared__ double s_colmax, s_rowmax;
  __shared__ int s_imax, s_jmax;
  __shared__ int s_bad;

  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    A[idx] = (i >= j) ? Ts[idx] : make_double2(0.0, 0.0);
    C[idx] = make_double2(0.0, 0.0);
  }
  for (int i = tid; i < n; i += nt) perm[i] = i;
  if (tid == 0) s_bad = 0;
  tf_sync<CL>();

  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  int k = 0, n2 = 0;
  while (k < n) {
    // largest off-diagonal entry of column k
    double v = -1.0;
    int vi = n;
    for (int i = k + 1 + tid; i < n; i += nt) {
      const double c = cabs1(A[(int64_t)i * n + k]);
      if (c > v) {
        v = c;
        vi = i;
      }
    }
    block_argmax(v, vi, red_v, red_i, &c_colv, &c_coli);
    cluster_argmax<CL>(&c_colv, &c_coli, &s_colmax, &s_imax);
    const double colmax = (k + 1 < n) ? s_colmax : 0.0;
    const int imax = s_imax;
    const double absakk = fabs(A[(int64_t)k * n + k].x);
    int kstep = 1, kp = k;
    if (fmax(absakk, colmax) == 0.0) {
      kstep = 1;
      kp = k;  // zero column: zero pivot, dropped below
    } else if (absakk >= alpha * colmax) {
      kstep = 1;
      kp = k;
    } else {
      // largest off-diagonal entry of row/column imax in the trailing matrix
      double r = -1.0;
      int ri = n;
      for (int j = k + tid; j < n; j += nt) {
        if (j == imax) continue;
        const double c = (j < imax) ? cabs1(A[(int64_t)imax * n + j]) : cabs1(A[(int64_t)j * n + imax]);
        if (c > r) {
          r = c;
          ri = j;
        }
      }
      block_argmax(r, ri, red_v, red_i, &c_rowv, &c_rowi);
      cluster_argmax<CL>(&c_rowv, &c_rowi, &s_rowmax, &s_jmax);
      const double rowmax = s_rowmax;
      if (absakk >= alpha * colmax * (colmax / rowmax)) {
        kstep = 1;
        kp = k;
      } else if (fabs(A[(int64_t)imax * n + imax].x) >= alpha * rowmax) {
        kstep = 1;
        kp = imax;
      } else {
        kstep = 2;
        kp = imax;
      }
    }
    const int kk = k + kstep - 1;
    if (kp != kk) {
      // symmetric interchange of rows/cols kk and kp (kk < kp), lower storage;
      // also swaps the rows of the L columns already computed.
      for (int j = tid; j < n; j += nt) {
        if (j < kk) {
          const double2 t = A[(int64_t)kk * n + j];
          A[(int64_t)kk * n + j] = A[(int64_t)kp * n + j];
          A[(int64_t)kp * n + j] = t;
        } else if (j > kk && j < kp) {
          const double2 t = A[(int64_t)j * n + kk];
          A[(int64_t)j * n + kk] = cconj(A[(int64_t)kp * n + j]);
          A[(int64_t)kp * n + j] = cconj(t);
        } else if (j > kp) {
          const double2 t = A[(int64_t)j * n + kk];
          A[(int64_t)j * n + kk] = A[(int64_t)j * n + kp];
          A[(int64_t)j * n + kp] = t;
        }
      }
      if (tid == 0) {
        const double2 dk = A[(int64_t)kk * n + kk];
        A[(int64_t)kk * n + kk] = make_double2(A[(int64_t)kp * n + kp].x, 0.0);
        A[(int64_t)kp * n + kp] = make_double2(dk.x, 0.0);
        A[(int64_t)kp * n + kk] = cconj(A[(int64_t)kp * n + kk]);
        const int t = perm[kk];
        perm[kk] = perm[kp];
        perm[kp] = t;
      }
    }
    tf_sync<CL>();
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    if (kstep == 1) {
      const double d = A[(int64_t)k * n + k].x;
      if (d != 0.0) {
        const double rd = 1.0 / d;
        // pivot column a (unscaled) and L column l = a / d, once per step
        for (int i = k + 1 + tid; i < n; i += nt) {
          const double2 a = A[(int64_t)i * n + k];
          col0[i] = a;
          lc0[i] = make_double2(a.x * rd, a.y * rd);
        }
        __syncthreads();
        // A[i][j] -= l_i conj(a_j) on the lower trailing triangle: a warp per
        // row, lanes along the row (contiguous j)
        for (int i = k + 1 + warp; i < n; i += nw) {
          const double2 li = lc0[i];
          double2* row = A + (int64_t)i * n;
          for (int j = k + 1 + lane; j <= i; j += 32) {
            const double2 aj = col0[j];
            double2 x = row[j];
            x.x = fma(-li.x, aj.x, fma(-li.y, aj.y, x.x));
            x.y = (i == j) ? 0.0 : fma(-li.y, aj.x, fma(li.x, aj.y, x.y));
            row[j] = x;
          }
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < n; i += nt) A[(int64_t)i * n + k] = lc0[i];
      }
      if (tid == 0) {
        lam[k] = d;
        blk[k] = 1;
        qv[k][0] = make_double2(1.0, 0.0);
        qv[k][1] = make_double2(0.0, 0.0);
      }
    } else {
      const double d11 = A[(int64_t)k * n + k].x, d22 = A[(int64_t)(k + 1) * n + k + 1].x;
      const double2 d21 = A[(int64_t)(k + 1) * n + k];
      const double det = d11 * d22 - (d21.x * d21.x + d21.y * d21.y);
      if (det == 0.0) {
        if (tid == 0) s_bad = 1;
      } else {
        const double rdet = 1.0 / det;
        // pivot columns w1, w2 (unscaled) and L = W D^{-1}:
        //   l1 = (w1 d22 - w2 d21)/det,  l2 = (w2 d11 - w1 conj(d21))/det
        for (int i = k + 2 + tid; i < n; i += nt) {
          const double2 w1 = A[(int64_t)i * n + k], w2 = A[(int64_t)i * n + k + 1];
          const double2 t1 = cmul(w2, d21);
          const double2 t2 = cmul(w1, cconj(d21));
          col0[i] = w1;
          col1[i] = w2;
          lc0[i] = make_double2((w1.x * d22 - t1.x) * rdet, (w1.y * d22 - t1.y) * rdet);
          lc1[i] = make_double2((w2.x * d11 - t2.x) * rdet, (w2.y * d11 - t2.y) * rdet);
        }
        __syncthreads();
        // A[i][j] -= l1_i conj(w1_j) + l2_i conj(w2_j), lower trailing triangle
        for (int i = k + 2 + warp; i < n; i += nw) {
          const double2 l1 = lc0[i], l2 = lc1[i];
          double2* row = A + (int64_t)i * n;
          for (int j = k + 2 + lane; j <= i; j += 32) {
            const double2 v1 = col0[j], v2 = col1[j];
            double2 x = row[j];
            x.x = fma(-l1.x, v1.x, fma(-l1.y, v1.y, fma(-l2.x, v2.x, fma(-l2.y, v2.y, x.x))));
            x.y = (i == j) ? 0.0
                           : fma(-l1.y, v1.x, fma(l1.x, v1.y, fma(-l2.y, v2.x, fma(l2.x, v2.y, x.y))));
            row[j] = x;
          }
        }
        __syncthreads();
        for (int i = k + 2 + tid; i < n; i += nt) {
          A[(int64_t)i * n + k] = lc0[i];
          A[(int64_t)i * n + k + 1] = lc1[i];
        }
      }
      if (tid == 0) {
        // D = [[a, conj(b)], [b, c]] = Q diag(l+, l-) Q^H
        const double a = d11, c = d22;
        const double bb = sqrt(d21.x * d21.x + d21.y * d21.y);
        const double h = 0.5 * (a - c);
        const double rt = sqrt(h * h + bb * bb);
        const double lp = 0.5 * (a + c) + rt, lm = 0.5 * (a + c) - rt;
        // v+ = [conj(b), l+ - a], v- = [l- - c, b]  (orthogonal since l+ + l- = a + c)
        double2 p0 = cconj(d21), p1 = make_double2(lp - a, 0.0);
        double2 q0 = make_double2(lm - c, 0.0), q1 = d21;
        const double np = sqrt(p0.x * p0.x + p0.y * p0.y + p1.x * p1.x);
        const double nq = sqrt(q0.x * q0.x + q1.x * q1.x + q1.y * q1.y);
        p0 = make_double2(p0.x / np, p0.y / np);
        p1 = make_double2(p1.x / np, 0.0);
        q0 = make_double2(q0.x / nq, 0.0);
        q1 = make_double2(q1.x / nq, q1.y / nq);
        lam[k] = lp;
        lam[k + 1] = lm;
        qv[k][0] = p0;      // Q[0][0]
        qv[k][1] = p1;      // Q[1][0]
        qv[k + 1][0] = q0;  // Q[0][1]
        qv[k + 1][1] = q1;  // Q[1][1]
        blk[k] = 2;
        blk[k + 1] = 0;
        ++n2;
      }
    }
    __syncthreads();
    k += kstep;
  }
  if (tid == 0) {
    int np = 0, nn = 0;
    for (int r = 0; r < n; ++r)
      if (lam[r] > 0) ++np;
      else if (lam[r] < 0) ++nn;
    int ip = 0, in = np;
    for (int r = 0; r < n; ++r) {
      if (lam[r] > 0) outrow[r] = ip++;
      else if (lam[r] < 0) outrow[r] = in++;
      else outrow[r] = -1;
    }
    npos[slot] = np;
    nneg[slot] = nn;
    atomicAdd(npiv2, n2);
    if (s_bad) atomicExch(err, FLAPW_ERR_FACTOR);
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    perm_out[slot * n + i] = perm[i];
    outrow_out[slot * n + i] = outrow[i];
  }
  // M[r][i] = sqrt|lam_r| sum_{j in block(r)} conj(Q[j][r]) (L^H)[j][i],
  // (L^H)[j][i] = conj(L[i][j]) with unit diagonal and zero for i < j.
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx / n, i = idx % n;
    const int b0 = (blk[r] == 0) ? r - 1 : r;  // first row of r's block
    const int bs = (blk[b0] == 2) ? 2 : 1;
    double2 acc = make_double2(0.0, 0.0);
    for (int e = 0; e < bs; ++e) {
      const int j = b0 + e;
      double2 lv;
      if (i == j) lv = make_double2(1.0, 0.0);
      else if (i > b0 + bs - 1) lv = cconj(A[(int64_t)i * n + j]);
      else lv = make_double2(0.0, 0.0);
      const double2 q = (bs == 2) ? qv[r][e] : make_double2(1.0, 0.0);
      const double2 t = cmul(cconj(q), lv);
      acc.x += t.x;
      acc.y += t.y;
    }
    const double sq = sqrt(fabs(lam[r]));
    C[(int64_t)r * n + i] = make_double2(sq * acc.x, sq * acc.y);
  }
}

// ---- the cluster variant with the matrix in distributed shared memory -------
//
// A cluster of kTfCluster CTAs per slot.  Row i of the lower triangle (its
// entries 0..i) lives in the shared memory of CTA i mod kTfCluster, packed:
// the CTA's t-th row (i = q + kTfCluster t) starts at t (q + 1) +
// kTfCluster t (t - 1) / 2.  Every CTA lays its dynamic shared memory out alike
// (fixed arrays first, its rows last), so the cluster address of any element
// is the owner's rank applied to the local address (mapa).  Per pivot step:
// each CTA scans its own rows (column search; the row search where
// Bunch-Kaufman needs it) and posts an argmax candidate; after a cluster
// barrier every CTA takes the same decision.  An interchange gathers the two
// rows and the column entries it moves, meets at a barrier, then each CTA
// rewrites its own rows, and meets again.  Every CTA gathers the pivot
// column(s) from their owners, computes the L column and updates its own
// rows; after one more barrier (all gathers done) the owners write the L
// column back.  The decisions, the arithmetic per element and the tie-breaks
// are those of tfactor_kernel.
constexpr int kDsmThreads = 256;
constexpr int kDsmFixedBytes =
    (7 * kMaxN * 16 + 2 * kMaxN * 16 + kMaxN * 8 + 3 * kMaxN * 4 + 15) / 16 * 16;

__host__ __device__ inline int dsm_row_off(int i) {
  const int q = i % kTfCluster, t = i / kTfCluster;
  return t * (q + 1) + kTfCluster * t * (t - 1) / 2;
}
// Largest packed row storage of any CTA for an n x n block (elements).
inline int dsm_rows_elems(int n) {
  int mx = 0;
  for (int q = 0; q < kTfCluster; ++q) {
    const int rows = (n > q) ? (n - q + kTfCluster - 1) / kTfCluster : 0;
    mx = std::max(mx, rows * (q + 1) + kTfCluster * rows * (rows - 1) / 2);
  }
  return mx;
}
__device__ __forceinline__ double2 dsm_ld(const double2* rows, int i, int j) {
  const uint32_t local = (uint32_t)__cvta_generic_to_shared(rows + dsm_row_off(i) + j);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(ra)
               : "r"(local), "r"((uint32_t)(i % kTfCluster)));
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(ra) : "memory");
  return v;
}
// smallest i >= x owned by CTA q
__device__ __forceinline__ int dsm_first(int x, int q) {
  return x + ((q - x % kTfCluster) + kTfCluster) % kTfCluster;
}

__global__ void __launch_bounds__(kDsmThreads) tfactor_dsm_kernel(const double2* T, int n,
                                                                  double2* CH, int* perm_out,
                                                                  int* outrow_out, int* npos,
                                                                  int* nneg, int* npiv2,
                                                                  int* err) {
  constexpr int CL = kTfCluster;
  extern __shared__ __align__(16) unsigned char dsm_smem[];
  double2* col0 = reinterpret_cast<double2*>(dsm_smem);
  double2* col1 = col0 + kMaxN;
  double2* lc0 = col1 + kMaxN;
  double2* lc1 = lc0 + kMaxN;
  double2* rkk = lc1 + kMaxN;  // gathered row kk, row kp, column kk (interchange)
  double2* rkp = rkk + kMaxN;
  double2* ckk = rkp + kMaxN;
  double2* qv = ckk + kMaxN;   // [r][2]
  double* lam = reinterpret_cast<double*>(qv + 2 * kMaxN);
  int* perm = reinterpret_cast<int*>(lam + kMaxN);
  int* blk = perm + kMaxN;
  int* outrow = blk + kMaxN;
  double2* Al = reinterpret_cast<double2*>(dsm_smem + kDsmFixedBytes);  // this CTA's rows
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  // argmax candidates, double-buffered by step parity: a CTA rewrites a slot
  // only two steps later, after a cluster barrier every reader has passed
  // (a step with a zero pivot has no barrier after the candidates' one)
  __shared__ double c_colv[2], c_rowv[2];
  __shared__ int c_coli[2], c_rowi[2];
  __shared__ double s_colmax, s_rowmax;
  __shared__ int s_imax, s_jmax;
  __shared__ double2 s_d[3];
  __shared__ int s_bad;

  const int slot = blockIdx.x / CL;
  const int q = (int)tf_cluster_rank();
  const double2* Ts = T + (int64_t)slot * n * n;
  double2* Cm = CH + (int64_t)slot * n * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;

  // this CTA's rows of the lower triangle of T
  for (int i = q; i < n; i += CL) {
    double2* row = Al + dsm_row_off(i);
    for (int j = tid; j <= i; j += nt) row[j] = Ts[(int64_t)i * n + j];
  }
  for (int i = tid; i < n; i += nt) perm[i] = i;
  if (tid == 0) s_bad = 0;
  tf_sync<CL>();

  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  int k = 0, n2 = 0, it = 0;
  for (; k < n; ++it) {
    const int cb = it & 1;
    // largest off-diagonal entry of column k, over this CTA's rows
    double v = -1.0;
    int vi = n;
    for (int i = dsm_first(k + 1, q) + CL * tid; i < n; i += CL * nt) {
      const double c = cabs1(Al[dsm_row_off(i) + k]);
      if (c > v) {
        v = c;
        vi = i;
      }
    }
    if (tid == 0) s_d[0] = dsm_ld(Al, k, k);  // final since the last step's barrier
    block_argmax(v, vi, red_v, red_i, &c_colv[cb], &c_coli[cb]);
    cluster_argmax<CL>(&c_colv[cb], &c_coli[cb], &s_colmax, &s_imax);
    const double colmax = (k + 1 < n) ? s_colmax : 0.0;
    const int imax = s_imax;
    const double absakk = fabs(s_d[0].x);
    int kstep = 1, kp = k;
    if (fmax(absakk, colmax) == 0.0) {
      kstep = 1;
      kp = k;
    } else if (absakk >= alpha * colmax) {
      kstep = 1;
      kp = k;
    } else {
      // largest off-diagonal entry of row/column imax in the trailing matrix:
      // row imax (its owner) for k <= j < imax, column imax (each row's owner) below
      double r = -1.0;
      int ri = n;
      if (imax % CL == q) {
        const double2* rowm = Al + dsm_row_off(imax);
        for (int j = k + tid; j < imax; j += nt) {
          const double c = cabs1(rowm[j]);
          if (c > r) {
            r = c;
            ri = j;
          }
        }
      }
      for (int j = dsm_first(imax + 1, q) + CL * tid; j < n; j += CL * nt) {
        const double c = cabs1(Al[dsm_row_off(j) + imax]);
        if (c > r || (c == r && j < ri)) {
          r = c;
          ri = j;
        }
      }
      if (tid == 0) s_d[1] = dsm_ld(Al, imax, imax);
      block_argmax(r, ri, red_v, red_i, &c_rowv[cb], &c_rowi[cb]);
      cluster_argmax<CL>(&c_rowv[cb], &c_rowi[cb], &s_rowmax, &s_jmax);
      const double rowmax = s_rowmax;
      if (absakk >= alpha * colmax * (colmax / rowmax)) {
        kstep = 1;
        kp = k;
      } else if (fabs(s_d[1].x) >= alpha * rowmax) {
        kstep = 1;
        kp = imax;
      } else {
        kstep = 2;
        kp = imax;
      }
    }
    const int kk = k + kstep - 1;
    if (kp != kk) {
      // symmetric interchange of rows/cols kk and kp (kk < kp): gather, meet,
      // rewrite the own rows, meet
      for (int j = tid; j <= kp; j += nt) {
        if (j <= kk) rkk[j] = dsm_ld(Al, kk, j);
        rkp[j] = dsm_ld(Al, kp, j);
        if (j > kk && j < kp) ckk[j] = dsm_ld(Al, j, kk);
      }
      tf_sync<CL>();
      if (kk % CL == q) {
        double2* row = Al + dsm_row_off(kk);
        for (int j = tid; j < kk; j += nt) row[j] = rkp[j];
        if (tid == 0) row[kk] = make_double2(rkp[kp].x, 0.0);
      }
      if (kp % CL == q) {
        double2* row = Al + dsm_row_off(kp);
        for (int j = tid; j < kp; j += nt) {
          if (j < kk) row[j] = rkk[j];
          else if (j > kk) row[j] = cconj(ckk[j]);
          else row[j] = cconj(rkp[kk]);
        }
        if (tid == 0) row[kp] = make_double2(rkk[kk].x, 0.0);
      }
      for (int j = dsm_first(kk + 1, q) + CL * tid; j < n; j += CL * nt) {
        double2* row = Al + dsm_row_off(j);
        if (j < kp) {
          row[kk] = cconj(rkp[j]);
        } else if (j > kp) {
          const double2 t = row[kk];
          row[kk] = row[kp];
          row[kp] = t;
        }
      }
      if (tid == 0) {
        const int t = perm[kk];
        perm[kk] = perm[kp];
        perm[kp] = t;
      }
      tf_sync<CL>();
    }
    if (kstep == 1) {
      for (int i = k + 1 + tid; i < n; i += nt) col0[i] = dsm_ld(Al, i, k);
      if (tid == 0) s_d[0] = dsm_ld(Al, k, k);
      __syncthreads();
      const double d = s_d[0].x;
      if (d != 0.0) {
        const double rd = 1.0 / d;
        for (int i = k + 1 + tid; i < n; i += nt) {
          const double2 a = col0[i];
          lc0[i] = make_double2(a.x * rd, a.y * rd);
        }
        __syncthreads();
        // A[i][j] -= l_i conj(a_j), k < j <= i, on this CTA's rows: a warp per row
        for (int i = dsm_first(k + 1, q) + CL * warp; i < n; i += CL * nw) {
          const double2 li = lc0[i];
          double2* row = Al + dsm_row_off(i);
          for (int j = k + 1 + lane; j <= i; j += 32) {
            const double2 aj = col0[j];
            double2 x = row[j];
            x.x = fma(-li.x, aj.x, fma(-li.y, aj.y, x.x));
            x.y = (i == j) ? 0.0 : fma(-li.y, aj.x, fma(li.x, aj.y, x.y));
            row[j] = x;
          }
        }
        // every CTA has gathered column k before its owners overwrite it
        tf_sync<CL>();
        for (int i = dsm_first(k + 1, q) + CL * tid; i < n; i += CL * nt) Al[dsm_row_off(i) + k] = lc0[i];
      }
      if (tid == 0) {
        lam[k] = d;
        blk[k] = 1;
        qv[2 * k] = make_double2(1.0, 0.0);
        qv[2 * k + 1] = make_double2(0.0, 0.0);
      }
    } else {
      for (int i = k + 2 + tid; i < n; i += nt) {
        col0[i] = dsm_ld(Al, i, k);
        col1[i] = dsm_ld(Al, i, k + 1);
      }
      if (tid == 0) s_d[0] = dsm_ld(Al, k, k);
      if (tid == 32) s_d[1] = dsm_ld(Al, k + 1, k + 1);
      if (tid == 64) s_d[2] = dsm_ld(Al, k + 1, k);
      __syncthreads();
      const double d11 = s_d[0].x, d22 = s_d[1].x;
      const double2 d21 = s_d[2];
      const double det = d11 * d22 - (d21.x * d21.x + d21.y * d21.y);
      if (det == 0.0) {
        if (tid == 0) s_bad = 1;
      } else {
        const double rdet = 1.0 / det;
        for (int i = k + 2 + tid; i < n; i += nt) {
          const double2 w1 = col0[i], w2 = col1[i];
          const double2 t1 = cmul(w2, d21);
          const double2 t2 = cmul(w1, cconj(d21));
          lc0[i] = make_double2((w1.x * d22 - t1.x) * rdet, (w1.y * d22 - t1.y) * rdet);
          lc1[i] = make_double2((w2.x * d11 - t2.x) * rdet, (w2.y * d11 - t2.y) * rdet);
        }
        __syncthreads();
        for (int i = dsm_first(k + 2, q) + CL * warp; i < n; i += CL * nw) {
          const double2 l1 = lc0[i], l2 = lc1[i];
          double2* row = Al + dsm_row_off(i);
          for (int j = k + 2 + lane; j <= i; j += 32) {
            const double2 v1 = col0[j], v2 = col1[j];
            double2 x = row[j];
            x.x = fma(-l1.x, v1.x, fma(-l1.y, v1.y, fma(-l2.x, v2.x, fma(-l2.y, v2.y, x.x))));
            x.y = (i == j) ? 0.0
                           : fma(-l1.y, v1.x, fma(l1.x, v1.y, fma(-l2.y, v2.x, fma(l2.x, v2.y, x.y))));
            row[j] = x;
          }
        }
        tf_sync<CL>();
        for (int i = dsm_first(k + 2, q) + CL * tid; i < n; i += CL * nt) {
          Al[dsm_row_off(i) + k] = lc0[i];
          Al[dsm_row_off(i) + k + 1] = lc1[i];
        }
      }
      if (tid == 0) {
        const double a = d11, c = d22;
        const double bb = sqrt(d21.x * d21.x + d21.y * d21.y);
        const double h = 0.5 * (a - c);
        const double rt = sqrt(h * h + bb * bb);
        const double lp = 0.5 * (a + c) + rt, lm = 0.5 * (a + c) - rt;
        double2 p0 = cconj(d21), p1 = make_double2(lp - a, 0.0);
        double2 q0 = make_double2(lm - c, 0.0), q1 = d21;
        const double np_ = sqrt(p0.x * p0.x + p0.y * p0.y + p1.x * p1.x);
        const double nq = sqrt(q0.x * q0.x + q1.x * q1.x + q1.y * q1.y);
        p0 = make_double2(p0.x / np_, p0.y / np_);
        p1 = make_double2(p1.x / np_, 0.0);
        q0 = make_double2(q0.x / nq, 0.0);
        q1 = make_double2(q1.x / nq, q1.y / nq);
        lam[k] = lp;
        lam[k + 1] = lm;
        qv[2 * k] = p0;
        qv[2 * k + 1] = p1;
        qv[2 * (k + 1)] = q0;
        qv[2 * (k + 1) + 1] = q1;
        blk[k] = 2;
        blk[k + 1] = 0;
        ++n2;
      }
    }
    __syncthreads();
    k += kstep;
  }
  tf_sync<CL>();  // the last L columns are written
  if (tid == 0) {
    int np = 0, nn = 0;
    for (int r = 0; r < n; ++r)
      if (lam[r] > 0) ++np;
      else if (lam[r] < 0) ++nn;
    int ip = 0, in = np;
    for (int r = 0; r < n; ++r) {
      if (lam[r] > 0) outrow[r] = ip++;
      else if (lam[r] < 0) outrow[r] = in++;
      else outrow[r] = -1;
    }
    if (q == 0) {
      npos[slot] = np;
      nneg[slot] = nn;
      atomicAdd(npiv2, n2);
      if (s_bad) atomicExch(err, FLAPW_ERR_FACTOR);
    }
  }
  __syncthreads();
  if (q == 0)
    for (int i = tid; i < n; i += nt) {
      perm_out[slot * n + i] = perm[i];
      outrow_out[slot * n + i] = outrow[i];
    }
  // M[r][i] = sqrt|lam_r| sum_{j in block(r)} conj(Q[j][r]) conj(L[i][j]): the
  // owner of row i writes column i of M
  for (int i = q; i < n; i += CL) {
    const double2* row = Al + dsm_row_off(i);
    for (int r = tid; r < n; r += nt) {
      const int b0 = (blk[r] == 0) ? r - 1 : r;
      const int bs = (blk[b0] == 2) ? 2 : 1;
      double2 acc = make_double2(0.0, 0.0);
      for (int e = 0; e < bs; ++e) {
        const int j = b0 + e;
        double2 lv;
        if (i == j) lv = make_double2(1.0, 0.0);
        else if (i > b0 + bs - 1) lv = cconj(row[j]);
        else lv = make_double2(0.0, 0.0);
        const double2 qq = (bs == 2) ? qv[2 * r + e] : make_double2(1.0, 0.0);
        const double2 t = cmul(cconj(qq), lv);
        acc.x += t.x;
        acc.y += t.y;
      }
      const double sq = sqrt(fabs(lam[r]));
      Cm[(int64_t)r * n + i] = make_double2(sq * acc.x, sq * acc.y);
    }
  }
  tf_sync<CL>();  // no CTA leaves while another may still read its rows
}

__global__ void layout_kernel(const int* npos, const int* nneg, const int* atom_slot, int n_atoms,
                              int n_k, int* pos_off, int* neg_off, int* kpk, Prob* probs,
                              int k_total) {
  if (threadIdx.x != 0) return;
  int p = 0, q = 0;
  for (int a = 0; a < n_atoms; ++a) {
    pos_off[a] = p;
    neg_off[a] = q;
    p += npos[atom_slot[a]];
    q += nneg[atom_slot[a]];
  }
  kpk[0] = neg_base(p);
  kpk[1] = p;
  kpk[2] = q;
  for (int k = 0; k < n_k; ++k) {  // problems [0, n_k) are the H problems
    probs[k].kp = p;
    probs[k].kn = q;
  }
  (void)k_total;
}

}  // namespace

cudaError_t launch_tfactor(const double2* T, int n, int n_slots, double2* work, double2* CH,
                           int* perm, int* outrow, int* npos, int* nneg, int* npiv2, int* err,
                           bool cluster, cudaStream_t st) {
  if (n > kMaxN) return cudaErrorInvalidValue;
  if (n_slots == 0) return cudaSuccess;
  if (!cluster) {
    tfactor_kernel<<<n_slots, kTfThreads, 0, st>>>(T, n, work, CH, perm, outrow, npos, nneg, npiv2,
                                                   err);
    return cudaGetLastError();
  }
  const size_t dyn = (size_t)kDsmFixedBytes + (size_t)dsm_rows_elems(n) * 16;
  cudaError_t e = cudaFuncSetAttribute(tfactor_dsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dyn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(n_slots * kTfCluster));
  cfg.blockDim = dim3(kDsmThreads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTfCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)work;
  return cudaLaunchKernelEx(&cfg, tfactor_dsm_kernel, T, n, CH, perm, outrow, npos, nneg, npiv2, err);
}

cudaError_t launch_layout(const int* npos, const int* nneg, const int* atom_slot, int n_atoms,
                          int n_k, int* pos_off, int* neg_off, int* kpk, Prob* probs,
                          int k_total, cudaStream_t st) {
  layout_kernel<<<1, 32, 0, st>>>(npos, nneg, atom_slot, n_atoms, n_k, pos_off, neg_off, kpk,
                                  probs, k_total);
  return cudaGetLastError();
}

}  // namespace flapw
