// Operand formation for the two rank-K contractions (Sec. 3, Eqs. (h), (s),
// the stacking of Fig. agg):
//
//   H:  Z_a = C_{slot(a)}^H [A_a; B_a]      (2N_L rows per atom, sigma-grouped)
//   S:  Z_S,a = [A_a; U_a B_a]              (U = diag ||udot_l||, Eq. (s))
//
// Z is stored row-major per plane wave: row g of a problem holds the K
// operand entries of column g, contiguous, so that the contraction reads
// K-major tiles.  In the H operand the rows with sigma = +1 of every atom come
// first (offset pos_off[a]), then, from column Kp_pad (a multiple of 64), the
// sigma = -1 rows (offset neg_off[a]).
//
// FP64 SIMT: a 32 (C^H rows) x 64 (plane waves) tile per CTA, the 2N_L-long
// reduction staged through shared memory 16 at a time.  C^H = M P^T with M
// block upper triangular in pivoted order: the W rows are gathered through
// the permutation and the reduction starts at the tile's first nonzero column,
// which halves the FP64 work of a dense product.
//
// The factored variant uses A_a = diag(e^{iK.tau_a}) A_t (A depends on the
// atom only through its structure-factor phase): Z_{slot,t} = C^H [A_t; B_t]
// is formed once per (slot, type) pair and multiplied by each atom's phase.
//
// The paper's Alg. 3 needs no factorisation: its operands (alg3.cuh) are the
// rows of M [A_a; B_a] placed into L and R, plus copies of A_a and B_a.
#include "alg3.cuh"
#include "flapw_internal.h"

namespace flapw {
namespace {

constexpr int kRT = 32;  // C^H rows per CTA
constexpr int kGT = 64;  // plane waves per CTA
constexpr int kCT = 16;  // reduction chunk

__constant__ int c_l_of_L[kMaxNL];

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}

// W row c (c < 2 N_L) of atom a at plane wave g of k-point k (A/B input).
__device__ __forceinline__ double2 w_from_ab(const OpformArgs& p, int a, int c, int k, int g,
                                             int64_t ng) {
  const int64_t base = (int64_t)p.n_L * p.n_atoms * p.goff[k] + (int64_t)a * p.n_L * ng + g;
  return (c < p.n_L) ? p.A[base + (int64_t)c * ng] : p.B[base + (int64_t)(c - p.n_L) * ng];
}

// W row c of type t (no atom phase) at global plane wave gi.
__device__ __forceinline__ double2 w_type(const OpformArgs& p, int t, int c, int64_t gi,
                                          int64_t G) {
  const int L = (c < p.n_L) ? c : c - p.n_L;
  const int l = c_l_of_L[L];
  const double2 y = p.Yc[(int64_t)L * G + gi];
  const int64_t ro = ((int64_t)t * (p.lmax + 1) + l) * G + gi;
  const double r = (c < p.n_L) ? p.al[ro] : p.bl[ro];
  return make_double2(y.x * r, y.y * r);
}

// grid: (g-tiles, ceil(n/32), atoms or combos); 256 threads.
template <bool kFactored>
__global__ void __launch_bounds__(256) opform_h_kernel(OpformArgs p, int64_t G) {
  __shared__ double2 chs[kCT][kRT];
  __shared__ double2 ws[kCT][kGT];
  const int k = p.gtiles[2 * blockIdx.x], g0 = p.gtiles[2 * blockIdx.x + 1];
  const int64_t ng = p.goff[k + 1] - p.goff[k];
  const int r0 = blockIdx.y * kRT;
  int slot, type, a_single;
  if (kFactored) {
    slot = p.combo_slot[blockIdx.z];
    type = p.combo_type[blockIdx.z];
    a_single = -1;
  } else {
    a_single = blockIdx.z;
    slot = p.atom_slot[a_single];
    type = p.atom_type[a_single];
  }
  const int n = p.n;
  const double2* CH = p.CH + (int64_t)slot * n * n;
  const int tid = threadIdx.x, rl = tid & 31, gq = tid >> 5;
  double2 acc[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = make_double2(0.0, 0.0);
  const int* perm = p.perm + (int64_t)slot * n;
  const int c_begin = (r0 > 0 ? r0 - 1 : 0) / kCT * kCT;  // M[r][c] = 0 for c < r - 1
  for (int c0 = c_begin; c0 < n; c0 += kCT) {
    for (int idx = tid; idx < kCT * kRT; idx += 256) {
      const int rr = idx / kCT, cc = idx % kCT;
      const int r = r0 + rr, c = c0 + cc;
      chs[cc][rr] = (r < n && c < n) ? CH[(int64_t)r * n + c] : make_double2(0.0, 0.0);
    }
    for (int idx = tid; idx < kCT * kGT; idx += 256) {
      const int cc = idx / kGT, gg = idx % kGT;
      const int c = c0 + cc, g = g0 + gg;
      double2 w = make_double2(0.0, 0.0);
      if (c < n && g < ng) {
        const int src = perm[c];
        if (kFactored) w = w_type(p, type, src, p.goff[k] + g, G);
        else w = w_from_ab(p, a_single, src, k, g, ng);
      }
      ws[cc][gg] = w;
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < kCT; ++cc) {
      const double2 ch = chs[cc][rl];
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = cfma(ch, ws[cc][gq * 8 + e], acc[e]);
    }
    __syncthreads();
  }
  if (r0 + rl >= n) return;
  const int r = p.outrow[(int64_t)slot * n + r0 + rl];  // sigma-grouped position
  const int np = p.npos[slot];
  if (r < 0) return;  // zero pivot: the row carries nothing
  const int64_t row0 = p.h_row0 + p.goff[k];
  if (kFactored) {
    for (int ai = p.combo_start[blockIdx.z]; ai < p.combo_start[blockIdx.z + 1]; ++ai) {
      const int a = p.combo_atoms[ai];
      int col;
      if (r < np) col = p.pos_off[a] + r;
      else col = p.kpk[0] + p.neg_off[a] + (r - np);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int g = g0 + gq * 8 + e;
        if (g < ng) {
          const double2 f = p.ph[(int64_t)a * G + p.goff[k] + g];
          const double2 z = make_double2(f.x * acc[e].x - f.y * acc[e].y, f.x * acc[e].y + f.y * acc[e].x);
          p.Z[(row0 + g) * p.k_alloc + col] = z;
        }
      }
    }
  } else {
    const int a = a_single;
    int col;
    if (r < np) col = p.pos_off[a] + r;
    else col = p.kpk[0] + p.neg_off[a] + (r - np);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int g = g0 + gq * 8 + e;
      if (g < ng) p.Z[(row0 + g) * p.k_alloc + col] = acc[e];
    }
  }
}

// S operand: Z[g][a*n + c] = c < N_L ? A_a[c][g] : U_{t,l} B_a[c - N_L][g].
// grid: (g-tiles, ceil(n/32), atoms).
template <bool kFactored>
__global__ void __launch_bounds__(256) opform_s_kernel(OpformArgs p, int64_t G) {
  __shared__ double2 tile[kRT][kGT + 1];
  const int k = p.gtiles[2 * blockIdx.x], g0 = p.gtiles[2 * blockIdx.x + 1];
  const int64_t ng = p.goff[k + 1] - p.goff[k];
  const int c0 = blockIdx.y * kRT;
  const int a = blockIdx.z;
  const int t = p.atom_type[a];
  const int n = p.n;
  for (int idx = threadIdx.x; idx < kRT * kGT; idx += 256) {
    const int cc = idx / kGT, gg = idx % kGT;
    const int c = c0 + cc, g = g0 + gg;
    double2 w = make_double2(0.0, 0.0);
    if (c < n && g < ng) {
      if (kFactored) {
        const int64_t gi = p.goff[k] + g;
        const double2 u = w_type(p, t, c, gi, G);
        const double2 f = p.ph[(int64_t)a * G + gi];
        w = make_double2(f.x * u.x - f.y * u.y, f.x * u.y + f.y * u.x);
      } else {
        w = w_from_ab(p, a, c, k, g, ng);
      }
      if (c >= p.n_L) {
        const double s = p.U[t * (p.lmax + 1) + c_l_of_L[c - p.n_L]];
        w.x *= s;
        w.y *= s;
      }
    }
    tile[cc][gg] = w;
  }
  __syncthreads();
  const int64_t row0 = p.s_row0 + p.goff[k];
  for (int idx = threadIdx.x; idx < kRT * kGT; idx += 256) {
    const int gg = idx / kRT, cc = idx % kRT;
    const int c = c0 + cc, g = g0 + gg;
    if (c < n && g < ng) p.Z[(row0 + g) * p.k_alloc + (int64_t)a * n + c] = tile[cc][gg];
  }
}

// X and Y rows of Alg. 3: row r of M [A_a; B_a] goes to column N_L + r of R_a
// and, for r < N_L (an X row), to column r of L_a; with Alg. 1's C^H rows a
// Y row goes to column N_L + r of L_a too.
// grid: (g-tiles, ceil(n/32), atoms or combos); 256 threads.
template <bool kFactored>
__global__ void __launch_bounds__(256) opform_alg3_kernel(OpformArgs p, int64_t G) {
  __shared__ double2 ms[kCT][kRT];
  __shared__ double2 ws[kCT][kGT];
  const int k = p.gtiles[2 * blockIdx.x], g0 = p.gtiles[2 * blockIdx.x + 1];
  const int64_t ng = p.goff[k + 1] - p.goff[k];
  const int r0 = blockIdx.y * kRT;
  int slot, type, a_single;
  if (kFactored) {
    slot = p.combo_slot[blockIdx.z];
    type = p.combo_type[blockIdx.z];
    a_single = -1;
  } else {
    a_single = blockIdx.z;
    slot = p.atom_slot[a_single];
    type = p.atom_type[a_single];
  }
  const int n = p.n, nL = p.n_L;
  const double2* Ms = p.M + (int64_t)slot * n * n;
  const bool y_in_l = p.hpd && p.hpd[slot];  // Alg. 1 with C^H: Y rows in L as well
  const int tid = threadIdx.x, rl = tid & 31, gq = tid >> 5;
  double2 acc[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = make_double2(0.0, 0.0);
  const int c_end = (r0 >= nL) ? nL : n;  // Y rows read the A half only
  for (int c0 = 0; c0 < c_end; c0 += kCT) {
    for (int idx = tid; idx < kCT * kRT; idx += 256) {
      const int rr = idx / kCT, cc = idx % kCT;
      const int r = r0 + rr, c = c0 + cc;
      ms[cc][rr] = (r < n && c < n) ? Ms[(int64_t)r * n + c] : make_double2(0.0, 0.0);
    }
    for (int idx = tid; idx < kCT * kGT; idx += 256) {
      const int cc = idx / kGT, gg = idx % kGT;
      const int c = c0 + cc, g = g0 + gg;
      double2 w = make_double2(0.0, 0.0);
      if (c < n && g < ng) {
        if (kFactored) w = w_type(p, type, c, p.goff[k] + g, G);
        else w = w_from_ab(p, a_single, c, k, g, ng);
      }
      ws[cc][gg] = w;
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < kCT; ++cc) {
      const double2 m = ms[cc][rl];
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = cfma(m, ws[cc][gq * 8 + e], acc[e]);
    }
    __syncthreads();
  }
  const int r = r0 + rl;
  if (r >= n) return;
  const int64_t lrow0 = p.h_row0 + p.goff[k], rrow0 = p.r_row0 + p.goff[k];
  const int a_begin = kFactored ? p.combo_start[blockIdx.z] : 0;
  const int a_end = kFactored ? p.combo_start[blockIdx.z + 1] : 1;
  for (int ai = a_begin; ai < a_end; ++ai) {
    const int a = kFactored ? p.combo_atoms[ai] : a_single;
    const int64_t base = (int64_t)a * 3 * nL;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int g = g0 + gq * 8 + e;
      if (g < ng) {
        double2 z = acc[e];
        if (kFactored) {
          const double2 f = p.ph[(int64_t)a * G + p.goff[k] + g];
          z = make_double2(f.x * acc[e].x - f.y * acc[e].y, f.x * acc[e].y + f.y * acc[e].x);
        }
        p.Z[(rrow0 + g) * p.k_alloc + base + nL + r] = z;
        if (r < nL) p.Z[(lrow0 + g) * p.k_alloc + base + r] = z;
        else if (y_in_l) p.Z[(lrow0 + g) * p.k_alloc + base + nL + r] = z;
      }
    }
  }
}

// The Alg. 3 / Alg. 1 operand matrix M of one slot (alg3.cuh) into Mo
// ([n][n] row-major).  With alg1, T^AA = C C^H by the left-looking Cholesky
// factorisation (column j: the pivot T^AA_jj - sum_k |C_jk|^2, then
// C_ij = (T^AA_ij - sum_k C_ik conj(C_jk)) / C_jj below it), in FP64, into the
// scratch W; a pivot that is not positive (or not finite) fails the slot as
// the paper's zpotrf would, and its Y rows stay T^AA.  One CTA per slot.
__global__ void __launch_bounds__(256) alg_m_kernel(const double2* __restrict__ T, int n, int nL, int alg1,
                                                    double2* __restrict__ M, double2* __restrict__ W,
                                                    int* __restrict__ hpd) {
  __shared__ double red[256];
  __shared__ int failed;
  const int slot = blockIdx.x, tid = threadIdx.x;
  const double2* Ts = T + (int64_t)slot * n * n;
  double2* Ms = M + (int64_t)slot * n * n;
  double2* Ws = W + (int64_t)slot * n * n;  // C (lower), row-major nL x nL
  for (int i = tid; i < nL * n; i += 256) Ms[i] = alg3::m_elem(Ts, n, nL, i / n, i % n);  // X rows
  if (tid == 0) failed = alg1 ? 0 : 1;
  __syncthreads();
  for (int j = 0; j < nL && !failed; ++j) {
    double part = 0.0;
    for (int k = tid; k < j; k += 256) {
      const double2 c = Ws[(int64_t)j * nL + k];
      part += c.x * c.x + c.y * c.y;
    }
    red[tid] = part;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    const double d = alg3::t_elem(Ts, n, j, j).x - red[0];
    __syncthreads();
    if (!(d > 0.0) || !isfinite(d)) {
      if (tid == 0) failed = 1;
      __syncthreads();
      break;
    }
    const double cjj = sqrt(d);
    if (tid == 0) Ws[(int64_t)j * nL + j] = make_double2(cjj, 0.0);
    for (int i = j + 1 + tid; i < nL; i += 256) {
      double2 s = alg3::t_elem(Ts, n, i, j);
      for (int k = 0; k < j; ++k) {
        const double2 a = Ws[(int64_t)i * nL + k], b = Ws[(int64_t)j * nL + k];
        s.x -= a.x * b.x + a.y * b.y;  // a conj(b)
        s.y -= a.y * b.x - a.x * b.y;
      }
      Ws[(int64_t)i * nL + j] = make_double2(s.x / cjj, s.y / cjj);
    }
    __syncthreads();
  }
  // Y rows: C^H (row i, column c >= i: conj(C_ci)) where the factorisation
  // succeeded, else T^AA; zero on the B half
  const bool chol = !failed;
  for (int e = tid; e < nL * n; e += 256) {
    const int i = e / n, c = e % n;
    double2 v = make_double2(0.0, 0.0);
    if (c < nL) {
      if (chol) {
        if (c >= i) {
          const double2 w = Ws[(int64_t)c * nL + i];
          v = make_double2(w.x, -w.y);
        }
      } else {
        v = alg3::m_elem(Ts, n, nL, nL + i, c);
      }
    }
    Ms[(int64_t)(nL + i) * n + c] = v;
  }
  if (tid == 0) hpd[slot] = chol ? 1 : 0;
}

// A_a and B_a into the Alg. 3 operands: L_a = [X; B; A] takes W row c at
// column N_L + c (B rows) or 2 N_L + c (A rows); R_a = [B; X; Y] takes the B
// rows at column c - N_L.  grid: (g-tiles, ceil(n/32), atoms).
template <bool kFactored>
__global__ void __launch_bounds__(256) opform_alg3_copy_kernel(OpformArgs p, int64_t G) {
  __shared__ double2 tile[kRT][kGT + 1];
  const int k = p.gtiles[2 * blockIdx.x], g0 = p.gtiles[2 * blockIdx.x + 1];
  const int64_t ng = p.goff[k + 1] - p.goff[k];
  const int c0 = blockIdx.y * kRT;
  const int a = blockIdx.z;
  const int t = p.atom_type[a];
  const int n = p.n, nL = p.n_L;
  for (int idx = threadIdx.x; idx < kRT * kGT; idx += 256) {
    const int cc = idx / kGT, gg = idx % kGT;
    const int c = c0 + cc, g = g0 + gg;
    double2 w = make_double2(0.0, 0.0);
    if (c < n && g < ng) {
      if (kFactored) {
        const int64_t gi = p.goff[k] + g;
        const double2 u = w_type(p, t, c, gi, G);
        const double2 f = p.ph[(int64_t)a * G + gi];
        w = make_double2(f.x * u.x - f.y * u.y, f.x * u.y + f.y * u.x);
      } else {
        w = w_from_ab(p, a, c, k, g, ng);
      }
    }
    tile[cc][gg] = w;
  }
  __syncthreads();
  const int64_t lrow0 = p.h_row0 + p.goff[k], rrow0 = p.r_row0 + p.goff[k];
  const int64_t base = (int64_t)a * 3 * nL;
  const bool y_in_l = p.hpd && p.hpd[p.atom_slot[a]];  // Alg. 1 with C^H: L's third block is Y
  for (int idx = threadIdx.x; idx < kRT * kGT; idx += 256) {
    const int gg = idx / kRT, cc = idx % kRT;
    const int c = c0 + cc, g = g0 + gg;
    if (c < n && g < ng) {
      const double2 v = tile[cc][gg];
      if (c < nL) {
        if (!y_in_l) p.Z[(lrow0 + g) * p.k_alloc + base + 2 * nL + c] = v;
      } else {
        p.Z[(lrow0 + g) * p.k_alloc + base + c] = v;
        p.Z[(rrow0 + g) * p.k_alloc + base + (c - nL)] = v;
      }
    }
  }
}

// Z[g][k'] = Zin[g*ldz + kmap[k']] (kmap < 0: zero), for the standalone contraction.
__global__ void gather_z_kernel(const double2* Zin, int64_t ldz, int K, int N, const int* kmap,
                                int64_t k_alloc, double2* Z) {
  const int g = blockIdx.y;
  for (int64_t kc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kc < k_alloc;
       kc += (int64_t)gridDim.x * blockDim.x) {
    const int src = kmap[kc];
    Z[(int64_t)g * k_alloc + kc] = (src >= 0) ? Zin[(int64_t)g * ldz + src] : make_double2(0.0, 0.0);
  }
  (void)N;
}

}  // namespace

// Uploads the L -> l table; called once per handle before any launch (not
// inside stream capture).
cudaError_t opform_init() {
  int h[kMaxNL];
  for (int l = 0; l <= kMaxLmax; ++l)
    for (int L = l * l; L < (l + 1) * (l + 1); ++L) h[L] = l;
  return cudaMemcpyToSymbol(c_l_of_L, h, sizeof(h));
}

cudaError_t launch_opform_H(const OpformArgs& a, bool factored, cudaStream_t st) {
  if (a.n_gtiles == 0) return cudaSuccess;
  const int64_t G = a.g_total;
  dim3 grid(a.n_gtiles, (a.n + kRT - 1) / kRT, factored ? a.n_combo : a.n_atoms);
  if (factored) opform_h_kernel<true><<<grid, 256, 0, st>>>(a, G);
  else opform_h_kernel<false><<<grid, 256, 0, st>>>(a, G);
  return cudaGetLastError();
}

cudaError_t launch_opform_S(const OpformArgs& a, bool factored, cudaStream_t st) {
  if (a.n_gtiles == 0) return cudaSuccess;
  const int64_t G = a.g_total;
  dim3 grid(a.n_gtiles, (a.n + kRT - 1) / kRT, a.n_atoms);
  if (factored) opform_s_kernel<true><<<grid, 256, 0, st>>>(a, G);
  else opform_s_kernel<false><<<grid, 256, 0, st>>>(a, G);
  return cudaGetLastError();
}

cudaError_t launch_opform_alg3(const OpformArgs& a, bool factored, bool product, cudaStream_t st) {
  if (a.n_gtiles == 0) return cudaSuccess;
  const int64_t G = a.g_total;
  dim3 grid(a.n_gtiles, (a.n + kRT - 1) / kRT, factored ? a.n_combo : a.n_atoms);
  if (product && factored) opform_alg3_kernel<true><<<grid, 256, 0, st>>>(a, G);
  if (product && !factored) opform_alg3_kernel<false><<<grid, 256, 0, st>>>(a, G);
  dim3 grid_copy(a.n_gtiles, (a.n + kRT - 1) / kRT, a.n_atoms);
  if (factored) opform_alg3_copy_kernel<true><<<grid_copy, 256, 0, st>>>(a, G);
  else opform_alg3_copy_kernel<false><<<grid_copy, 256, 0, st>>>(a, G);
  return cudaGetLastError();
}

cudaError_t launch_alg_m(const double2* T, int n, int n_L, int n_slots, bool alg1, double2* M, double2* work,
                         int* hpd, cudaStream_t st) {
  if (n_slots == 0) return cudaSuccess;
  alg_m_kernel<<<n_slots, 256, 0, st>>>(T, n, n_L, alg1 ? 1 : 0, M, work, hpd);
  return cudaGetLastError();
}

cudaError_t launch_gather_Z(const double2* Zin, int64_t ldz, int K, int N, const int* kmap,
                            int64_t k_alloc, double2* Z, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  dim3 grid((unsigned)((k_alloc + 255) / 256), N);
  gather_z_kernel<<<grid, 256, 0, st>>>(Zin, ldz, K, N, kmap, k_alloc, Z);
  return cudaGetLastError();
}

}  // namespace flapw
