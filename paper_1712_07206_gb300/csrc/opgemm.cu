// H operand formation of the emulated path on the tensor cores (factored
// operands).
//
// For every (T slot s, atom type t) combination present the row block of the
// Hamiltonian operand (Sec. 3: Z_a = C^H [A_a; B_a], 2N_L rows per atom) is
//     P_{s,t}(r, g) = sum_c C^H_s(r, c) W_t(perm_s(c), g),
// W_t = [A_t; B_t] the type's matching coefficients without the atom phase,
// and Z_a = P_{slot(a),type(a)} diag(e^{i K.tau_a}) lands in atom a's
// sigma-grouped operand rows.  The product uses the split-precision scheme of
// the contraction on operands of its own:
//     A(r, c') = conj(C^H_s(r, c)) with c' = perm_s(c)     (rows r, k = c')
//     B(g, c') = W_t(c', g)                                  (rows g, k = c')
// both cut into kOpSlices = 8 digit slices with per-row scaling (slicer.cu),
// so that the contraction's complex combination conj(A)^T B gives C^H W.
// With 8 slices the dropped pairs (i + j >= 8) weigh below 2^-53 of the
// scaled product, about FP64 rounding.
//
// The reduction is short, K = 2N_L <= 384 (lmax <= 12), so all slice pairs of
// one level t = i + j sum exactly in one FP32 TMEM accumulator: a term of
// level t is at most 2 x 2^13 + (t - 1) x 2^12 (only the pairs (0, t), (t, 0)
// hold a leading digit; (0, 0) alone is 2^14), and 384 x (2^14 + 6 x 2^12) <
// 2^24.  A tile so takes 2 x kOpSlices accumulations (an R and an I pass per
// level) instead of one per slice pair, each drained into the 64-bit
// fixed-point accumulators as in the contraction.
//
// The tiles leave P in fixed point (64-bit integers with the scale exponents
// of its row and plane wave, [combo][g][r]); opgemm_phase_kernel then writes
// every atom's operand rows with the atom's phase, on the integer pipes.
//
// The same product forms the operands of the paper's Alg. 3 (Sec. 5.1) with
// A(r, c) = conj(M_s(r, c)), M = [[T^BA, T^BB / 2], [T^AA, 0]] (alg3.cuh): the
// phase kernel then places row r in column N_L + r of R_a and, for r < N_L,
// in column r of L_a.
//
// CTA tile: 128 rows r x 64 plane waves g; M = 128, N = 128 MMAs (cta_group::1)
// with B = [Re W_j; Im W_j] for the 64 plane waves; 128-wide K stages (two
// 64-wide chunks of any slice pair of the current level).  Four 128-column
// TMEM accumulators rotate over the (level, pass) steps.  Warp roles: 0 TMA
// producer, 1 TMEM allocator and MMA issuer, 2..9 drain and epilogue (warp w
// reads TMEM lanes 32 (w % 4)..+31 and owns plane waves 32 ((w - 2) / 4)..+31
// of the tile, Re and Im).  Every wait is bounded; on expiry the CTA records
// an error, lets its copies and MMAs complete, frees TMEM and exits.
#include <algorithm>
#include <cstdint>

#include "alg3.cuh"
#include "fixed64.cuh"
#include "tc_common.cuh"

namespace flapw {
namespace {

using namespace tc;

constexpr int kThreads = 320;
constexpr int kStages = 3;
constexpr int kStageChunks = 2;
constexpr uint32_t kTileA = 128 * 128;  // 128 rows x 64 k fp16
constexpr uint32_t kTileB = 128 * 128;  // Re and Im planes x 64 plane waves x 64 k
constexpr uint32_t kOffB = kStageChunks * kTileA;
constexpr uint32_t kStageBytes = kStageChunks * (kTileA + kTileB);
constexpr int kBufs = 4;                // TMEM accumulators of 128 columns
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxKChunks = 6;          // K = 2 N_L <= 384
constexpr int kFrac = 50;               // fixed-point fraction bits (sums < 2 x 384)

// D = F32, A = B = F16, K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// The (level t, pass p) steps of a tile, each the chunk sequence q =
// i * kc + c (slice pair (i, t - i), 64-wide K chunk c), cut into stages of
// two chunks.  Every role walks the same order.
struct OpCursor {
  int kc, t, p, q, nq;
  __device__ void begin(int kchunks) {
    kc = kchunks;
    t = 0;
    p = 0;
    q = 0;
    nq = kc;
  }
  __device__ int nv() const { return min(kStageChunks, nq - q); }
  __device__ bool last_in_step() const { return q + kStageChunks >= nq; }
  __device__ bool next_stage() {
    q += kStageChunks;
    if (q < nq) return true;
    q = 0;
    if (++p == 2) {
      p = 0;
      if (++t >= kOpSlices) return false;
    }
    nq = (t + 1) * kc;
    return true;
  }
};

__global__ void __launch_bounds__(kThreads, 1)
    opgemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                  const OpGemmArgs g, const OpTile* __restrict__ tiles, int n_tiles,
                  int* __restrict__ err, unsigned long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  // bars: full[kStages], empty[kStages], tfull[kBufs], tempty[kBufs], drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16);
  int* abort_word = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * kStages + kBufs + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 2 * kBufs);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 8);  // one arrival per drain warp
    }
    mbar_init(drain_bar, 1);
    *abort_word = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const Abort ab{abort_word, 0u, false, wait_ns};

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const OpTile T = tiles[tile];
        const int rowA = g.combo_slot[T.combo] * g.n + T.rb * 128;
        const int rowB = (int)(g.combo_type[T.combo] * g.G) + T.gb * 64;
        OpCursor cur;
        cur.begin(g.kchunks);
        do {
          const int nv = cur.nv();
          const int stage = it % kStages;
          if (!mbar_wait(empty_bar(stage), ((it / kStages) & 1u) ^ 1u, ab)) {
            ok = false;
            break;
          }
          const uint32_t sbase = smem_u32(smem + stage * kStageBytes);
          const uint32_t fb = full_bar(stage);
          mbar_expect_tx(fb, (uint32_t)nv * (kTileA + kTileB));
          for (int v = 0; v < nv; ++v) {
            const int qq = cur.q + v, i = qq / cur.kc, kc = (qq % cur.kc) * kChunk;
            tma_load_4d(sbase + v * kTileA, &map_a, fb, kc, rowA, cur.p, i);
            tma_load_4d(sbase + kOffB + v * kTileB, &map_b, fb, kc, rowB, 0, cur.t - i);
          }
          ++it;
        } while (cur.next_stage());
      }
      if (!ok) {
        for (uint32_t q = (it > kStages ? it - kStages : 0); q < it; ++q)
          mbar_wait_bounded(full_bar(q % kStages), (q / kStages) & 1u);
        atomicExch(err, FLAPW_ERR_TIMEOUT);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t it = 0, step = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        OpCursor cur;
        cur.begin(g.kchunks);
        uint32_t d = 0;
        int buf = 0;
        do {
          if (cur.q == 0) {
            buf = step % kBufs;
            if (!mbar_wait(tempty_bar(buf), ((step / kBufs) & 1u) ^ 1u, ab)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d = tmem_base + (uint32_t)buf * 128u;
          }
          const int stage = it % kStages;
          if (!mbar_wait(full_bar(stage), (it / kStages) & 1u, ab)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sbase = smem_u32(smem + stage * kStageBytes);
          const int nv = cur.nv();
          for (int v = 0; v < nv; ++v) {
            const uint64_t da = sdesc(sbase + v * kTileA), db = sdesc(sbase + kOffB + v * kTileB);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              umma(d, da + 2 * kk, db + 2 * kk, (cur.q > 0 || v > 0 || kk > 0) ? 1u : 0u);
          }
          umma_commit(empty_bar(stage));
          ++it;
          if (cur.last_in_step()) {
            umma_commit(tfull_bar(buf));
            ++step;
          }
        } while (cur.next_stage());
      }
      umma_commit(drain_bar);
      mbar_wait_bounded(drain_bar, 0);
      if (!ok) atomicExch(err, FLAPW_ERR_TIMEOUT);
    }
  } else {
    // ---------------- drain + epilogue ----------------
    const int q4 = warp & 3;          // TMEM lane quadrant
    const int hc = (warp - 2) >> 2;   // plane waves 32 hc .. 32 hc + 31 of the tile
    uint32_t step = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      const OpTile T = tiles[tile];
      long long acc[64];  // [0, 32): Re, [32, 64): Im
#pragma unroll
      for (int n = 0; n < 64; ++n) acc[n] = 0;
      for (int t = 0; t < kOpSlices && ok; ++t) {
        const int sh = kFrac - kSliceBits * (t + 2);
        for (int p = 0; p < 2; ++p) {
          const int buf = step % kBufs;
          if (!mbar_wait(tfull_bar(buf), (step / kBufs) & 1u, ab)) {
            ok = false;
            break;
          }
          tc_fence_after();
          __syncwarp();
          const uint32_t tb = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)buf * 128u +
                              (uint32_t)hc * 32u;
          // accumulator columns: [0, 64) A_p x Re W, [64, 128) A_p x Im W
          // R pass: Re += RR, Im += RI;  I pass: Re += II, Im -= IR
          if (p == 0) {
            drain_fixed<32>(tb, acc, 0, sh, false);
            drain_fixed<32>(tb + 64u, acc, 32, sh, false);
          } else {
            drain_fixed<32>(tb + 64u, acc, 0, sh, false);
            drain_fixed<32>(tb, acc, 32, sh, true);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty_bar(buf));
          ++step;
        }
      }
      if (!ok) break;
      // P(r, g) in fixed point, scale 2^(e_r + e_g - kFrac): [combo][g][r]
      const int r = T.rb * 128 + q4 * 32 + lane;
      if (r < g.n) {
        const int64_t gi0 = (int64_t)T.gb * 64 + hc * 32;
        longlong2* prow = g.P + ((int64_t)T.combo * g.G + gi0) * g.n + r;
#pragma unroll
        for (int n = 0; n < 32; ++n)
          if (gi0 + n < g.G) prow[(int64_t)n * g.n] = make_longlong2(acc[n], acc[32 + n]);
      }
    }
    if (!ok) atomicExch(err, FLAPW_ERR_TIMEOUT);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// A(slot n + r, perm_s(c)) = conj(C^H_s(r, c)); columns n..kp-1 zero.
// grid: n_slots * n rows.
__global__ void __launch_bounds__(128) opgemm_build_a_kernel(const double2* __restrict__ CH,
                                                             const int* __restrict__ perm, int n,
                                                             int kp, double2* __restrict__ A) {
  const int row = blockIdx.x, slot = row / n, r = row % n;
  const double2* src = CH + ((int64_t)slot * n + r) * n;
  const int* pm = perm + (int64_t)slot * n;
  double2* dst = A + (int64_t)row * kp;
  for (int c = threadIdx.x; c < kp; c += blockDim.x) {
    if (c < n) {
      const double2 v = src[c];
      dst[pm[c]] = make_double2(v.x, -v.y);
    } else {
      dst[c] = make_double2(0.0, 0.0);
    }
  }
}

// A(slot n + r, c) = conj(M_s(r, c)) for Alg. 3 or Alg. 1 (M from
// alg_m_kernel); columns n..kp-1 zero.  grid: n_slots * n rows.
__global__ void __launch_bounds__(128) opgemm_build_a_alg3_kernel(const double2* __restrict__ M,
                                                                  int n, int kp,
                                                                  double2* __restrict__ A) {
  const int row = blockIdx.x, slot = row / n, r = row % n;
  const double2* Ms = M + ((int64_t)slot * n + r) * n;
  double2* dst = A + (int64_t)row * kp;
  for (int c = threadIdx.x; c < kp; c += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (c < n) {
      const double2 m = Ms[c];
      v = make_double2(m.x, -m.y);
    }
    dst[c] = v;
  }
}

// B(t G + gi, c) = W_t(c, gi) = [Yc(L, gi) a_l(t, gi); Yc(L, gi) b_l(t, gi)];
// columns n..kp-1 zero.  A 32 plane-wave x 32 column tile per CTA goes
// through shared memory so that both the reads (plane waves contiguous) and
// the writes (columns contiguous) are coalesced.  grid: (ceil(G/32),
// ceil(kp/32), n_types), 32 x 8 threads.
__global__ void __launch_bounds__(256) opgemm_build_b_kernel(const double2* __restrict__ Yc,
                                                             const double* __restrict__ al,
                                                             const double* __restrict__ bl,
                                                             int n_L, int lmax, int n, int kp,
                                                             int64_t G, double2* __restrict__ B) {
  __shared__ double2 tile[32][33];
  const int t = blockIdx.z;
  const int64_t g0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc;
    const int64_t gi = g0 + tx;
    double2 w = make_double2(0.0, 0.0);
    if (c < n && gi < G) {
      const int L = (c < n_L) ? c : c - n_L;
      int l = 0;  // L = l^2 + (l + m)
      while ((l + 1) * (l + 1) <= L) ++l;
      const double2 y = Yc[(int64_t)L * G + gi];
      const int64_t ro = ((int64_t)t * (lmax + 1) + l) * G + gi;
      const double rad = (c < n_L) ? al[ro] : bl[ro];
      w = make_double2(y.x * rad, y.y * rad);
    }
    tile[tx][cc] = w;
  }
  __syncthreads();
  for (int gg = ty; gg < 32; gg += 8) {
    const int64_t gi = g0 + gg;
    const int c = c0 + tx;
    if (gi < G && c < kp) B[((int64_t)t * G + gi) * kp + c] = tile[gg][tx];
  }
}

// Z(h_row0 + g, column of (a, r)) = P_{slot(a),type(a)}(r, g) e^{i K.tau_a}
// for every atom a of a combination: the Q62 phase product of the fixed-point
// P, then the FP64 value built from its bits (no FP64 arithmetic).  The column
// is the sigma-grouped one of the factorisation, or for Alg. 3 column
// N_L + r of the R row (r_row0 + g) and, for r < N_L, column r of the L row.
// grid: (G, combos), 128 threads over the rows r.
__global__ void __launch_bounds__(128) opgemm_phase_kernel(const OpGemmArgs g) {
  const int64_t gi = blockIdx.x;
  const int combo = blockIdx.y;
  const int slot = g.combo_slot[combo], type = g.combo_type[combo];
  const int eb = g.rexp_b[type * g.G + gi] - kFrac;
  const int np = g.alg3_nl ? g.n : g.npos[slot];
  const int a0 = g.combo_start[combo], a1 = g.combo_start[combo + 1];
  double2* zrow = g.Z + (g.h_row0 + gi) * g.k_alloc;
  double2* zrow_r = g.Z + (g.r_row0 + gi) * g.k_alloc;
  const longlong2* prow = g.P + ((int64_t)combo * g.G + gi) * g.n;
  const int nL = g.alg3_nl;
  const bool y_in_l = g.hpd && g.hpd[slot];
  for (int r = threadIdx.x; r < g.n; r += blockDim.x) {
    const int rr = nL ? r : g.outrow[slot * g.n + r];  // sigma-grouped position
    if (rr < 0) continue;                               // zero pivot: the row carries nothing
    const longlong2 P = prow[r];
    const int ex = g.rexp_a[slot * g.n + r] + eb;
    for (int ai = a0; ai < a1; ++ai) {
      const int a = g.combo_atoms[ai];
      const double2 f = g.ph[(int64_t)a * g.G + gi];
      const long long qr = fx::fixed_point(f.x, 62), qi = fx::fixed_point(f.y, 62);
      const long long zr = fx::mul_q62(P.x, qr) - fx::mul_q62(P.y, qi);
      const long long zi = fx::mul_q62(P.x, qi) + fx::mul_q62(P.y, qr);
      const double2 z = make_double2(fx::to_double(zr, ex), fx::to_double(zi, ex));
      if (nL) {
        const int64_t base = (int64_t)a * 3 * nL;
        zrow_r[base + nL + r] = z;
        if (r < nL) zrow[base + r] = z;
        else if (y_in_l) zrow[base + nL + r] = z;  // Alg. 1 with C^H: Y in L too
      } else {
        zrow[(rr < np) ? g.pos_off[a] + rr : g.kpk[0] + g.neg_off[a] + (rr - np)] = z;
      }
    }
  }
}

// round(z 2^sh) for an integer z (half away from zero), 0 below 2^-63,
// clamped to |X| <= lim.
__device__ __forceinline__ long long shift_round(long long z, int sh, long long lim) {
  long long x;
  if (sh >= 0) {
    x = (sh >= 62) ? 0 : z << sh;  // only zero entries of a row reach sh >= 62
  } else {
    const int r = -sh;
    if (r > 62) return 0;
    const unsigned long long m = (z < 0) ? 0ull - (unsigned long long)z : (unsigned long long)z;
    x = (long long)((m + (1ull << (r - 1))) >> r);
    if (z < 0) x = -x;
  }
  return x > lim ? lim : (x < -lim ? -lim : x);
}

// The NS balanced base-128 digits of X (|X| <= 2^{7 NS}, NS >= 4; the digits
// of slicer.cu), written as fp16 values to dst[i * stride], on 32-bit integers:
// X = hi 2^28 + lo with 0 <= lo < 2^28; the low min(4, NS - 1) digits come
// from lo, their carry goes into hi, the rest from hi.
template <int NS>
__device__ __forceinline__ void put_digits(long long X, __half* dst, int64_t stride) {
  constexpr int kLo = (NS - 1 < 4) ? NS - 1 : 4;
  int x = (int)(X & 0xFFFFFFFll);
  int y = (int)(X >> 28);
#pragma unroll
  for (int j = 0; j < kLo; ++j) {
    const int a = ((x + 64) & 127) - 64;
    dst[(NS - 1 - j) * stride] = __float2half_rn(fx::small_int_to_float(a));
    x = (x - a) >> kSliceBits;
  }
  y = y * (1 << (28 - kSliceBits * kLo)) + x;
#pragma unroll
  for (int i = NS - 1 - kLo; i >= 1; --i) {
    const int a = ((y + 64) & 127) - 64;
    dst[i * stride] = __float2half_rn(fx::small_int_to_float(a));
    y = (y - a) >> kSliceBits;
  }
  dst[0] = __float2half_rn(fx::small_int_to_float(y));
}

// put_digits for two adjacent columns: digit i of X0 and of X1 go out as one
// fp16 pair to dst2[i * stride2] (4-byte stores; dst2 4-byte aligned).
template <int NS>
__device__ __forceinline__ void put_digits2(long long X0, long long X1, __half2* dst2, int64_t stride2) {
  constexpr int kLo = (NS - 1 < 4) ? NS - 1 : 4;
  int x0 = (int)(X0 & 0xFFFFFFFll), x1 = (int)(X1 & 0xFFFFFFFll);
  int y0 = (int)(X0 >> 28), y1 = (int)(X1 >> 28);
#pragma unroll
  for (int j = 0; j < kLo; ++j) {
    const int a0 = ((x0 + 64) & 127) - 64, a1 = ((x1 + 64) & 127) - 64;
    dst2[(NS - 1 - j) * stride2] = __floats2half2_rn(fx::small_int_to_float(a0), fx::small_int_to_float(a1));
    x0 = (x0 - a0) >> kSliceBits;
    x1 = (x1 - a1) >> kSliceBits;
  }
  y0 = y0 * (1 << (28 - kSliceBits * kLo)) + x0;
  y1 = y1 * (1 << (28 - kSliceBits * kLo)) + x1;
#pragma unroll
  for (int i = NS - 1 - kLo; i >= 1; --i) {
    const int a0 = ((y0 + 64) & 127) - 64, a1 = ((y1 + 64) & 127) - 64;
    dst2[i * stride2] = __floats2half2_rn(fx::small_int_to_float(a0), fx::small_int_to_float(a1));
    y0 = (y0 - a0) >> kSliceBits;
    y1 = (y1 - a1) >> kSliceBits;
  }
  dst2[0] = __floats2half2_rn(fx::small_int_to_float(y0), fx::small_int_to_float(y1));
}

// Smallest k with |(x, y)| < 2^k (0 for x = y = 0), |x|, |y| < 2^62: the bit
// length of x^2 + y^2 in 128-bit integer arithmetic, halved upwards.
__device__ __forceinline__ int mag_bits(long long x, long long y) {
  const unsigned long long ax = (x < 0) ? 0ull - (unsigned long long)x : (unsigned long long)x;
  const unsigned long long ay = (y < 0) ? 0ull - (unsigned long long)y : (unsigned long long)y;
  const unsigned long long lx = ax * ax, hx = __umul64hi(ax, ax);
  const unsigned long long ly = ay * ay, hy = __umul64hi(ay, ay);
  const unsigned long long lo = lx + ly;
  const unsigned long long hi = hx + hy + (lo < lx ? 1ull : 0ull);
  const int bl = hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 0);
  return (bl + 1) >> 1;
}

// The H operand rows of the factored emulated path straight into the
// contraction's slices: for plane wave g, every atom's entries
// Z(g, column of (a, r)) = P_{slot(a),type(a)}(r, g) e^{i K.tau_a} are formed on
// the integer pipes (Q62 phase products of the fixed-point P, as in
// opgemm_phase_kernel) and, without an FP64 copy of Z, rounded to the row's
// fixed point X = round(Z 2^{7 NS - e_g}) and written as NS balanced base-128
// fp16 digits per plane, the layout and digits of slicer.cu
// (SL[slice][plane][row][k]).  The row exponent e_g bounds every entry:
// |Re Z|, |Im Z| <= |Z| = |P| (|e^{i K.tau}| = 1), so e_g is the largest
// exact bit length of |P| over the row's (combination, r), at most one bit
// above the slicer's max(|Re|, |Im|); X is clamped to 2^{7 NS} against the
// phase's rounding.  Padding columns of the sigma-grouped K layout get zero
// digits.  grid: G (one CTA per plane wave), 256 threads: warp w takes atoms
// w, w + 8, ... of a combination, its lanes consecutive sigma-grouped rows
// (consecutive columns).
template <int NS>
__global__ void __launch_bounds__(256) opgemm_slice_kernel(const OpGemmArgs g, int n_combo,
                                                           __half* __restrict__ SL, int64_t rows,
                                                           int* __restrict__ rexp) {
  __shared__ long long px[kMaxNL * 2], py[kMaxNL * 2];
  __shared__ int pe[kMaxNL * 2];
  __shared__ int red[8];
  const int64_t gi = blockIdx.x;
  const int64_t row = g.h_row0 + gi;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.n;
  const int64_t plane_stride = rows * g.k_alloc;
  __half* srow = SL + row * g.k_alloc;
  // the row exponent from |P|
  int e_row = -100000;
  for (int combo = 0; combo < n_combo; ++combo) {
    const int slot = g.combo_slot[combo], type = g.combo_type[combo];
    const int eb = g.rexp_b[type * g.G + gi] - kFrac;
    for (int r = tid; r < n; r += blockDim.x) {
      if (g.outrow[slot * n + r] < 0) continue;
      const longlong2 P = g.P[((int64_t)combo * g.G + gi) * n + r];
      if (P.x != 0 || P.y != 0) e_row = max(e_row, mag_bits(P.x, P.y) + g.rexp_a[slot * n + r] + eb);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e_row = max(e_row, __shfl_xor_sync(0xffffffffu, e_row, o));
  if (lane == 0) red[warp] = e_row;
  __syncthreads();
  e_row = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) e_row = max(e_row, red[w]);
  if (e_row == -100000) e_row = 0;  // an all-zero row
  if (tid == 0) rexp[row] = e_row;
  const long long lim = 1ll << (kSliceBits * NS);
  for (int combo = 0; combo < n_combo; ++combo) {
    const int slot = g.combo_slot[combo], type = g.combo_type[combo];
    const int eb = g.rexp_b[type * g.G + gi] - kFrac;
    const int np = g.npos[slot];
    __syncthreads();  // the previous combination's rows are consumed
    for (int r = tid; r < n; r += blockDim.x) {
      const int rr = g.outrow[slot * n + r];
      if (rr >= 0) {
        const longlong2 P = g.P[((int64_t)combo * g.G + gi) * n + r];
        px[rr] = P.x;
        py[rr] = P.y;
        pe[rr] = g.rexp_a[slot * n + r] + eb;
      }
    }
    // rows with a zero pivot carry nothing: the live rows are np + nneg
    const int cnt = np + g.nneg[slot];
    __syncthreads();
    for (int ai = g.combo_start[combo] + warp; ai < g.combo_start[combo + 1]; ai += 8) {
      const int a = g.combo_atoms[ai];
      const double2 f = g.ph[(int64_t)a * g.G + gi];
      const long long qr = fx::fixed_point(f.x, 62), qi = fx::fixed_point(f.y, 62);
      for (int rr = lane; rr < cnt; rr += 32) {
        const long long Px = px[rr], Py = py[rr];
        const long long zr = fx::mul_q62(Px, qr) - fx::mul_q62(Py, qi);
        const long long zi = fx::mul_q62(Px, qi) + fx::mul_q62(Py, qr);
        const int sh = pe[rr] + kSliceBits * NS - e_row;
        const int64_t col = (rr < np) ? g.pos_off[a] + rr : g.kpk[0] + g.neg_off[a] + (rr - np);
        put_digits<NS>(shift_round(zr, sh, lim), srow + col, 2 * plane_stride);
        put_digits<NS>(shift_round(zi, sh, lim), srow + plane_stride + col, 2 * plane_stride);
      }
    }
  }
  // zero digits in the padding columns [Kp, Kp_pad) and [Kp_pad + Kn, k_alloc)
  const int kp_pad = g.kpk[0], kp = g.kpk[1], kn = g.kpk[2];
  const __half zero = __float2half_rn(0.0f);
  for (int64_t c = tid; c < g.k_alloc; c += blockDim.x) {
    if ((c >= kp && c < kp_pad) || c >= kp_pad + kn) {
#pragma unroll
      for (int pl = 0; pl < 2 * NS; ++pl) srow[pl * plane_stride + c] = zero;
    }
  }
}

// The S operand rows of the factored emulated path straight into the
// contraction's slices (Eq. (s)): Z_S(g, a n + c) = e^{i K.tau_a} W_t(c, g) u_t(c),
// W_t = [A_t; B_t] the type's matching coefficients without the atom phase
// (the operand product's B factor, rows t G + g), u = 1 on the A rows and
// U_{t,l} on the B rows.  Each W_t(c, g) u_t(c) becomes a fixed-point integer
// below 2^60 with an exponent of its own, each atom phase a Q62 integer; the
// products run on the integer pipes and are sliced as in opgemm_slice_kernel
// (the row exponent from |W u|, then the digits).  Columns [N_A n, k_alloc)
// get zero digits.  grid: G; 256 threads: warp w takes atoms w, w + 8, ... of
// a combination, its lanes consecutive c (consecutive columns).
template <int NS>
__global__ void __launch_bounds__(256) sop_slice_kernel(const SopArgs a, __half* __restrict__ SL,
                                                        int64_t rows, int* __restrict__ rexp) {
  __shared__ long long wx[kMaxNL * 2], wy[kMaxNL * 2];
  __shared__ int we[kMaxNL * 2];
  __shared__ int red[8];
  const int64_t gi = blockIdx.x;
  const int64_t row = a.s_row0 + gi;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int64_t plane_stride = rows * a.k_alloc;
  __half* srow = SL + row * a.k_alloc;
  // W_t(c, g) u_t(c) of type t as a fixed-point integer below 2^60 and its exponent
  auto load_w = [&](int t, int c, long long& X, long long& Y, int& E) {
    double2 w = a.W[((int64_t)t * a.G + gi) * a.kpw + c];
    if (c >= a.n_L) {
      const int L = c - a.n_L;
      int l = 0;
      while ((l + 1) * (l + 1) <= L) ++l;
      const double u = a.U[t * (a.lmax + 1) + l];
      w = make_double2(w.x * u, w.y * u);
    }
    const uint64_t m = max(fx::absbits(w.x), fx::absbits(w.y));
    const int e = (m == 0) ? 0 : (int)((m >> 52) & 0x7FF) - 1022;  // |w| < 2^e
    X = fx::fixed_point(w.x, 60 - e);
    Y = fx::fixed_point(w.y, 60 - e);
    E = e - 60;
  };
  // the row exponent from |W u| of the types present
  int e_row = -100000;
  for (int combo = 0; combo < a.n_combo; ++combo) {
    const int t = a.combo_type[combo];
    for (int c = tid; c < n; c += blockDim.x) {
      long long X, Y;
      int E;
      load_w(t, c, X, Y, E);
      if (X != 0 || Y != 0) e_row = max(e_row, mag_bits(X, Y) + E);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e_row = max(e_row, __shfl_xor_sync(0xffffffffu, e_row, o));
  if (lane == 0) red[warp] = e_row;
  __syncthreads();
  e_row = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) e_row = max(e_row, red[w]);
  if (e_row == -100000) e_row = 0;
  if (tid == 0) rexp[row] = e_row;
  const long long lim = 1ll << (kSliceBits * NS);
  for (int combo = 0; combo < a.n_combo; ++combo) {
    const int t = a.combo_type[combo];
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) load_w(t, c, wx[c], wy[c], we[c]);
    __syncthreads();
    for (int ai = a.combo_start[combo] + warp; ai < a.combo_start[combo + 1]; ai += 8) {
      const int at = a.combo_atoms[ai];
      const double2 f = a.ph[(int64_t)at * a.G + gi];
      const long long qr = fx::fixed_point(f.x, 62), qi = fx::fixed_point(f.y, 62);
      // two adjacent columns per lane (n = 2 N_L is even, so an atom's columns
      // start even): each digit of both entries goes out as one fp16 pair
      for (int c = 2 * lane; c < n; c += 64) {
        long long X[2][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const long long Wx = wx[c + q], Wy = wy[c + q];
          const long long zr = fx::mul_q62(Wx, qr) - fx::mul_q62(Wy, qi);
          const long long zi = fx::mul_q62(Wx, qi) + fx::mul_q62(Wy, qr);
          const int sh = we[c + q] + kSliceBits * NS - e_row;
          X[q][0] = shift_round(zr, sh, lim);
          X[q][1] = shift_round(zi, sh, lim);
        }
        const int64_t col = (int64_t)at * n + c;
        put_digits2<NS>(X[0][0], X[1][0], reinterpret_cast<__half2*>(srow + col), plane_stride);
        put_digits2<NS>(X[0][1], X[1][1], reinterpret_cast<__half2*>(srow + plane_stride + col), plane_stride);
      }
    }
  }
  const int64_t k_used = (int64_t)a.n_atoms * n;
  const __half zero = __float2half_rn(0.0f);
  for (int64_t c = k_used + tid; c < a.k_alloc; c += blockDim.x) {
#pragma unroll
    for (int pl = 0; pl < 2 * NS; ++pl) srow[pl * plane_stride + c] = zero;
  }
}

}  // namespace

size_t opgemm_smem_bytes() { return kStages * kStageBytes + 1024 + 256; }

cudaError_t opgemm_init() {
  return cudaFuncSetAttribute(opgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)opgemm_smem_bytes());
}

cudaError_t launch_opgemm_build(const double2* CH, const int* perm, int n_slots, int n, int kp,
                                const double2* Yc, const double* al, const double* bl,
                                int n_L, int lmax, int n_types, int64_t G,
                                double2* A, double2* B, cudaStream_t st, bool build_a) {
  if (build_a) {
    if (n_slots * n > 0) opgemm_build_a_kernel<<<n_slots * n, 128, 0, st>>>(CH, perm, n, kp, A);
  } else if (G > 0 && n_types > 0) {
    dim3 grid((unsigned)((G + 31) / 32), (unsigned)((kp + 31) / 32), (unsigned)n_types);
    opgemm_build_b_kernel<<<grid, 256, 0, st>>>(Yc, al, bl, n_L, lmax, n, kp, G, B);
  }
  return cudaGetLastError();
}

cudaError_t launch_opgemm_build_alg3(const double2* M, int n_slots, int n, int n_L, int kp,
                                     double2* A, cudaStream_t st) {
  (void)n_L;
  if (n_slots * n > 0) opgemm_build_a_alg3_kernel<<<n_slots * n, 128, 0, st>>>(M, n, kp, A);
  return cudaGetLastError();
}

cudaError_t launch_opgemm(const CUtensorMap& map_a, const CUtensorMap& map_b, const OpGemmArgs& g,
                          const OpTile* tiles, int n_tiles, int* err, int max_ctas,
                          unsigned long long wait_ns, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  if (g.kchunks < 1 || g.kchunks > kMaxKChunks) return cudaErrorInvalidValue;
  const int grid = std::max(1, std::min(n_tiles, max_ctas));
  opgemm_kernel<<<grid, kThreads, opgemm_smem_bytes(), st>>>(map_a, map_b, g, tiles, n_tiles, err,
                                                             wait_ns ? wait_ns : kWaitNs);
  return cudaGetLastError();
}

cudaError_t launch_opgemm_slice(const OpGemmArgs& g, int n_combo, int n_slices, __half* SL,
                                int64_t rows, int* rexp, cudaStream_t st) {
  if (g.G == 0 || n_combo == 0) return cudaSuccess;
  if (g.n > 2 * kMaxNL) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)g.G;
  switch (n_slices) {
#define FLAPW_OPSLICE_CASE(NS)                                                            \
  case NS:                                                                                \
    opgemm_slice_kernel<NS><<<grid, 256, 0, st>>>(g, n_combo, SL, rows, rexp);           \
    break;
    FLAPW_OPSLICE_CASE(4)
    FLAPW_OPSLICE_CASE(5)
    FLAPW_OPSLICE_CASE(6)
    FLAPW_OPSLICE_CASE(7)
    FLAPW_OPSLICE_CASE(8)
#undef FLAPW_OPSLICE_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sop_slice(const SopArgs& a, int n_slices, __half* SL, int64_t rows, int* rexp,
                             cudaStream_t st) {
  if (a.G == 0 || a.n_combo == 0) return cudaSuccess;
  if (a.n > 2 * kMaxNL) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)a.G;
  switch (n_slices) {
#define FLAPW_SOPSLICE_CASE(NS)                                                   \
  case NS:                                                                        \
    sop_slice_kernel<NS><<<grid, 256, 0, st>>>(a, SL, rows, rexp);               \
    break;
    FLAPW_SOPSLICE_CASE(4)
    FLAPW_SOPSLICE_CASE(5)
    FLAPW_SOPSLICE_CASE(6)
    FLAPW_SOPSLICE_CASE(7)
    FLAPW_SOPSLICE_CASE(8)
#undef FLAPW_SOPSLICE_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_opgemm_phase(const OpGemmArgs& g, int n_combo, cudaStream_t st) {
  if (g.G == 0 || n_combo == 0) return cudaSuccess;
  opgemm_phase_kernel<<<dim3((unsigned)g.G, (unsigned)n_combo), 128, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace flapw
