// Emulated complex-FP64 lower-triangle contraction  X = Z^H diag(sigma) Z  on
// the FP16 tensor cores (tcgen05.mma, TMEM accumulators, TMA operand loads).
// The output rows read the operand rows from Prob::row_base and the output
// columns those from Prob::col_base: the same rows for a Hermitian rank-K
// update, two operands L, R for the paper's Alg. 3 form X = L^H R (its
// zher2k + zherkx, where the result is Hermitian although L != R).
//
// The operand is given as s integer slices per entry (see slicer.cu):
//     Z = 2^{e_row} sum_i d_i 128^{-(i+1)}   (Re and Im planes separately).
// Then X_{G'G} = 2^{e_G' + e_G} sum_{t} 128^{-t} sum_{i+j=t} D_i(G')^H D_j(G),
// and the truncated sum keeps the s(s+1)/2 slice pairs with i + j <= s - 1
// (Ozaki-style split-precision product).  Each slice product is computed
// EXACTLY: a TMEM FP32 accumulator is drained before its sum can pass 2^24 --
// after 1024 terms for the pair (0,0) (digit products <= 2^14), 2048 for the
// pairs (0,j), (i,0) (<= 2^13) and at most kPassChunks*64 for the rest.  Every
// drain converts the FP32 partial sums to integers and adds them, shifted by
// the level of the slice pair, into 64-bit fixed-point accumulators held in
// registers (F fractional bits, F = 61 - ceil(log2 K): with max(|Re|,|Im|) < 1
// per entry a sum of K products stays below 2K, which then fits in 62 bits),
// so the cross-slice, cross-atom accumulation is integer arithmetic rounded
// only where a level's weight falls below 2^-F; FP64 is used once per output
// element at the end.
//
// The kernel runs on CTA pairs (a 2-CTA cluster, tcgen05 cta_group::2).  A
// pair owns an output tile of 256 rows (G') x 64 columns (G) of complex
// output: the 64 columns of one strip against four 64-row blocks, CTA r
// holding blocks rb[2r], rb[2r+1] (one 128-row load when they are adjacent,
// two 64-row loads otherwise) and their accumulators.  The blocks form the
// cyclic cover of tiles.cuh: blocks above the strip's diagonal are written
// conjugate-transposed, so every lower 64 x 64 block is computed once.
// Slice pairs are taken in groups (i; j, j+1) sharing the row slice i.  Per
// 128-wide K stage each CTA loads with TMA (128-byte swizzle), for two 64-wide
// K chunks, one plane of slice i for its 128 rows (the MMA's A) and its half
// of B = [Re_j; Im_j | Re_{j+1}; Im_{j+1}] for the tile's 64 columns (CTA 0 the
// slice j planes, CTA 1 the slice j+1 planes; for a lone slice j, CTA 0 Re_j
// and CTA 1 Im_j).  One thread of CTA 0 issues M=256, N=256 (or 128), K=16
// MMAs that read A and B from both CTAs' shared memory and write each CTA's
// rows into its own TMEM.  Each K sub-span runs twice: an R pass (A = Re_i)
// into accumulator acc_R = [RR_j | RI_j | RR_j+1 | RI_j+1] and an I pass
// (A = Im_i) into acc_I = [IR_j | II_j | IR_j+1 | II_j+1]; the drains add
//     Re += RR (R pass), Re += II (I pass), Im += RI (R pass), Im -= IR (I pass)
// so the two 256-column accumulators also double-buffer each other: the drain
// of one pass overlaps the MMAs of the next.  Against one CTA per tile (M=128)
// the pair halves the B bytes each SM loads per MMA flop, and 128-wide stages
// halve the producer/MMA hand-offs per flop; both bound the tensor pipe's
// occupancy.  Rows with sigma = -1 sit in the K columns from neg_base(kp), the
// next multiple of the 16-wide MMA K step; the MMAs of those steps set the
// descriptor's negate-B bit, so H = Z^H diag(sigma) Z accumulates both signs in
// the same sums and has the schedule of S.
//
// Warp roles (both CTAs): warp 0 TMA producer, warp 1 TMEM allocator (and in
// CTA 0 the MMA issuer), warps 2-3 idle, warps 4..11 drain/epilogue (warp w
// reads TMEM lanes 32*(w%4)..+31; warps 4-7 own Re, 8-11 own Im).  The first
// warpgroup hands registers to the two drain warpgroups (setmaxnreg), whose
// 64 fixed-point accumulators per thread then fit with the loop state; with
// one budget for all roles the spills the compiler placed landed in the
// producer and MMA loops and lengthened every stage hand-off.  Stage and accumulator
// barriers live in CTA 0 (full, tempty) or in both CTAs (empty, tfull,
// signalled by multicast commits).  Persistent pairs walk the tile list.
// Every wait is bounded by a wall-clock limit; on expiry the CTA records an
// error, raises the abort flag of both CTAs, lets its in-flight copies and
// MMAs complete, frees TMEM and exits.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "fixed64.cuh"
#include "tc_common.cuh"

namespace flapw {
namespace {

using namespace tc;

constexpr int kThreads = 384;      // three warpgroups
constexpr int kDrainWarp0 = 4;     // first drain warp (warpgroups 1 and 2)
// Registers per thread after the split: 384 threads x 168 at launch = 64512;
// 128 x 80 + 256 x 208 = 63488 fits (per SM sub-partition: one warp of the
// first warpgroup and two drain warps, 32 x (80 + 2 x 208) = 15872 of 16384).
constexpr int kRegsCtl = 80;
constexpr int kRegsDrain = 208;
constexpr uint32_t kTileA = 128 * 128;                   // A: 128 rows x 128 B, one chunk
constexpr uint32_t kTileB = 128 * 128;                   // this CTA's B half: <= 128 rows
constexpr uint32_t kTmemCols = 512;
// Two pipeline shapes, both about 192 KB of shared memory: 3 stages of two
// 64-wide K chunks (fewer stage hand-offs per MMA) and 5 stages of one chunk
// (more loads in flight to hide DRAM latency when the operand rows of the
// concurrent tiles outgrow L2).  Config 2 (N_G 3990): 6.06 against 6.48 ms;
// config 3 (N_G 11996): 314.8 against 303.2 ms.
template <int STAGES, int CHUNKS>
struct Pipe {
  static constexpr int kStages = STAGES;
  static constexpr int kStageChunks = CHUNKS;                       // 64-wide K chunks per stage
  static constexpr uint32_t kOffB = CHUNKS * kTileA;               // B after the A chunks
  static constexpr uint32_t kStageBytes = CHUNKS * (kTileA + kTileB);
  static constexpr size_t kSmemBytes = (size_t)STAGES * kStageBytes + 1024 + 256;
  static_assert(2 * STAGES + 5 <= 16, "the mbarriers share 128 bytes before the TMEM slot");
};
using PipeShallow = Pipe<3, 2>;
using PipeDeep = Pipe<5, 1>;
constexpr int kMaxS = 8;
// longest K sub-span of a pass: 48 chunks (3072 terms <= 2^12, exact) let a
// 2592-term reduction take one sub-span per group; 32 cost config 2 1.2 %
constexpr int kPassChunks = 48;
constexpr int kMaxDevices = 64;

// instruction descriptors: D = F32, A = B = F16, K-major both, M = 256, N = 256 / 128
constexpr uint32_t kIdesc256 = (1u << 4) | (0u << 7) | (0u << 10) | ((256u >> 3) << 17) |
                               ((256u >> 4) << 24);
constexpr uint32_t kIdesc128 = (1u << 4) | (0u << 7) | (0u << 10) | ((128u >> 3) << 17) |
                               ((256u >> 4) << 24);
constexpr uint32_t kNegateB = 1u << 14;  // instruction descriptor: D += A (-B)

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA tile load into this CTA's shared memory, completion counted on a
// barrier of either CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t cbar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(cbar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// One pair MMA: A rows from both CTAs (128 each), B halves from both CTAs,
// D rows into each CTA's TMEM at the same address.
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
// Arrive on the barrier at this offset in both CTAs once the MMAs issued so
// far have completed.
__device__ __forceinline__ void umma_commit_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"((uint16_t)3)
      : "memory");
}
// Slice pairs (i, j), 0-based, are visited by level: t = i + j = 0..s-1
// (i.e. 1-based levels i + j + 2 <= s + 1), i = 0..t.  Every role walks the
// same order.

// K units: the chunks [0, k_chunks(kp, kn)) holding the sigma = +1 rows from
// column 0 and the sigma = -1 rows from column neg_base(kp), a multiple of the
// 16-wide MMA K step (the MMAs of the steps from there on negate B, so both
// signs accumulate in one sum, bounded by the magnitudes alone), cut into the
// fewest equal units of at most kUnitChunks.
struct Units {
  int kns;       // first 16-wide K step of the sigma = -1 rows
  int cb, ce;    // the chunk window of this tile part: [cb, ce)
  __device__ int total() const { return ce - cb; }
  __device__ int count() const { return (total() + kUnitChunks - 1) / kUnitChunks; }
  // unit u -> [c0, c1) chunk range
  __device__ void get(int u, int& c0, int& c1) const {
    const int n = count(), t = total();
    c0 = cb + (int)((long long)u * t / n);
    c1 = cb + (int)((long long)(u + 1) * t / n);
  }
};

// Chunks (64 terms each) a TMEM accumulator may sum exactly for slice pair
// (i, j): the leading digit is up to 128 in magnitude, later digits up to 64.
__device__ __forceinline__ int pair_span(int i, int j) {
  return (i == 0 && j == 0) ? kUnitChunks / 4 : (i == 0 || j == 0) ? kUnitChunks / 2 : kUnitChunks;
}

// A tile's K chunks, or part `part` of `parts` equal parts of them (a tile of
// the last wave split over several pairs; EmuTile::split).
__device__ __forceinline__ Units units_of(const Prob& P, int split) {
  Units u;
  u.kns = neg_base(P.kp) / kSignAlign;
  const int parts = split_parts(split), part = split_part(split), t = k_chunks(P.kp, P.kn);
  u.cb = (int)((long long)part * t / parts);
  u.ce = (int)((long long)(part + 1) * t / parts);
  return u;
}

// The drain steps of one tile, in the order every role walks them: for each
// K unit (<= kUnitChunks chunks), for each slice group
// (i; j, j+1) with i + j + 1 <= s - 1, for each sub-span of the unit, an R
// pass then an I pass.  A sub-span is as long as both pairs of the group may
// accumulate exactly (and at most kPassChunks).
struct Sched {
  Units U;
  int s, nu;
  int u, c0, c1;
  int i, j, two;
  int nsub, k;  // sub-spans of the unit for this group, current one
  int s0, s1, pass;

  __device__ int bound(int m) const { return c0 + (int)((long long)m * (c1 - c0) / nsub); }
  __device__ void set_group() {
    two = (j + 1 <= s - 1 - i) ? 1 : 0;
    int span = pair_span(i, j);
    if (two) span = min(span, pair_span(i, j + 1));
    span = min(span, kPassChunks);
    nsub = (c1 - c0 + span - 1) / span;
    k = 0;
    s0 = c0;
    s1 = bound(1);
  }
  __device__ bool begin(const Units& units, int n_slices) {
    U = units;
    s = n_slices;
    nu = U.count();
    u = 0;
    if (nu == 0) return false;
    U.get(0, c0, c1);
    i = 0;
    j = 0;
    pass = 0;
    set_group();
    return true;
  }
  __device__ bool next() {
    if (pass == 0) {
      pass = 1;
      return true;
    }
    pass = 0;
    if (++k < nsub) {
      s0 = s1;
      s1 = bound(k + 1);
      return true;
    }
    j += 2;
    if (j > s - 1 - i) {
      j = 0;
      if (++i >= s) {
        i = 0;
        if (++u >= nu) return false;
        U.get(u, c0, c1);
      }
    }
    set_group();
    return true;
  }
};

// This thread's row of a finished tile of the cyclic cover into the lower
// triangle: output columns gc0 + 32h + n, n < 32, Re in acc[n] and Im in
// acc[32 + n], written as whole complex elements (16-byte stores): in place
// below the strip's diagonal (on and below it in the diagonal block),
// conjugated and transposed above it (element (gr, gc) to (gc, gr); the result
// is Hermitian).  Element n goes to offset o_n, o_{n+1} = o_n + step_n,
// step_{n+1} = step_n + dstep (the packed layout's columns shorten by one).
// Out of line: it runs once per tile, and kept inline it changed how the
// compiler laid out the MMA and load loops (measured 5-10 % on the contraction).
__device__ __noinline__ void write_tile_row(const EmuTile& T, const Prob& P, uint32_t rank, int m, int h,
                                           const long long (&acc)[64], const int* rexp, int frac) {
  const int blk = 2 * (int)rank + (m >> 6);
  const int rbk = (blk & 2) ? ((blk & 1) ? T.rb[3] : T.rb[2]) : ((blk & 1) ? T.rb[1] : T.rb[0]);
  const int64_t ng = P.n_g;
  const int64_t gr = (int64_t)rbk * 64 + (m & 63);
  const int64_t gc0 = (int64_t)T.jb * 64 + 32 * h;
  if (!(((T.wmask >> blk) & 1) && gr < ng)) return;
  const bool packed = P.layout == FLAPW_LAYOUT_LOWER_PACKED;
  const bool trans = rbk < T.jb;
  int64_t o, step, dstep = 0;
  if (trans) {
    o = (packed ? gr * ng - gr * (gr - 1) / 2 - gr : gr * P.ld) + gc0;
    step = 1;
  } else if (packed) {
    o = gc0 * ng - gc0 * (gc0 - 1) / 2 + (gr - gc0);
    step = ng - 1 - gc0;
    dstep = -1;
  } else {
    o = gc0 * P.ld + gr;
    step = P.ld;
  }
  const int64_t lim = trans ? ng - gc0 : min(ng - gc0, gr - gc0 + 1);
  const int nlim = lim < 32 ? (int)lim : 32;
  const int er = rexp[P.row_base + gr] - frac;
  const int* ec = rexp + P.col_base + gc0;
  double2* out = P.out;
#pragma unroll
  for (int n = 0; n < 32; ++n) {
    if (n < nlim) {
      const int e = er + ec[n];
      out[o] = make_double2(fx::to_double(acc[n], e), fx::to_double(trans ? -acc[32 + n] : acc[32 + n], e));
    }
    o += step;
    step += dstep;
  }
}

// The producer's loads of one tile: for every drain step of the tile, its K
// stages (A: plane `pass` of slice i, this CTA's 128 rows; B: this CTA's half
// of the slice group).  SPLIT: the CTA's two 64-row blocks are not adjacent
// and A goes as two 64-row boxes.  `it` counts the stages; false if a wait
// ran out.
template <bool SPLIT, class PP>
__device__ __forceinline__ bool produce_tile(const SliceMaps& maps, const Prob& P, const EmuTile& T,
                                             int rowA0, int rowA1, int rowB, uint32_t rank, int n_slices,
                                             uint8_t* smem, uint32_t bar0, uint32_t& it, const Abort& ab) {
  constexpr int kStages = PP::kStages, kStageChunks = PP::kStageChunks;
  Sched sc;
  for (bool more = sc.begin(units_of(P, T.split), n_slices); more; more = sc.next()) {
    const uint32_t b_bytes = sc.two ? kTileB : kTileB / 2;
    for (int c = sc.s0; c < sc.s1; c += kStageChunks) {
      const int nv = min(kStageChunks, sc.s1 - c);
      const int stage = it % kStages;
      const uint32_t round = it / kStages;
      if (!mbar_wait(bar0 + 8u * (kStages + stage), (round & 1u) ^ 1u, ab)) return false;  // empty
      const uint32_t sbase = smem_u32(smem + stage * PP::kStageBytes);
      const uint32_t fb = bar0 + 8u * stage;  // full
      // CTA 0's barrier counts the bytes of both CTAs
      if (rank == 0) mbar_expect_tx(fb, 2u * (uint32_t)nv * (kTileA + b_bytes));
      const uint32_t cfb = map_to_rank(fb, 0);
      for (int q = 0; q < nv; ++q) {
        const int kc = (c + q) * kChunk;
        if (SPLIT) {
          tma_load_4d(sbase + q * kTileA, &maps.b1, cfb, kc, rowA0, sc.pass, sc.i);
          tma_load_4d(sbase + q * kTileA + kTileA / 2, &maps.b1, cfb, kc, rowA1, sc.pass, sc.i);
        } else {
          tma_load_4d(sbase + q * kTileA, &maps.a, cfb, kc, rowA0, sc.pass, sc.i);
        }
        // B half: slice j + rank, both planes (or plane `rank` of a lone slice j)
        if (sc.two)
          tma_load_4d(sbase + PP::kOffB + q * kTileB, &maps.b2, cfb, kc, rowB, 0, sc.j + (int)rank);
        else
          tma_load_4d(sbase + PP::kOffB + q * kTileB, &maps.b1, cfb, kc, rowB, (int)rank, sc.j);
      }
      ++it;
    }
  }
  return true;
}
// CYC: tiles of the cyclic cover (tiles.cuh: a CTA's two row blocks may be
// apart, blocks above the strip's diagonal are written transposed);
// otherwise tiles of the aligned cover (256-row blocks: one 128-row load per
// CTA, lower parts written in place).  Separate instantiations: the aligned
// one keeps its load loop and epilogue free of the cyclic cover's cases.
template <class PP, bool CYC>
__global__ void __launch_bounds__(kThreads, 1)
    herk_emu_kernel(const __grid_constant__ SliceMaps maps, const Prob* __restrict__ probs,
                    const EmuTile* __restrict__ tiles, int n_tiles, const int* __restrict__ rexp,
                    int n_slices, int frac, int* __restrict__ err, SplitScratch split,
                    unsigned long long wait_ns) {
  constexpr int kStages = PP::kStages;
  constexpr int kStageChunks = PP::kStageChunks;
  constexpr uint32_t kOffB = PP::kOffB;
  constexpr uint32_t kStageBytes = PP::kStageBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  // bars: full[kStages], empty[kStages], tfull[2], tempty[2], drain[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16);
  int* abort_word = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 16);  // one arrival per drain warp of both CTAs
    }
    mbar_init(drain_bar, 1);
    *abort_word = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b2)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b1)) : "memory");
  }
  if (warp == 1) {
    // both CTAs of the pair allocate together: the same columns in each TMEM
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();  // barriers initialised and TMEM allocated in both CTAs
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const Abort ab{abort_word, map_to_rank(smem_u32(abort_word), rank ^ 1u), true, wait_ns};
  if (warp < kDrainWarp0) {
  // the first warpgroup gives registers up (its role code is dominated by this)
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs) {
        const EmuTile T = tiles[tile];
        const Prob P = probs[T.prob];
        const int rowB = P.col_base + T.jb * 64;
        if constexpr (CYC) {
          // this CTA's two 64-row blocks: one 128-row box when adjacent (the
          // common case), else two 64-row boxes, each case a loop of its own
          const int ra0 = rank ? T.rb[2] : T.rb[0], ra1 = rank ? T.rb[3] : T.rb[1];
          const int rowA0 = P.row_base + ra0 * 64;
          if (ra1 == ra0 + 1)
            ok = produce_tile<false, PP>(maps, P, T, rowA0, 0, rowB, rank, n_slices, smem, bar0, it, ab);
          else
            ok = produce_tile<true, PP>(maps, P, T, rowA0, P.row_base + ra1 * 64, rowB, rank, n_slices, smem,
                                        bar0, it, ab);
          continue;
        }
        // aligned cover: this CTA's rows 128 rank .. 128 rank + 127 of the 256-row block
        const int rowA = P.row_base + T.rb[0] * 64 + (int)rank * 128;
        Sched sc;
        for (bool more = sc.begin(units_of(P, T.split), n_slices); more && ok; more = sc.next()) {
          const uint32_t b_bytes = sc.two ? kTileB : kTileB / 2;
          for (int c = sc.s0; c < sc.s1; c += kStageChunks) {
            const int nv = min(kStageChunks, sc.s1 - c);
            const int stage = it % kStages;
            const uint32_t round = it / kStages;
            if (!mbar_wait(empty_bar(stage), (round & 1u) ^ 1u, ab)) {
              ok = false;
              break;
            }
            const uint32_t sbase = smem_u32(smem + stage * kStageBytes);
            const uint32_t fb = full_bar(stage);
            // CTA 0's barrier counts the bytes of both CTAs
            if (rank == 0) mbar_expect_tx(fb, 2u * (uint32_t)nv * (kTileA + b_bytes));
            const uint32_t cfb = map_to_rank(fb, 0);
            for (int q = 0; q < nv; ++q) {
              const int kc = (c + q) * kChunk;
              // A: plane `pass` of slice i, this CTA's 128 rows
              tma_load_4d(sbase + q * kTileA, &maps.a, cfb, kc, rowA, sc.pass, sc.i);
              // B half: slice j + rank, both planes (or plane `rank` of a lone slice j)
              if (sc.two)
                tma_load_4d(sbase + kOffB + q * kTileB, &maps.b2, cfb, kc, rowB, 0, sc.j + (int)rank);
              else
                tma_load_4d(sbase + kOffB + q * kTileB, &maps.b1, cfb, kc, rowB, (int)rank, sc.j);
            }
            ++it;
          }
        }
      }
      if (!ok) {
        // CTA 0 sees both CTAs' copies land on its barriers; the pair's
        // closing cluster barrier keeps CTA 1 resident until then
        if (rank == 0)
          for (uint32_t q = (it > kStages ? it - kStages : 0); q < it; ++q)
            mbar_wait_bounded(full_bar(q % kStages), (q / kStages) & 1u);
        atomicExch(err, FLAPW_ERR_TIMEOUT);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (CTA 0 only) ----------------
    if (lane == 0 && rank == 0) {
      uint32_t it = 0, acc_it = 0;
      bool ok = true;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs) {
        const EmuTile T = tiles[tile];
        const Prob P = probs[T.prob];
        Sched sc;
        for (bool more = sc.begin(units_of(P, T.split), n_slices); more && ok; more = sc.next()) {
          const int buf = acc_it & 1;  // equals sc.pass: R passes use acc_R, I passes acc_I
          const uint32_t use = acc_it >> 1;
          if (!mbar_wait(tempty_bar(buf), (use & 1u) ^ 1u, ab)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)buf * 256u;
          const uint32_t idesc = sc.two ? kIdesc256 : kIdesc128;
          for (int c = sc.s0; c < sc.s1; c += kStageChunks) {
            const int nv = min(kStageChunks, sc.s1 - c);
            const int stage = it % kStages;
            if (!mbar_wait(full_bar(stage), (it / kStages) & 1u, ab)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sbase = smem_u32(smem + stage * kStageBytes);
            for (int q = 0; q < nv; ++q) {
              const uint64_t da = sdesc(sbase + q * kTileA), db = sdesc(sbase + kOffB + q * kTileB);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t id = (4 * (c + q) + kk >= sc.U.kns) ? (idesc | kNegateB) : idesc;  // sigma = -1
                umma_pair(d, da + 2 * kk, db + 2 * kk, id, (c > sc.s0 || q > 0 || kk > 0) ? 1u : 0u);
              }
            }
            umma_commit_both(empty_bar(stage));
            ++it;
          }
          if (!ok) break;
          umma_commit_both(tfull_bar(buf));
          ++acc_it;
        }
      }
      // all MMAs issued so far complete before teardown (both CTAs learn it)
      umma_commit_both(drain_bar);
      mbar_wait_bounded(drain_bar, 0);
      if (!ok) atomicExch(err, FLAPW_ERR_TIMEOUT);
    } else if (lane == 0) {
      // CTA 1: its TMEM is written until CTA 0's last MMA completes
      mbar_wait_bounded(drain_bar, 0);
    }
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsDrain));
    // ---------------- drain + epilogue (256 threads per CTA) ----------------
    const int ew = warp - kDrainWarp0;
    const int q = warp & 3;       // TMEM lane quadrant this warp may access
    const int h = ew >> 2;        // aligned: 0 Re, 1 Im; cyclic: output columns 32h .. 32h + 31
    const int m = q * 32 + lane;  // row within this CTA's 128 rows
    uint32_t acc_it = 0;
    bool ok = true;
    for (int tile = pair; tile < n_tiles && ok; tile += n_pairs) {
      const EmuTile T = tiles[tile];
      const Prob P = probs[T.prob];
      long long acc[64];
#pragma unroll
      for (int n = 0; n < 64; ++n) acc[n] = 0;
      Sched sc;
      for (bool more = sc.begin(units_of(P, T.split), n_slices); more && ok; more = sc.next()) {
        const int buf = acc_it & 1;
        const uint32_t use = acc_it >> 1;
        if (!mbar_wait(tfull_bar(buf), use & 1u, ab)) {
          ok = false;
          break;
        }
        tc_fence_after();
        __syncwarp();  // tcgen05.ld is warp-collective
        // R pass: Re += RR (cols 0..63 of a pair block), Im += RI (64..127);
        // I pass: Re += II (64..127), Im -= IR (0..63).
        if constexpr (CYC) {
          // warp half h owns output columns 32h .. 32h + 31, Re in acc[0..31]
          // and Im in acc[32..63] (whole complex elements for the epilogue)
          const uint32_t rcol = (sc.pass ? 64u : 0u) + 32u * h, icol = (sc.pass ? 0u : 64u) + 32u * h;
          for (int pq = 0; pq <= sc.two; ++pq) {
            const int sh = frac - kSliceBits * (sc.i + sc.j + pq + 2);
            const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * 256u +
                                (uint32_t)pq * 128u;
            drain_fixed<32>(tb + rcol, acc, 0, sh, false);
            drain_fixed<32>(tb + icol, acc, 32, sh, sc.pass == 1);
          }
        } else {
          const uint32_t col = (h == 0) ? (sc.pass ? 64u : 0u) : (sc.pass ? 0u : 64u);
          const bool sub = (h == 1 && sc.pass == 1);
          for (int pq = 0; pq <= sc.two; ++pq) {
            const int sh = frac - kSliceBits * (sc.i + sc.j + pq + 2);
            const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * 256u +
                                (uint32_t)pq * 128u + col;
            drain_fixed<64>(tb, acc, 0, sh, sub);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(map_to_rank(tempty_bar(buf), 0));
        ++acc_it;
      }
      if (!ok) break;
      if (split_parts(T.split) > 1) {
        // This pair summed one K part of the tile: leave the partial sums in
        // the scratch; per drain warp (32 rows x 64 columns of Re or Im) the
        // part that finishes last adds the others' and writes.  Only
        // warp-level synchronisation is involved.
        const int parts = split_parts(T.split), part = split_part(T.split);
        const int64_t base = ((int64_t)split_id(T.split) * 2 + rank) * 8 + ew;  // this warp's slice
        long long* mine = split.partial + ((base * kMaxSplit + part) * 64) * 32 + lane;
#pragma unroll
        for (int n = 0; n < 64; ++n) mine[n * 32] = acc[n];
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          const int done = atomicAdd(split.count + base, 1);
          last = (done == parts - 1);
          if (last) split.count[base] = 0;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) continue;
        __threadfence();
        for (int o = 0; o < parts; ++o) {
          if (o == part) continue;
          const long long* other = split.partial + ((base * kMaxSplit + o) * 64) * 32 + lane;
#pragma unroll
          for (int n = 0; n < 64; ++n) acc[n] += __ldcg(other + n * 32);
        }
      }
      // write this thread's row of the tile: in place below the strip's
      // diagonal (on and below it in the diagonal block), conjugate-
      // transposed into the lower triangle above it.  Element n of the row
      // goes to offset o_n, o_{n+1} = o_n + step_n, step_{n+1} = step_n + dstep.
      if constexpr (CYC) {
        write_tile_row(T, P, rank, m, h, acc, rexp, frac);
        continue;
      }
      // aligned cover: this thread's row of the 256-row block, in place, on
      // and below the diagonal (blocks above it are computed, not written)
      const int64_t ng = P.n_g;
      const int64_t gr = (int64_t)T.rb[0] * 64 + (int64_t)rank * 128 + m;
      if (gr < ng) {
        const int er = rexp[P.row_base + gr];
        double* outd = reinterpret_cast<double*>(P.out);
#pragma unroll
        for (int n = 0; n < 64; ++n) {
          const int64_t gc = (int64_t)T.jb * 64 + n;
          if (gc < ng && gc <= gr) {
            const double val = fx::to_double(acc[n], er + rexp[P.col_base + gc] - frac);
            const int64_t o = (P.layout == FLAPW_LAYOUT_LOWER_PACKED)
                                  ? gc * ng - gc * (gc - 1) / 2 + (gr - gc)
                                  : gc * P.ld + gr;
            outd[2 * o + h] = val;
          }
        }
      }
    }
    if (!ok) atomicExch(err, FLAPW_ERR_TIMEOUT);
  }

  // neither CTA leaves while the other may still touch its shared memory
  settle_after_abort(ab);
  tc_fence_before();
  cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

struct DevState {
  bool ready = false;
  int max_pairs = 0;
};
std::mutex g_state_mutex;
DevState g_state[kMaxDevices];

}  // namespace

size_t herk_emu_smem_bytes(bool deep) { return deep ? PipeDeep::kSmemBytes : PipeShallow::kSmemBytes; }

// partial sums: [id][cta][drain warp][part][64][32] int64; counts: [id][cta][drain warp]
size_t split_scratch_bytes(int n_ids) {
  return (size_t)n_ids * 2 * 8 * (kMaxSplit * 64 * 32 * 8 + 4);
}

int fixed_frac_bits(int64_t k_terms) {
  int lg = 0;
  while (lg < 62 && ((int64_t)1 << lg) < k_terms) ++lg;
  const int f = 61 - lg;  // |sum| < 2K 2^F <= 2^62
  return f < 40 ? 40 : (f > 50 ? 50 : f);  // <= 50: one (0,0) drain, < 2^25 2^(F-14), fits too
}

cudaError_t herk_emu_init() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_state_mutex);
  if (g_state[dev].ready) return cudaSuccess;
  const size_t smem = PipeShallow::kSmemBytes;
  for (auto k : {herk_emu_kernel<PipeShallow, false>, herk_emu_kernel<PipeShallow, true>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  for (auto k : {herk_emu_kernel<PipeDeep, false>, herk_emu_kernel<PipeDeep, true>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeDeep::kSmemBytes);
    if (e != cudaSuccess) return e;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * (sms / 2));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0, nd = 0;
  e = cudaOccupancyMaxActiveClusters(&n, herk_emu_kernel<PipeShallow, false>, &cfg);
  if (e != cudaSuccess) return e;
  cfg.dynamicSmemBytes = PipeDeep::kSmemBytes;
  e = cudaOccupancyMaxActiveClusters(&nd, herk_emu_kernel<PipeDeep, false>, &cfg);
  if (e != cudaSuccess) return e;
  if (n < 1 || nd < 1) return cudaErrorInvalidConfiguration;
  g_state[dev].max_pairs = std::min(n, nd);  // one pair per 2 SMs in both shapes
  g_state[dev].ready = true;
  return cudaSuccess;
}

int herk_emu_pairs(int busy_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || !g_state[dev].ready) return 0;
  return std::max(1, g_state[dev].max_pairs - std::max(0, busy_sms));
}

cudaError_t launch_herk_emu(const SliceMaps& maps, const Prob* probs, const EmuTile* tiles,
                            int n_tiles, const int* rexp, int n_slices, int frac, int* err,
                            int busy_sms, const SplitScratch& split, bool deep, bool cyclic,
                            unsigned long long wait_ns, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  if (n_slices < 1 || n_slices > kMaxS || frac < 40 || frac > 50) return cudaErrorInvalidValue;
  cudaError_t e = herk_emu_init();
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // A persistent pair that cannot be placed at launch starts only when the
  // concurrent work ends and then delays the whole launch; each SM held
  // elsewhere can cost at most one pair its place.
  const int pairs = std::max(1, std::min(n_tiles, g_state[dev].max_pairs - std::max(0, busy_sms)));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = herk_emu_smem_bytes(deep);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  auto k = deep ? (cyclic ? herk_emu_kernel<PipeDeep, true> : herk_emu_kernel<PipeDeep, false>)
                : (cyclic ? herk_emu_kernel<PipeShallow, true> : herk_emu_kernel<PipeShallow, false>);
  e = cudaLaunchKernelEx(&cfg, k, maps, probs, tiles, n_tiles, rexp, n_slices, frac, err, split,
                         wait_ns ? wait_ns : kWaitNs);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

bool make_tmap_4d(CUtensorMap* map, void* base, int64_t k_alloc, int64_t rows, int n_slices,
                  uint32_t box_rows, uint32_t box_planes, std::string* err) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      *err = "cuTensorMapEncodeTiled is not available from the driver";
      return false;
    }
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const cuuint64_t dims[4] = {(cuuint64_t)k_alloc, (cuuint64_t)rows, 2, (cuuint64_t)n_slices};
  const cuuint64_t strides[3] = {(cuuint64_t)k_alloc * 2, (cuuint64_t)(rows * k_alloc * 2),
                                 (cuuint64_t)(2 * rows * k_alloc * 2)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t box[4] = {64, box_rows, box_planes, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *err = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
    return false;
  }
  return true;
}

// Tensor maps over SL[slice][plane][row][k] (fp16), 128-byte swizzle, boxes of
// 64 k by: 128 rows (a), 64 rows x 2 planes (b2), 64 rows (b1).
bool make_slice_tmaps(SliceMaps* maps, void* base, int64_t k_alloc, int64_t rows, int n_slices,
                      std::string* err) {
  return make_tmap_4d(&maps->a, base, k_alloc, rows, n_slices, 128, 1, err) &&
         make_tmap_4d(&maps->b2, base, k_alloc, rows, n_slices, 64, 2, err) &&
         make_tmap_4d(&maps->b1, base, k_alloc, rows, n_slices, 64, 1, err);
}

}  // namespace flapw
