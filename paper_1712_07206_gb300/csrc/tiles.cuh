// Lower-triangle cover of the emulated contraction's output, shared by the
// host tile lists (api.cu) and the device-side list of the allocation-free
// entry point (noalloc.cu).
//
// The N_G x N_G output of one problem is cut into 64 x 64 blocks, ncb per
// side.  Column strip j (64 output columns, the B operand of a CTA pair) needs
// the blocks of rows r >= j.  A CTA-pair tile multiplies one strip by four
// 64-row blocks (two per CTA, each CTA's pair loaded as one 128-row box when
// contiguous).  The result is Hermitian (Eqs. (h), (s); also the paper's
// zherkx form of Alg. 3), so a block (r, j) with r < j is the conjugate
// transpose of the lower block (j, r): a strip may take rows above its
// diagonal and write them transposed.  Every strip takes a cyclic window of
// the blocks of its segment, which computes each unordered pair {r, j} of
// block indices exactly once; against tiles of 256 contiguous rows aligned
// to multiples of 256, where the diagonal 256 x 256 squares are computed in
// full, only the diagonal 64 x 64 blocks and each strip's rounding up to a
// multiple of four blocks are computed twice (N_G 3990: 504 tiles against
// 543, 1.037 against 1.117 times the triangle's elements).
//
// Segments: the blocks [0, ncb) are cut into consecutive segments [a, e).  A
// strip j = a + i of segment [a, e), n = e - a, takes the blocks
//   a + (i + d) mod n, d = 0..D_i     (D_i = m for n = 2m + 1; for n = 2m,
//                                       D_i = m if i < m else m - 1)
// and then every block of [e, ncb) (all below its diagonal).  A pair inside
// the segment at cyclic distance d from i is taken by strip i if d <= D_i and
// otherwise by the strip at distance n - d (then n - d <= D); exactly one of
// the two holds.  A segment's end is chosen among its last 8 candidates to
// minimise the padding of its strips and of the rest of the limit; segments
// never cross `limit` (the column split of an H contraction whose first
// columns go to host memory while the rest is computed: the strips below the
// limit then cover all their columns' lower blocks and write no others).
#pragma once

namespace flapw {
namespace cover {

__host__ __device__ inline int window_d(int n, int i) {
  const int m = n >> 1;
  return (n & 1) ? m : (i < m ? m : m - 1);
}

__host__ __device__ inline int pad4(int x) { return (4 - (x & 3)) & 3; }

// Padding blocks of the strips of segment [a, e) when the problem has ncb blocks.
__host__ __device__ inline int seg_waste(int a, int e, int ncb) {
  const int n = e - a, m = n >> 1, below = ncb - e;
  if (n & 1) return n * pad4(m + 1 + below);
  return m * pad4(m + 1 + below) + m * pad4(m + below);
}

// End of the segment that starts at block a and may not cross limit.
__host__ __device__ inline int seg_end(int a, int limit, int ncb) {
  int best_e = limit, best_w = seg_waste(a, limit, ncb);
  for (int r = 1; r <= 7 && limit - r > a; ++r) {
    const int e = limit - r;
    const int w = seg_waste(a, e, ncb) + seg_waste(e, limit, ncb);
    if (w < best_w) {
      best_w = w;
      best_e = e;
    }
  }
  return best_e;
}

// Row block number t of strip j inside segment [a, e), or -1 past its rows.
__host__ __device__ inline int strip_row(int a, int e, int ncb, int j, int t) {
  const int n = e - a, i = j - a, D = window_d(n, i);
  if (t <= D) return a + (i + t) % n;
  t -= D + 1;
  return (t < ncb - e) ? e + t : -1;
}

__host__ __device__ inline int strip_count(int a, int e, int ncb, int j) {
  return window_d(e - a, j - a) + 1 + (ncb - e);
}

// Tiles of strip j of segment [a, e): ceil(count / 4).
__host__ __device__ inline int strip_tiles(int a, int e, int ncb, int j) {
  return (strip_count(a, e, ncb, j) + 3) >> 2;
}

// Row blocks and write mask of tile number t of strip j in segment [a, e).
// Bit b of the mask marks rb[b] as one of the strip's blocks; padding blocks
// (bit clear) repeat a neighbouring block and are not written.
__host__ __device__ inline int strip_tile(int a, int e, int ncb, int j, int t, int (&rb)[4]) {
  const int c = strip_count(a, e, ncb, j);
  int mask = 0, prev = j;
  for (int q = 0; q < 4; ++q) {
    const int r = (4 * t + q < c) ? strip_row(a, e, ncb, j, 4 * t + q) : -1;
    if (r >= 0) {
      rb[q] = r;
      mask |= 1 << q;
    } else {
      rb[q] = (prev + 1 < ncb) ? prev + 1 : prev;
    }
    prev = rb[q];
  }
  return mask;
}

// Segment [a, e) of strip j when the segments are cut at `limit`.
__host__ __device__ inline void segment_of(int ncb, int limit, int j, int& a, int& e) {
  a = 0;
  for (;;) {
    e = seg_end(a, (a < limit) ? limit : ncb, ncb);
    if (j < e || e >= ncb) return;
    a = e;
  }
}

// Calls emit(jb, wmask, rb0, rb1, rb2, rb3) for the tiles of the strips
// [s0, s1) of a problem with ncb blocks per side, segments cut at `limit`
// (ncb for none), strip by strip.
template <class Emit>
__host__ __device__ void for_each_tile(int ncb, int limit, int s0, int s1, Emit&& emit) {
  int a = 0;
  while (a < ncb) {
    const int e = seg_end(a, (a < limit) ? limit : ncb, ncb);
    for (int j = (a > s0 ? a : s0); j < e && j < s1; ++j) {
      const int nt = strip_tiles(a, e, ncb, j);
      for (int t = 0; t < nt; ++t) {
        int rb[4];
        const int mask = strip_tile(a, e, ncb, j, t, rb);
        emit(j, mask, rb[0], rb[1], rb[2], rb[3]);
      }
    }
    a = e;
  }
}

// The aligned cover: the four blocks of a tile are one 256-row block
// 4 ib .. 4 ib + 3 (each CTA's half one 128-row load), every strip takes
// the 256-row blocks that reach its diagonal or below, and blocks above the
// diagonal are computed but not written.  It computes up to three blocks per
// strip twice more than the cyclic cover (N_G 3990: 543 tiles against 504;
// N_G 11996: 4512 against 4443), but the concurrent tiles of a band share
// whole 256-row blocks, which keeps the operand rows of the largest problems
// in L2 better (N_G 11996: 300 against 338 ms for the contraction).
template <class Emit>
__host__ __device__ void for_each_aligned_tile(int ncb, int s0, int s1, Emit&& emit) {
  const int nib = (ncb + 3) / 4;
  for (int j = s0; j < s1; ++j)
    for (int ib = j / 4; ib < nib; ++ib) {
      int mask = 0;
      for (int q = 0; q < 4; ++q)
        if (4 * ib + q >= j) mask |= 1 << q;
      emit(j, mask, 4 * ib, 4 * ib + 1, 4 * ib + 2, 4 * ib + 3);
    }
}

// Covers: 0 by size (the cyclic one up to N_G 8192, the aligned one above),
// 1 cyclic, 2 aligned.
constexpr int kCoverAuto = 0, kCoverCyclic = 1, kCoverAligned = 2;
__host__ __device__ inline int cover_for(int cover, long long ng) {
  return cover == kCoverAuto ? (ng <= 8192 ? kCoverCyclic : kCoverAligned) : cover;
}

// Tile orders of a problem's list: 0 strip by strip; k = 1..5 bands of
// 4 << (k - 1) row blocks (the band of a tile is that of its first row
// block), strip by strip within a band.  Concurrent tiles then share the
// band's rows (the A operand) and a few strips (the B operand) in L2.
constexpr int kNumOrders = 6;
__host__ __device__ inline int order_band(int order) { return order <= 0 ? 0 : 4 << (order - 1); }

// Default order for a cover and the largest N_G.  Cyclic: strip by strip
// (each strip's tiles share its B rows and overlap their neighbours' windows;
// measured on the contraction, N_G 2540..5868: 370 ms against 395 for bands of
// 32 blocks).  Aligned: bands of 32 blocks (2048 rows) up to N_G 16384, bands
// of 8 (512 rows) above, where the operand rows of the concurrent tiles
// outgrow L2 unless they overlap more.
__host__ __device__ inline int default_order(int cover, long long max_ng) {
  if (cover_for(cover, max_ng) == kCoverCyclic) return 0;
  return max_ng <= 16384 ? 4 : 2;
}

}  // namespace cover
}  // namespace flapw
