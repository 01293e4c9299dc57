// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "flapw.h"

namespace flapw {

constexpr int kMaxLmax = 12;
constexpr int kMaxNL = (kMaxLmax + 1) * (kMaxLmax + 1);
constexpr int kChunk = 64;        // columns of K per pipeline step (one 128-byte fp16 row)
// The sigma = -1 rows of an operand start at the first multiple of kSignAlign
// at or after the sigma = +1 rows (one tcgen05 MMA K step of fp16), so that the
// two groups together fill whole K chunks up to the last one.
constexpr int kSignAlign = 16;
__host__ __device__ inline int neg_base(int kp) { return (kp + kSignAlign - 1) / kSignAlign * kSignAlign; }
// K chunks of an operand with kp rows of sigma = +1 and kn of sigma = -1.
__host__ __device__ inline int k_chunks(int kp, int kn) { return (neg_base(kp) + kn + kChunk - 1) / kChunk; }
constexpr int kSliceBits = 7;     // magnitude bits per emulation slice
constexpr int kUnitChunks = 64;   // K chunks per unit: the longest exact FP32 accumulation
                                  // (4096 terms, digit products <= 2^12)
constexpr int kOpSlices = 8;      // slices of the H operand formation product

// One lower-triangle contraction problem X = L^H diag(sigma) R: H or S of
// one k-point.  L (the output rows G') and R (the output columns G) are rows
// of the operand / slice arrays; a Hermitian rank-K update has L = R.
struct Prob {
  int row_base;   // first row of L in the operand / slice arrays
  int n_g;        // N_G of the problem
  int kp;         // operand rows (K index) with sigma = +1; columns [0, kp)
  int kn;         // rows with sigma = -1; columns [neg_base(kp), ... + kn)
  int layout;     // FLAPW_LAYOUT_*
  int col_base;   // first row of R (= row_base for L = R)
  int64_t ld;     // leading dimension of the full layout
  double2* out;   // lower triangle, complex128
};

// Output tile of the emulated contraction, computed by a CTA pair: the 64
// columns of strip jb (64-column block) against four 64-row blocks rb[0..3]
// (CTA 0 rb[0], rb[1]; CTA 1 rb[2], rb[3]); see tiles.cuh for the cover.
// Bit b of wmask: block rb[b] is written (clear for padding).  A block
// below the strip's diagonal (rb > jb) is written in place, the diagonal
// block (rb == jb) on and below the diagonal, a block above it (rb < jb)
// conjugate-transposed into the lower triangle.  `split` is 0 for a whole
// tile, or, for one of the `parts` K parts of a tile of the last wave,
// parts | part << 4 | id << 8 (id: the split tile's scratch slot).
struct EmuTile {
  int prob;
  int jb;
  int split;
  int wmask;
  int rb[4];
};
constexpr int kMaxSplit = 4;  // K parts of a split tile
__host__ __device__ inline int split_parts(int s) { return (s & 15) ? (s & 15) : 1; }
__host__ __device__ inline int split_part(int s) { return (s >> 4) & 15; }
__host__ __device__ inline int split_id(int s) { return s >> 8; }
inline int make_split(int parts, int part, int id) { return parts | (part << 4) | (id << 8); }
// Scratch of the split tiles: 64-bit partial sums per (id, cta, drain warp,
// part) and one completion count per (id, cta, drain warp), zero between
// launches (split_scratch_bytes: both, counts after the partial sums).
struct SplitScratch {
  long long* partial;
  int* count;
};
size_t split_scratch_bytes(int n_ids);

// Output tile of the FP64 contraction: 64 x 64.
struct F64Tile {
  int prob;
  int ib;
  int jb;
  int pad;
};

// Per-G data for A/B generation, indexed by the global plane-wave index.
struct GData {
  const int* n3;      // [G_total][3]
  const int* gk;      // [G_total] k-point of each plane wave
  const int64_t* goff;  // [n_k+1]
};

// Geometry on the device.
struct Geom {
  int n_atoms, n_types, lmax, n_L, n_k;
  int64_t g_total;
  const double* rec;        // [9] reciprocal rows b1,b2,b3
  const double* pos;        // [n_atoms][3]
  const int* type;          // [n_atoms]
  const double* radius;     // [n_types]
  const double* kfrac;      // [n_k][3]
  const double* ktau;       // [n_k][n_atoms]: k . tau_frac
  double pref;              // 4 pi / sqrt(Omega)
};

// ---- kernels (launch wrappers) -------------------------------------------

// Per plane wave: Yc[L][g] = pref i^l conj(Y_lm(K_hat)), radial factors
// al/bl[t][l][g], atom phases ph[a][g].
cudaError_t launch_ab_prep(const Geom& geo, const GData& gd, const double* radial,
                           const double* ylm_coef, double2* Yc, double* al, double* bl,
                           double2* ph, cudaStream_t st);
// A/B assembly for all k-points into [k][a][L][G] blocks.
cudaError_t launch_ab_assemble_tiles(const Geom& geo, const int* gtiles, int n_gtiles,
                                     const int64_t* goff, const double2* Yc, const double* al,
                                     const double* bl, const double2* ph, double2* A, double2* B,
                                     cudaStream_t st);

// Bunch-Kaufman LDL^H of each T block: M = |Lambda|^{1/2} Q^H L^H (pivoted
// order), the pivot permutation and each row's place in the sigma-grouped operand.
// cluster: a cluster of CTAs per slot (shorter, more SMs) instead of one CTA.
cudaError_t launch_tfactor(const double2* T, int n, int n_slots, double2* work, double2* CH,
                           int* perm, int* outrow, int* npos, int* nneg, int* npiv2, int* err,
                           bool cluster, cudaStream_t st);

// Atom offsets in the sigma-grouped K order and chunk counts of the H problems.
cudaError_t launch_layout(const int* npos, const int* nneg, const int* atom_slot, int n_atoms,
                          int n_k, int* pos_off, int* neg_off, int* kpk, Prob* probs,
                          int k_total, cudaStream_t st);

struct OpformArgs {
  int n_atoms, n_L, n, n_k;
  const int* atom_slot;
  const int* atom_type;
  const double2* CH;    // [slot][n][n] M in pivoted order (block upper triangular)
  const int* perm;      // [slot][n] W row feeding pivoted column c
  const int* outrow;    // [slot][n] sigma-grouped position of row r, -1 if dropped
  const int* npos;      // [slot]
  const int* nneg;      // [slot]
  const int* pos_off;   // [atom]
  const int* neg_off;   // [atom]
  const int* kpk;       // [0]=Kp_pad (start of the negative block)
  const double* U;      // [type][lmax+1]
  int lmax;
  int64_t k_alloc;      // row stride of Z (complex elements)
  double2* Z;           // operand rows
  const int* gtiles;    // [n_gtiles][2] = (k, g0)
  int n_gtiles;
  const int64_t* goff;  // [n_k+1]
  int64_t g_total;      // plane waves over all k-points
  int64_t h_row0;       // operand row of the first H plane wave (k-point 0)
  int64_t s_row0;       // operand row of the first S plane wave
  int64_t r_row0;       // the paper's Alg. 3: operand row of the first right-hand H row
  const double2* T;     // the paper's Alg. 3: [slot][n][n] row-major T blocks (lower read)
  const double2* M;     // Alg. 3 / Alg. 1: [slot][n][n] row-major operand matrices (alg_m)
  const int* hpd;       // Alg. 1: [slot] Cholesky of T^AA succeeded; null for Alg. 3
  // from A/B
  const double2* A;
  const double2* B;
  // factored
  const double2* Yc;
  const double* al;
  const double* bl;
  const double2* ph;
  int n_types;
  const int* combo_slot;   // [n_combo]
  const int* combo_type;   // [n_combo]
  const int* combo_atoms;  // atoms grouped by combo
  const int* combo_start;  // [n_combo+1]
  int n_combo;
};
cudaError_t opform_init();

// H operand formation of the emulated path on the tensor cores (opgemm.cu).
// Tile: 128 rows of C^H (rb) x 64 plane waves (gb) of one (slot, type) combo.
struct OpTile {
  int combo;
  int rb;
  int gb;
  int pad;
};
struct OpGemmArgs {
  int n;          // rows of C^H = reduction length 2 N_L
  int kchunks;    // padded reduction / 64 (<= 6)
  int64_t G;      // plane waves over all k-points
  const int* combo_slot;
  const int* combo_type;
  const int* combo_atoms;
  const int* combo_start;
  const int* outrow;   // [slot][n]
  const int* npos;     // [slot]
  const int* nneg;     // [slot]
  const int* pos_off;  // [atom]
  const int* neg_off;  // [atom]
  const int* kpk;      // [0] = Kp_pad
  const int* rexp_a;   // [slot * n + r]: scale exponents of the A rows
  const int* rexp_b;   // [type * G + g]: scale exponents of the B rows
  const double2* ph;   // [atom][G] structure-factor phases
  longlong2* P;        // [combo][G][n] fixed-point product (Re, Im)
  double2* Z;          // operand rows (row h_row0 + g, column k')
  int64_t k_alloc;
  int64_t h_row0;
  int alg3_nl;         // 0: factored C^H rows; N_L: the paper's Alg. 3 rows (alg3.cuh)
  int64_t r_row0;      // Alg. 3: operand row of the first R row
  const int* hpd;      // Alg. 1: [slot] 1 where T^AA = C C^H (the Y rows are C^H A and go to
                       // both L and R); null for Alg. 3
};
cudaError_t opgemm_init();
size_t opgemm_smem_bytes();
// build_a: A[slot n + r][perm_s(c)] = conj(C^H_s[r][c]), rows of kp columns;
// otherwise B[t G + g][c] = W_t(c, g).  Columns n..kp-1 are zero.
cudaError_t launch_opgemm_build(const double2* CH, const int* perm, int n_slots, int n, int kp,
                                const double2* Yc, const double* al, const double* bl, int n_L,
                                int lmax, int n_types, int64_t G, double2* A, double2* B,
                                cudaStream_t st, bool build_a);
// The paper's Alg. 3: A[slot n + r][c] = conj(M_s(r, c)) (alg3.cuh) from the T blocks.
// The operand matrix of the paper's Alg. 3 or Alg. 1 per slot (alg3.cuh),
// [slot][n][n] row-major, from T's lower triangle; with alg1 the Y rows are
// C^H where T^AA = C C^H (Cholesky) succeeds (hpd[slot] = 1), else T^AA.
// work: [slot][n][n] scratch.  One CTA per slot.
cudaError_t launch_alg_m(const double2* T, int n, int n_L, int n_slots, bool alg1, double2* M, double2* work,
                         int* hpd, cudaStream_t st);
cudaError_t launch_opgemm_build_alg3(const double2* M, int n_slots, int n, int n_L, int kp,
                                     double2* A, cudaStream_t st);
// P for every tile (opgemm.cu), then every atom's operand rows from P (with
// alg3_nl set: the L and R columns of Alg. 3).
// wait_ns: bound of its abortable device waits (0: the default 4 s).
cudaError_t launch_opgemm(const CUtensorMap& map_a, const CUtensorMap& map_b, const OpGemmArgs& g,
                          const OpTile* tiles, int n_tiles, int* err, int max_ctas,
                          unsigned long long wait_ns, cudaStream_t st);
cudaError_t launch_opgemm_phase(const OpGemmArgs& g, int n_combo, cudaStream_t st);
// The same rows sliced directly (the factored, sigma-grouped layout only):
// writes the contraction's slices SL (rows x k_alloc per plane) and the row
// exponents of the H rows, with no FP64 copy of the operand.
cudaError_t launch_opgemm_slice(const OpGemmArgs& g, int n_combo, int n_slices, __half* SL,
                                int64_t rows, int* rexp, cudaStream_t st);
// The S operand rows (factored operands, emulated precision) formed from the
// type-level W of the operand product and sliced in one pass (opgemm.cu).
struct SopArgs {
  int n, n_L, lmax, n_atoms;
  int64_t G;
  const double2* W;        // [type G + g][kpw]: W_t(c, g)
  int64_t kpw;
  const double* U;         // [type][lmax + 1]
  const double2* ph;       // [atom][G]
  const int* combo_type;   // atoms grouped by (slot, type) combination
  const int* combo_atoms;
  const int* combo_start;
  int n_combo;
  int64_t s_row0;          // operand row of the first S plane wave
  int64_t k_alloc;
};
cudaError_t launch_sop_slice(const SopArgs& a, int n_slices, __half* SL, int64_t rows, int* rexp,
                             cudaStream_t st);
cudaError_t launch_opform_H(const OpformArgs& a, bool factored, cudaStream_t st);
cudaError_t launch_opform_S(const OpformArgs& a, bool factored, cudaStream_t st);
// H operands of the paper's Alg. 3 (h_row0: L rows, r_row0: R rows, 3 N_L
// columns per atom from a * 3 N_L): L_a = [X_a; B_a; A_a], R_a = [B_a; X_a; Y_a]
// with X_a = T^BA A_a + T^BB B_a / 2 and Y_a = T^AA A_a.  Copies A_a and B_a
// into place and, if `product`, forms the X and Y rows in FP64 (otherwise the
// tensor-core product of opgemm.cu writes them).
cudaError_t launch_opform_alg3(const OpformArgs& a, bool factored, bool product, cudaStream_t st);

// Copies a user Z (column-major K x N) into operand rows, sigma-grouped.
cudaError_t launch_gather_Z(const double2* Zin, int64_t ldz, int K, int N, const int* kmap,
                            int64_t k_alloc, double2* Z, cudaStream_t st);

// FP64 -> integer slices (fp16 carriers) with per-row power-of-two scaling.
// Rows [row0, row0 + nrows) of the operand; `rows` is the total row count.
// Valid K columns per row come from its problem (probs[row_prob[row]]), or
// are [0, k_valid) when probs is null.
cudaError_t launch_slicer(const double2* Z, int64_t k_alloc, const Prob* probs,
                          const int* row_prob, int64_t k_valid, int64_t rows, int64_t row0,
                          int64_t nrows, int n_slices, __half* SL, int* rexp, cudaStream_t st);
// The same for short rows (k_alloc <= 512): one warp per row, all columns valid.
cudaError_t launch_slicer_rows(const double2* Z, int64_t k_alloc, int64_t rows, int n_slices,
                               __half* SL, int* rexp, cudaStream_t st);

// S by the addition theorem (slegendre.cu), on the 64 x 64 lower tiles of the
// S problems.
struct SLegArgs {
  const Prob* probs;      // problems (row_base - s_row0 = first global plane wave)
  int64_t s_row0;
  int64_t g_total;
  int lmax, n_types;
  const double* khat;     // [G][3] unit vectors (z for K = 0)
  const double* al;       // [t][l][G] matching coefficients
  const double* bl;
  const double* U;        // [t][l]
  const double2* ph;      // [atom][G] e^{iK.tau_a}
  const int* type_atoms;  // atoms grouped by type
  const int* type_start;  // [n_types + 1]
  double scale;           // 4 pi / Omega
  int n_atoms;
  float2* dfw;            // double-float workspace (slegendre_df_floats2 pairs):
                          // evaluate in double-float; null: in FP64
};
size_t slegendre_df_floats2(int n_types, int lmax, int n_atoms, int64_t G);
// The spherical part of H by the addition theorem (slegendre.cu), on the
// 64 x 64 lower tiles of the H problems, in FP64 or double-float.
struct HLegArgs {
  const Prob* probs;       // problems (row_base - h_row0 = first global plane wave)
  int64_t h_row0;
  int64_t g_total;
  int lmax;
  const double* khat;      // [G][3]
  const double* al;        // [t][l][G]
  const double* bl;
  const double2* ph;       // [atom][G]
  const double* tsph;      // [slot][l][4]: t^AA, t^BB, Re t^BA, Im t^BA
  const int* combo_slot;   // atoms grouped by (slot, type) combination
  const int* combo_type;
  const int* combo_atoms;
  const int* combo_start;  // [n_combo + 1]
  int n_combo;
  double scale;            // 4 pi / Omega
  int n_atoms, n_types;
  float2* dfw;             // double-float workspace (slegendre_df_floats2 pairs):
                           // evaluate in double-float; null: in FP64
};
// add: the spherical part is added to the lower triangle already written.
// inputs_ready: a previous launch of this build_HS already split the inputs
// into double-float (a second part of the tiles).
cudaError_t launch_hlegendre(const HLegArgs& a, const F64Tile* tiles, int n_tiles, bool add, cudaStream_t st,
                             bool inputs_ready = false);
cudaError_t launch_khat(const Geom& geo, const GData& gd, double* khat, cudaStream_t st);
cudaError_t launch_slegendre(const SLegArgs& a, const F64Tile* tiles, int n_tiles, cudaStream_t st);

// Contractions.
cudaError_t launch_herk_f64(const double2* Z, int64_t k_alloc, const Prob* probs,
                            const F64Tile* tiles, int n_tiles, cudaStream_t st);
// Fractional bits of the contraction's 64-bit fixed-point accumulators for
// sums of at most k_terms complex products (each < 2 in magnitude after the
// per-row scaling): 61 - ceil(log2 k_terms), clamped to [40, 50].
int fixed_frac_bits(int64_t k_terms);
// Tensor maps of the slice array [slice][plane][row][k] (fp16) for the
// emulated contraction's operand loads.
struct SliceMaps {
  CUtensorMap a;   // 64 k x 128 rows (the MMA's A rows)
  CUtensorMap b2;  // 64 k x 64 rows x both planes (a B half of a slice pair)
  CUtensorMap b1;  // 64 k x 64 rows (a B half of a lone slice)
};
bool make_slice_tmaps(SliceMaps* maps, void* base, int64_t k_alloc, int64_t rows, int n_slices,
                      std::string* err);
// Tensor map of one slice array [n_slices][2][rows][k_alloc] (fp16), 128-byte
// swizzle, boxes of 64 k x box_rows rows x box_planes planes.
bool make_tmap_4d(CUtensorMap* map, void* base, int64_t k_alloc, int64_t rows, int n_slices,
                  uint32_t box_rows, uint32_t box_planes, std::string* err);
// Kernel attributes and the co-resident CTA-pair count of the current device
// (host side; call outside stream capture before the first launch).
cudaError_t herk_emu_init();
// Launches persistent CTA pairs: min(n_tiles, co-resident pairs - busy_sms),
// where busy_sms is the number of SMs that concurrent work holds.  deep: the
// pipeline of 5 one-chunk stages (large N_G) instead of 3 two-chunk stages.
// cyclic: the tiles are of the cyclic cover (tiles.cuh), else of the aligned one.
// wait_ns: bound of each abortable device wait (0: the default 4 s); a wait
// that runs out sets *err to FLAPW_ERR_TIMEOUT and the pair stops.
cudaError_t launch_herk_emu(const SliceMaps& maps, const Prob* probs, const EmuTile* tiles,
                            int n_tiles, const int* rexp, int n_slices, int frac, int* err,
                            int busy_sms, const SplitScratch& split, bool deep, bool cyclic,
                            unsigned long long wait_ns, cudaStream_t st);
// The pair count a launch beside busy_sms busy SMs gets (0 before herk_emu_init).
int herk_emu_pairs(int busy_sms);
size_t herk_emu_smem_bytes(bool deep);
// The pipeline for problems of at most max_ng plane waves: deep above 8192.
inline bool herk_emu_deep(int64_t max_ng) { return max_ng > 8192; }

// Message of the calling thread's last handle-less error (flapw_last_error(NULL)).
void set_thread_error(const char* msg);

// ---- host G enumeration ----------------------------------------------------
int enumerate_g(const double lat[9], const double k[3], double kmax, std::vector<int>* n3);
void reciprocal(const double lat[9], double rec[9], double* det);

}  // namespace flapw
