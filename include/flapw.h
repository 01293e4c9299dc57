/*
 * flapw.h -- C ABI of the GB300 (sm_103a) muffin-tin Hamiltonian/overlap builder.
 *
 * The library computes, for every k-point of a crystal, the LAPW matching
 * coefficients A and B and the muffin-tin Hamiltonian H and overlap S
 * (Davidovic et al., "Accelerating the computation of FLAPW methods on
 * heterogeneous architectures", Sec. 2 and Sec. 3):
 *
 *   A^{a,G}_{lm}, B^{a,G}_{lm}   matching coefficients          Sec. 2, Eq. (basis)
 *   S = sum_a A_a^H A_a + B_a^H U_a^H U_a B_a                    Eq. (s), Eq. (def_overlap)
 *   H = sum_a [A_a;B_a]^H [[T^AA T^AB];[T^BA T^BB]]_a [A_a;B_a]  Eq. (h), Eq. (def_hamilton)
 *
 * Plain pointers and sizes only.  Complex numbers are interleaved pairs of
 * doubles (re, im), the layout of C99 double _Complex and cuDoubleComplex.
 *
 * Conventions used by every call:
 *   lattice     double[9], rows are the lattice vectors a1, a2, a3 (bohr).
 *   k_frac      k-points in fractional coordinates of the reciprocal basis.
 *   N_L         (lmax+1)^2; the index L = l*l + l + m, -l <= m <= l.
 *   Y_lm        complex, orthonormal, Condon-Shortley phase.
 *   A_{lm}(G)   = 4 pi / sqrt(Omega) e^{i (k+G).tau_a} i^l conj(Y_lm(K_hat)) a_l(|K|),
 *   B_{lm}(G)   = same with b_l, where (a_l, b_l) solve
 *                 a u(R) + b udot(R) = j_l(|K| R),  a u'(R) + b udot'(R) = |K| j_l'(|K| R)
 *                 (continuity of value and slope at the sphere, Sec. 2).  K = k+G.
 *   G order     ascending |k+G|^2 quantised to 2^-40 K_max^2, ties by (n1,n2,n3).
 *   H, S        row G', column G; only the lower triangle G' >= G is written.
 *
 * Errors: every call returns FLAPW_OK (0) or a negative FLAPW_ERR_* code and
 * records a message readable with flapw_last_error(handle) (or with a NULL
 * handle for calls that have none: the calling thread's last such message).
 * Work is enqueued asynchronously on the given CUDA stream; errors detected
 * on the device (a bounded wait that ran out, a singular 2x2 pivot of a T
 * block) are reported by flapw_sync().  A handle is not thread-safe.
 */
#ifndef FLAPW_H
#define FLAPW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flapw_ctx* flapw_handle;

#define FLAPW_OK 0
#define FLAPW_ERR_ARG (-1)         /* invalid argument: the message names it */
#define FLAPW_ERR_CUDA (-2)        /* a CUDA runtime or driver call failed */
#define FLAPW_ERR_OOM (-3)         /* device memory could not be allocated */
#define FLAPW_ERR_FACTOR (-4)      /* a factorisation failed: a T block with a zero 2x2 pivot, or
                                      (flapw_eigh) an S that is not positive definite */
#define FLAPW_ERR_TIMEOUT (-5)     /* a bounded device-side wait ran out; results are invalid */
#define FLAPW_ERR_STATE (-6)       /* call out of order (e.g. a handle made for flapw_herk only) */
#define FLAPW_ERR_UNSUPPORTED (-7) /* size outside what the kernels support */

#define FLAPW_PREC_FP64 0 /* plain FP64 contraction (DMMA tensor cores) */
#define FLAPW_PREC_EMU 1  /* split-precision emulation of complex FP64 on FP16 tensor cores */

#define FLAPW_LAYOUT_LOWER_FULL 0   /* element (i, j), i >= j, at j*ld + i (column-major) */
#define FLAPW_LAYOUT_LOWER_PACKED 1 /* LAPACK 'L' packed: j*N - j*(j-1)/2 + (i - j) */

#define FLAPW_OPERANDS_FROM_AB 0  /* build_HS forms its operands from the A, B it is given */
#define FLAPW_OPERANDS_FACTORED 1 /* build_HS regenerates the per-type part of A, B itself */

/* How build_HS forms S.  FLAPW_S_LEGENDRE sums over m by the addition
 * theorem, sum_m Y_lm(u) conj(Y_lm(v)) = (2l+1)/(4 pi) P_l(u.v), so that
 *   S_{G'G} = (4 pi / Omega) sum_t rho_t(G', G) sum_l (2l+1) P_l(Khat'.Khat)
 *             [a_l(K') a_l(K) + U_l^2 b_l(K') b_l(K)],
 *   rho_t = sum over the atoms a of type t of conj(e^{iK'.tau_a}) e^{iK.tau_a}
 * (Eq. (def_overlap) with the matching of Sec. 2): no factor N_L, no slices. */
#define FLAPW_S_CONTRACTION 0
#define FLAPW_S_LEGENDRE 1

/* How build_HS forms H.  FLAPW_H_FACTORED factorises each T block (see
 * flapw_build_HS) and contracts one Hermitian rank-K update, K = 2 N_A N_L.
 * FLAPW_H_ALG3 follows the operation sequence of the paper's refined
 * algorithm (Sec. 5.1, Alg. 3) without any factorisation: with
 *   X_a = T^BA A_a + (1/2) T^BB B_a   and   Y_a = T^AA A_a,
 *   H = X^H B + B^H X + A^H Y          (zher2k + zherkx of Alg. 3),
 * evaluated as one lower-triangle contraction L^H R over K = 3 N_A N_L rows,
 * L_a = [X_a; B_a; A_a], R_a = [B_a; X_a; Y_a].  It reads the blocks
 * T^AA, T^BA, T^BB (T Hermitian, lower triangle given) and executes 1.5 x the
 * contraction flops of FLAPW_H_FACTORED. */
#define FLAPW_H_FACTORED 0
#define FLAPW_H_ALG3 1
/* FLAPW_H_SPHERICAL: H of the spherical part of T (per slot the l-diagonal
 * blocks t^XY_l delta_{L'L} given to flapw_set_spherical_T) by the addition
 * theorem, like FLAPW_S_LEGENDRE for S:
 *   H_sph = (4 pi / Omega) sum_c rho_c sum_l (2l+1) P_l(Khat'.Khat)
 *           [t^AA a'a + t^BB b'b + t^AB a'b + t^BA b'a]_l
 * (c the (slot, type) combinations of atoms, rho_c their phase sums), plus
 * the FLAPW_H_FACTORED contraction of the rest T - T_sph.  The factorisation
 * drops exact zero pivots, so a rest confined to r rows and columns of each
 * slot contracts over K = r per atom; a rest that is exactly zero (T is its
 * spherical part) runs no factorisation, operands or contraction for H.
 * Needs FLAPW_OPERANDS_FACTORED; the addition-theorem part runs in FP64 on
 * the FP64 path and in double-float FP32 pairs on the emulated path. */
#define FLAPW_H_SPHERICAL 2
/* FLAPW_H_ALG1: the paper's Alg. 1 (Sec. 3) on the engine of FLAPW_H_ALG3.  Per
 * slot it tries the Cholesky factorisation T^AA = C C^H (FP64 on the device);
 * where it succeeds the H_AA part is the Hermitian update (C^H A)^H (C^H A)
 * (the paper's ztrmm + zherk), where it fails A^H (T^AA A) (zhemm + zgemm).
 * In the stacked contraction L^H R of FLAPW_H_ALG3 (K = 3 N_A N_L) this only
 * changes the third block of L_a and R_a: both C^H A_a, or A_a and T^AA A_a.
 * stats.n_chol counts the slots that factorised.  The result is the same H;
 * the executed contraction work is that of FLAPW_H_ALG3. */
#define FLAPW_H_ALG1 3

typedef struct flapw_options {
  int precision; /* FLAPW_PREC_EMU (default) or FLAPW_PREC_FP64 */
  int n_slices;  /* emulation: 7-bit slices per operand entry, 4..8 (0 = default 7) */
  int layout;    /* FLAPW_LAYOUT_LOWER_FULL (default) or FLAPW_LAYOUT_LOWER_PACKED */
  int operands;  /* FLAPW_OPERANDS_FROM_AB (default) or FLAPW_OPERANDS_FACTORED */
  int use_graph; /* 1: capture build_HS into a CUDA graph and replay it while the
                    arguments repeat (default 0) */
  int autotune;  /* 1: once per problem shape, time the emulated contraction's tile
                    cover, tile order and load pipeline (coordinate descent over the
                    three, on the slices of the first call) and keep the fastest; the
                    choice is kept for the process and, if the environment variable
                    FLAPW_AUTOTUNE_CACHE names a file, read from and appended to it
                    (one line per shape).  Default 0: the fixed choices by size. */
  int tile_order; /* 0: library default (cyclic cover: strip by strip;
                     aligned cover: bands of 32 row blocks of 64 for N_G <= 16384,
                     else bands of 8); k+1 forces tile order k of the emulated
                     contraction (0 strip by strip, 1..5 bands of 4/8/16/32/64
                     row blocks of 64, strip by strip within a band), ignored
                     when autotune is on */
  int s_method;   /* FLAPW_S_CONTRACTION (default): S = Z_S^H Z_S like H;
                     FLAPW_S_LEGENDRE: S by the addition theorem (requires
                     FLAPW_OPERANDS_FACTORED; in FP64 on the FP64 path, in
                     double-float FP32 pairs on the emulated path) */
  int h_method;   /* FLAPW_H_FACTORED (default), FLAPW_H_ALG3, FLAPW_H_SPHERICAL or
                     FLAPW_H_ALG1 */
  int pipeline;   /* emulated contraction's load pipeline: 0 by size (5 stages of one
                     64-wide K chunk above N_G 8192, else 3 stages of two), 1 the
                     3-stage shape, 2 the 5-stage shape; results are identical */
  int tile_cover; /* how the emulated contraction's CTA-pair tiles (a 64-column
                     strip against four 64-row blocks) cover the lower triangle:
                     0 by size (cyclic up to N_G 8192, aligned above), 1 cyclic
                     (each strip takes a cyclic window of row blocks; blocks above
                     its diagonal are written conjugate-transposed, so every
                     64 x 64 block is computed once), 2 aligned (256-row blocks
                     aligned to 256; the upper parts of diagonal tiles are computed
                     and not written); results agree to rounding */
  int wait_us;    /* bound of each device-side wait of the tensor-core kernels, in
                     microseconds (0: the default, 4 s).  A wait that runs out stops
                     the kernel cleanly (no fault) and the next flapw_sync() returns
                     FLAPW_ERR_TIMEOUT; the results of that call are invalid and the
                     handle stays usable.  Small values exist to test that path. */
  int mem_cap_mb; /* cap on the device workspace this handle allocates, in MiB (0: no
                     cap).  A call whose workspaces would pass it returns
                     FLAPW_ERR_OOM before enqueueing anything; what the handle holds
                     stays owned by it (freed by flapw_destroy) and a later call
                     under a larger cap proceeds. */
  int part_count; /* split of the job over independent callers, one per GPU and
                     none communicating (0 or 1: no split).  See flapw_partition:
                     whole k-points go to the parts when that balances, otherwise
                     every part takes every part_count-th output tile of each
                     k-point.  A part computes A, B and the operands of every
                     k-point (they are cheap) and only its share of the
                     contraction; H[k], S[k] of k-points of other parts may be
                     NULL and are not touched.  With tiles split, a part writes its
                     blocks of each lower triangle: device-memory outputs keep
                     whatever they held elsewhere, host-memory outputs receive
                     zeros there, so the parts' zero-initialised buffers sum to H
                     and S. */
  int part_index; /* this caller's part, 0 .. part_count-1 */
  int reserved[1];
} flapw_options;

typedef struct flapw_stats {
  double ms_ab;        /* last build_AB, device time (ms), if timing was on */
  double ms_factor;    /* last build_HS: T factorisation */
  double ms_operands;  /* operand formation */
  double ms_slice;     /* slicing (emulated precision only) */
  double ms_contract;  /* contraction */
  double ms_hs_total;  /* whole build_HS */
  double flops_herk;   /* 16 N_A N_L sum_k N_G(k)^2: H and S in the Hermitian rank-K count */
  double flops_tensor; /* tensor-core flops executed by the contraction */
  int64_t k_total;     /* inner dimension of the H contraction: K = 2 N_A N_L
                          (3 N_A N_L with FLAPW_H_ALG3 and FLAPW_H_ALG1) */
  int n_pos;           /* rows of the H operand with sigma = +1 (all atoms) */
  int n_neg;           /* rows with sigma = -1 */
  int n_pivot2;        /* 2x2 pivots taken by the factorisation (all slots) */
  int n_slices;        /* slices used (emulated precision) */
  int n_tiles;         /* output tiles of the last contraction launch */
  int tile_order;      /* tile-order variant in use */
  int graph_replays;   /* build_HS calls served by CUDA-graph replay */
  int tile_cover;      /* tile cover in use for the largest problem (1 cyclic, 2 aligned) */
  int pipeline;        /* load pipeline in use (1: 3 stages of two chunks, 2: 5 of one) */
  int copy_ops;        /* device-to-host copies the last build_HS or herk enqueued */
  int64_t bytes_d2h;   /* bytes those copies move (host-memory outputs only) */
  int n_chol;          /* FLAPW_H_ALG1: slots whose T^AA Cholesky factorisation succeeded */
  int reserved[3];
  double ms_s;         /* the S half of ms_contract: its contraction, or with
                          FLAPW_S_LEGENDRE the addition-theorem evaluation */
  double ms_ab_assemble; /* the A/B assembly kernel of the last build_AB (part of ms_ab) */
} flapw_stats;

/* Defaults listed in flapw_options. */
void flapw_default_options(flapw_options* opt);

/* Plane-wave set of Sec. 2: all integer n with |(n + k_frac) . B| <= kmax,
 * B the reciprocal basis (b_i = 2 pi (a_j x a_k) / (a_1 . (a_2 x a_3))), in the
 * order stated above.  Host-only; needs no GPU.  Writes *n_g (always) and up
 * to max_g triples into n3[i*3 + 0..2] (n3 may be NULL to query the count).
 * Errors: FLAPW_ERR_ARG for a singular lattice, kmax <= 0 or NULL n_g. */
int flapw_enumerate_g(const double lattice[9], const double k_frac[3], double kmax, int max_g,
                      int* n3, int* n_g);

/* Creates a handle for one crystal (Sec. 2; the paper's matrix sizes are those of Sec. 3).
 *   n_atoms, pos_frac[n_atoms*3]  fractional atom positions (copied)
 *   atom_type[n_atoms]            type index in [0, n_types) (copied)
 *   mt_radius[n_types]            muffin-tin radius per type, > 0
 *   lmax                          0..12
 *   n_k, k_frac[n_k*3], kmax[n_k] k-points and their cut-offs (copied)
 *   opt                           NULL for defaults
 * Enumerates every k-point's plane waves on the host and uploads the
 * geometry to the current CUDA device.  Device workspaces are allocated on
 * first use and released by flapw_destroy.  *out receives the handle. */
int flapw_hs_create(const double lattice[9], int n_atoms, const double* pos_frac,
                    const int* atom_type, int n_types, const double* mt_radius, int lmax,
                    int n_k, const double* k_frac, const double* kmax,
                    const flapw_options* opt, flapw_handle* out);

/* The spherical part of T for options.h_method = FLAPW_H_SPHERICAL.
 *   t_sph[n_slots*(lmax+1)*4] (host, copied): per slot and l the real
 *       t^AA_l, the real t^BB_l and Re, Im of t^BA_l (t^AB_l = conj t^BA_l),
 *       such that the slot's T holds T^XY_{(lm),(lm)} = t^XY_l + (the rest).
 *   NULL or n_slots < 1 clears it.  build_HS returns FLAPW_ERR_STATE with
 *   FLAPW_H_SPHERICAL unless n_slots matches its own and lmax the handle's.
 * H is the same for any t_sph (linearity in T); the split only changes how
 * much is contracted.  Errors: FLAPW_ERR_ARG for non-finite entries. */
int flapw_set_spherical_T(flapw_handle h, const double* t_sph, int n_slots);

/* How a job of n_k k-points with n_g[k] plane waves is split over part_count
 * independent callers (options.part_count; the k-points and the output tiles
 * are independent, the paper's multi-device split of Sec. 5 with no exchange
 * step).  Whole k-points go to the parts, largest N_G^2 first to the least
 * loaded part (ties to the lower index), when there are at least part_count
 * of them and no part then exceeds 1.1 x the mean load: owner[k] receives
 * the part of k-point k.  Otherwise owner[k] = -1 for every k: each part
 * computes every part_count-th contraction tile of every k-point.  Host
 * only; every caller computes the same answer.  Errors: FLAPW_ERR_ARG. */
int flapw_partition(int n_k, const int* n_g, int part_count, int* owner);

/* A handle without a crystal, usable only with flapw_herk. */
int flapw_engine_create(const flapw_options* opt, flapw_handle* out);

/* Replaces the handle's options (takes effect at the next build call). */
int flapw_set_options(flapw_handle h, const flapw_options* opt);

/* Number of plane waves N_G(k) of k-point k. */
int flapw_num_g(flapw_handle h, int k, int* n_g);

/* The plane waves of k-point k as integer triples n3[i*3 + 0..2], i < N_G(k). */
int flapw_get_gvectors(flapw_handle h, int k, int* n3);

/* Offset, in complex elements, of k-point k's block inside the A and B
 * buffers of flapw_build_AB; offset(n_k) is the total element count. */
int flapw_ab_offset(flapw_handle h, int k, int64_t* offset);

/* Matching coefficients A and B of Sec. 2, Eq. (basis), for every k-point and atom.
 *   radial[n_types*(lmax+1)*4] (host): u_l(R), u_l'(R), udot_l(R), udot_l'(R)
 *                                      per (type, l); copied.
 *   A, B: complex128 buffers of flapw_ab_offset(h, n_k) elements, device or
 *         host memory (host memory is staged through the device).  Element
 *         (k, a, L, G) sits at offset(k) + (a*N_L + L)*N_G(k) + G.
 * The radial data is retained by the handle for FLAPW_OPERANDS_FACTORED. */
int flapw_build_AB(flapw_handle h, const double* radial, void* A, void* B, void* stream);

/* Hamiltonian and overlap of Eqs. (h) and (s) for every k-point.
 *   T[n_slots*(2N_L)^2] (host, complex row-major): per slot the Hermitian
 *       matrix [[T^AA, T^AB],[T^BA, T^BB]], rows/cols [A-part L; B-part L];
 *       only its lower triangle is read.
 *   atom_slot[n_atoms] (host): which T block each atom uses.
 *   U[n_types*(lmax+1)] (host): ||udot_l|| per (type, l); S carries U^2.
 *   A, B: the buffers written by flapw_build_AB (device or host memory);
 *       ignored (may be NULL) with FLAPW_OPERANDS_FACTORED, which requires a
 *       previous flapw_build_AB on this handle for the radial data.
 *   H[n_k], S[n_k]: per k-point output pointers (device or host memory),
 *       complex128, lower triangle in the handle's layout; the full layout
 *       uses ld = N_G(k).  Elements above the diagonal are not written in
 *       device memory.  Host memory is written in blocks of columns, each
 *       from its first diagonal element down, so the elements above the
 *       diagonal inside each block (about 1/nb of the upper triangle for nb
 *       blocks per matrix) receive unspecified values and the others are
 *       left untouched; nb is 32 for one host output per call and shrinks to
 *       keep one call's copies to about 320 (stats.copy_ops, stats.bytes_d2h).
 * Each T block is factorised as T = C diag(sigma) C^H (Bunch-Kaufman
 * pivoted LDL^H, then 2x2 eigen-splitting; Sec. 3, Alg. 1's Cholesky step
 * generalised to indefinite T), so that H = Z^H diag(sigma) Z with
 * Z_a = C^H [A_a; B_a] and S = Z_S^H Z_S with Z_S,a = [A_a; U B_a]: one
 * lower-triangle rank-K contraction each, K = 2 N_A N_L (Fig. agg stacking).
 * The other H methods (FLAPW_H_ALG3, FLAPW_H_ALG1, FLAPW_H_SPHERICAL) form H
 * as described at their definitions.
 * The call returns once its work is enqueued: T, U and the slots are staged
 * in one of two pinned buffers, each reused only after the copies of the call
 * that last used it have run, so a third call may wait for the first; the
 * host-memory outputs are complete after flapw_sync() or the stream.
 * A zero 1x1 pivot (a column that is zero on and below the diagonal after
 * the previous steps) contributes nothing and its row is dropped from Z.
 * Errors: FLAPW_ERR_OOM if the workspaces do not fit (returned here); a
 * 2x2 pivot with a zero determinant is found on the device and reported by
 * the next flapw_sync() as FLAPW_ERR_FACTOR. */
int flapw_build_HS(flapw_handle h, const double* T, int n_slots, const int* atom_slot,
                   const double* U, const void* A, const void* B, void* const* H,
                   void* const* S, void* stream);

/* The contraction step alone: lower triangle of Z^H diag(sigma) Z.
 *   Z: device, complex128, column-major K x N (element (k, g) at g*ldz + k).
 *   sigma[K] (host): +1 or -1 per row, or NULL for all +1.
 *   H: device or host, complex128, layout/ld as in flapw_build_HS (ldh >= N).
 * Precision and slice count come from the handle's options. */
int flapw_herk(flapw_handle h, const void* Z, int64_t ldz, int K, int N, const int* sigma,
               void* H, int64_t ldh, void* stream);

/* The generalised eigenproblem of Sec. 2 for one k-point, H c = lambda S c,
 * on matrices this library built (Hermitian H, Hermitian positive definite S).
 *   H, S: device, complex128, column-major, lower triangle read (the
 *       flapw_build_HS full layout: ldh = lds = N_G(k)); overwritten: H by the
 *       eigenvectors as columns, S-orthonormal (C^H S C = I), when vectors != 0
 *       (otherwise destroyed), S by its Cholesky factor L (S = L L^H, lower).
 *   w[n] (host or device): the eigenvalues, ascending.
 * The solve is cuSOLVER's zhegvd (Cholesky of S, reduction to standard form,
 * Hermitian eigensolver, back-transformation; FP64), loaded when this is
 * first called; its workspace belongs to the handle.  It runs on `stream`
 * and returns when it has finished there.  The muffin-tin S alone is
 * positive definite only where 2 N_A N_L >= N_G (a physical problem adds the
 * interstitial part, which is not built here).
 * Errors: FLAPW_ERR_FACTOR if S is not positive definite (the message names
 * the failing leading minor) or the eigensolver does not converge;
 * FLAPW_ERR_UNSUPPORTED if cuSOLVER cannot be loaded; FLAPW_ERR_ARG for n < 1,
 * ldh or lds < n, or H, S outside device memory; FLAPW_ERR_OOM if the
 * workspace does not fit. */
int flapw_eigh(flapw_handle h, int n, void* H, int64_t ldh, void* S, int64_t lds, double* w,
               int vectors, void* stream);

/* The contraction step alone (as flapw_herk, emulated precision) for callers
 * that must not allocate device memory: code that runs under a fixed device
 * memory budget or inside a framework whose caching allocator owns the GPU,
 * where a cudaMalloc from a library can fail, fragment the pool or stall the
 * device.  This entry point allocates nothing: its workspaces live in one
 * static device array of 64 MiB that every GPU loading the library holds
 * until the process exits.  The paper has no counterpart to this call.
 *   Z: device, complex128, column-major K x N (element (k, g) at g*ldz + k).
 *   sigma[K] (host): +1/-1 per row, or NULL for all +1.
 *   H: device, complex128, lower triangle in `layout` (ld = ldh for the full
 *      layout, ldh >= N).  n_slices 4..8 (0 = 7).  stream: the caller's stream.
 * Size limit: K below 131072, and about 44 bytes per N x K entry (7 slices)
 * plus small tables must fit in the 64 MiB array, e.g. N = 1024 with
 * K = 1400; larger problems return FLAPW_ERR_UNSUPPORTED before any work is
 * enqueued.  sigma and the problem's sizes reach the device in kernel
 * arguments: nothing of the caller's host memory is read after the call
 * returns.
 * The first call on each device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Calls share the array and it keeps the last
 * call's contents; calls whose work overlaps on the GPU race.  Errors are
 * reported by the return code (FLAPW_ERR_ARG, FLAPW_ERR_UNSUPPORTED,
 * FLAPW_ERR_CUDA) with a message for flapw_last_error(NULL).  A bounded
 * device wait that runs out (the GPU stalled for seconds) is not reported:
 * H is then invalid, and a caller that must know checks H itself (its
 * diagonal is real, and non-negative when every sigma is +1). */
int flapw_herk_noalloc(const void* Z, int64_t ldz, int K, int N, const int* sigma, void* H,
                       int64_t ldh, int layout, int n_slices, void* stream);

/* Waits for the handle's enqueued work; reports device-side errors. */
int flapw_sync(flapw_handle h);

/* Statistics of the last calls (stage times need flapw_sync first). */
int flapw_get_stats(flapw_handle h, flapw_stats* st);

/* Debug export of the last T factorisation of slot `slot`: CH[(2N_L)^2]
 * complex row-major receives C^H with its rows ordered sigma = +1 first,
 * then -1; *n_pos and *n_neg give the counts (rows past them are zero).
 * Synchronises the stream.  FLAPW_ERR_STATE if the last build_HS ran with
 * FLAPW_H_ALG3 (no factorisation). */
int flapw_get_factor(flapw_handle h, int slot, double* CH, int* n_pos, int* n_neg);

/* Message for the last error on h (or of the calling thread's last handle-less call
 * if h is NULL). */
const char* flapw_last_error(flapw_handle h);

/* Releases the handle and every device workspace it owns. */
int flapw_destroy(flapw_handle h);

#ifdef __cplusplus
}
#endif
#endif
