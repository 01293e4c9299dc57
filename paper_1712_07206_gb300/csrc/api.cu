// C ABI of the muffin-tin H/S builder: handle, workspaces and the enqueue
// sequence of each call.  See include/flapw.h for the contract of every entry
// point; the kernels live in the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <cusolverDn.h>
#include <dlfcn.h>

#include "flapw_internal.h"
#include "tiles.cuh"

using namespace flapw;

namespace {

thread_local std::string g_last_error;  // errors of calls without a handle, per thread
constexpr int kNumTileOrders = cover::kNumOrders;  // emulated tile orders (tiles.cuh)

// Device bytes a handle's workspaces hold, against its cap
// (options.mem_cap_mb, 0 for none).  A handle's calls make theirs the calling
// thread's current budget (BudgetScope); workspaces allocated then count
// against it until they are freed.
struct Budget {
  size_t cap = 0, used = 0;
};
thread_local Budget* g_budget = nullptr;

// Device buffer that grows on demand.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Budget* budget = nullptr;  // the budget it counts against
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      (void)cudaGetLastError();
      if (budget) budget->used -= bytes;
    }
    p = nullptr;
    bytes = 0;
    budget = nullptr;
  }
  cudaError_t ensure(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    release();
    if (n == 0) n = 16;
    Budget* b = g_budget;
    if (b && b->cap && b->used + n > b->cap) return cudaErrorMemoryAllocation;  // over the cap
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      return e;
    }
    bytes = n;
    budget = b;
    if (b) b->used += n;
    return cudaSuccess;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Pinned host staging that grows on demand.
struct PinBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~PinBuf() {
    if (p) cudaFreeHost(p);
    (void)cudaGetLastError();
  }
  cudaError_t ensure(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, n ? n : 16);
    if (e == cudaSuccess) bytes = n ? n : 16;
    return e;
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Which problems and tiles one part computes: problems with on[p] set, and of
// each problem's ordered tile list every stride-th tile from index.
struct PartFilter {
  const std::vector<char>* on = nullptr;
  int stride = 1, index = 0;
};

}  // namespace

namespace flapw {
void set_thread_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace flapw

struct flapw_ctx {
  std::string err;
  flapw_options opt{};
  Budget budget;  // declared before the workspaces, which count against it
  bool engine_only = false;
  int device = 0;
  int num_sms = 0;

  // crystal
  double lat[9]{}, rec[9]{}, volume = 0;
  int n_atoms = 0, n_types = 0, lmax = 0, n_L = 0, n_k = 0;
  std::vector<double> pos, radius, kfrac, kmax, ktau;
  std::vector<int> type;
  std::vector<std::vector<int>> n3;
  std::vector<int64_t> goff;
  int64_t g_total = 0;
  std::vector<int> gt128, gt64;

  DevBuf d_rec, d_pos, d_type, d_radius, d_kfrac, d_ktau, d_n3, d_gk, d_goff, d_coef, d_gt128,
      d_gt64;

  // radial data from build_AB
  std::vector<double> radial;
  bool have_radial = false;
  DevBuf d_radial;
  DevBuf d_Yc, d_al, d_bl, d_ph;
  bool prep_valid = false;

  // build_HS workspaces
  // H operands on the tensor cores (emulated path, factored operands): the two
  // factors in FP64 and sliced, their scale exponents, tiles and tensor maps
  DevBuf d_opA, d_opB, d_opSLA, d_opSLB, d_oprexp, d_optiles, d_opP;
  DevBuf d_khat, d_typeatoms;    // S by the addition theorem: Khat per G, atoms by type
  DevBuf d_sdf;                  // its double-float inputs (emulated precision)
  DevBuf d_hdf;                  // those of H's spherical part by the addition theorem
  bool khat_valid = false;       // both depend on the crystal only
  std::vector<OpTile> optiles;
  CUtensorMap opmap_a{}, opmap_b{};
  void* opmap_a_base = nullptr;
  void* opmap_b_base = nullptr;
  int64_t opmap_a_rows = 0, opmap_b_rows = 0;
  int opmap_kp = 0;
  DevBuf d_T, d_work, d_CH, d_fac, d_cnt, d_slot, d_U, d_off, d_probs, d_rowprob, d_Z, d_SL, d_rexp,
      d_emu_tiles, d_f64_tiles, d_combo, d_kmap, d_stageA, d_stageB, d_stageOut;
  // pinned inputs of build_HS: two slots, each guarded by an event recorded
  // after the copies that read it (graph replays use slot 0 only)
  PinBuf pin_ring[2], pin_probs_ring[2];
  cudaEvent_t pin_ev[2]{};
  bool pin_ev_used[2]{};
  int pin_slot = 0;
  int64_t k_alloc = 0, rows = 0;
  int64_t k_terms = 0;           // most products summed into one output element
  int n_emu_tiles = 0, n_f64_tiles = 0, split_emu = 0, split_f64 = 0, tiles_order = -1;
  int tile_order = 4;            // emulated tile order in use (tiles.cuh)
  int64_t max_ng = 0;            // largest N_G of the handle's problems (default tile order)
  std::vector<int> emu_tiles_per_prob;  // whole emulated tiles of each problem
  int tile_cover = 0;            // emulated tile cover in use (tiles.cuh; 0 by N_G)
  int tiles_cover = -1;          // cover of the uploaded lists
  // this caller's part of a partitioned job (options.part_count/part_index)
  std::vector<char> part_on;     // problems this part computes
  PartFilter part_filter;        // and its tile stride
  std::string part_key, tiles_part;  // the partition the uploaded lists were made for
  bool deep_pipe = false;        // the contraction's deep pipeline (herk_emu_deep of the largest N_G)
  std::string tuned_shape;       // shape the autotuner's choice in use belongs to
  int pipe_choice = 0;           // autotuner's load pipeline (1 shallow, 2 deep; 0 none)
  std::string device_name;       // for the autotuner's shape key
  int64_t tiles_rows_key = -1;
  int tiles_pairs = -1;          // pair counts the tile lists' last waves were split for
  int split_ids = 0;             // split tiles of a half (scratch slots)
  bool tiles_split = false;      // the first half's list is in two parts (H to host memory)
  int split_emu_b = 0, split_f64_b = 0;  // start of the first half's second part
  DevBuf d_split;                // their partial sums and completion counts
  SliceMaps tmap{};
  void* tmap_base = nullptr;
  int64_t tmap_k = 0, tmap_rows = 0;
  int tmap_s = 0;

  cudaStream_t cap_stream = nullptr, aux_stream = nullptr;
  // host-memory S outputs go back on their own stream while H is computed
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copy = nullptr;
  // events: 0 start, 1 factor done (aux), 2 S operands done, 3 S sliced, 4 S contracted,
  // 5 end, 6/7 build_AB, 8 H operands start, 9 S operands start, 10 H operands done,
  // 11 H sliced, 12 H contracted, 13 fork, 14/15 autotune, 16 auxiliary work done (join),
  // 17 A/B assembly start, 18 first part of a split H contraction done
  cudaEvent_t ev[19]{};
  bool ev_recorded = false, ev_ab = false, ev_engine = false;
  cudaStream_t last_stream = nullptr;
  flapw_stats stats{};
  int last_n_slots = 0;
  bool last_alg3 = false;        // the last build_HS formed H by the paper's Alg. 3
  // spherical part of T (flapw_set_spherical_T): [slot][l][4] = t^AA, t^BB, Re t^BA, Im t^BA
  std::vector<double> tsph;
  int tsph_slots = 0, tsph_lmax = -1;
  DevBuf d_tsph;
  DevBuf d_hpd;                  // Alg. 1: [slot] the Cholesky factorisation of T^AA succeeded
  bool last_alg1 = false;        // the last build_HS formed H by the paper's Alg. 1
  bool last_h_zero = false;      // the last build_HS's T was its spherical part (no H contraction)

  // CUDA graph replay of build_HS
  cudaGraphExec_t gexec = nullptr;
  std::vector<uintptr_t> gkey;

  // generalised eigensolve (flapw_eigh): the solver's handle and workspaces
  void* solver = nullptr;
  DevBuf d_eig_work, d_eig_w;

  ~flapw_ctx();
};

namespace {

// cuSOLVER, opened on the first flapw_eigh: the library loads and runs the
// H/S build without it.
struct Solver {
  bool ok = false;
  std::string why;
  decltype(&cusolverDnCreate) create = nullptr;
  decltype(&cusolverDnDestroy) destroy = nullptr;
  decltype(&cusolverDnSetStream) set_stream = nullptr;
  decltype(&cusolverDnZhegvd_bufferSize) zhegvd_buffer = nullptr;
  decltype(&cusolverDnZhegvd) zhegvd = nullptr;
};

Solver& solver_lib() {
  static Solver s;
  static std::once_flag once;
  std::call_once(once, [] {
    void* lib = nullptr;
    for (const char* name : {"libcusolver.so.12", "libcusolver.so", "/usr/local/cuda/lib64/libcusolver.so.12"})
      if ((lib = dlopen(name, RTLD_NOW | RTLD_LOCAL))) break;
    if (!lib) {
      const char* e = dlerror();
      s.why = std::string("cuSOLVER could not be loaded: ") + (e ? e : "not found");
      return;
    }
    s.create = reinterpret_cast<decltype(s.create)>(dlsym(lib, "cusolverDnCreate"));
    s.destroy = reinterpret_cast<decltype(s.destroy)>(dlsym(lib, "cusolverDnDestroy"));
    s.set_stream = reinterpret_cast<decltype(s.set_stream)>(dlsym(lib, "cusolverDnSetStream"));
    s.zhegvd_buffer = reinterpret_cast<decltype(s.zhegvd_buffer)>(dlsym(lib, "cusolverDnZhegvd_bufferSize"));
    s.zhegvd = reinterpret_cast<decltype(s.zhegvd)>(dlsym(lib, "cusolverDnZhegvd"));
    s.ok = s.create && s.destroy && s.set_stream && s.zhegvd_buffer && s.zhegvd;
    if (!s.ok) s.why = "cuSOLVER lacks the zhegvd entry points";
  });
  return s;
}

}  // namespace

flapw_ctx::~flapw_ctx() {
  if (solver) solver_lib().destroy(static_cast<cusolverDnHandle_t>(solver));
  {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (aux_stream) cudaStreamDestroy(aux_stream);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (ev_copy) cudaEventDestroy(ev_copy);
    for (auto& e : pin_ev)
      if (e) cudaEventDestroy(e);
    (void)cudaGetLastError();
  }
}

namespace {

// Makes the handle's budget current for the calling thread during one call.
struct BudgetScope {
  Budget* prev;
  explicit BudgetScope(flapw_ctx* h) : prev(g_budget) {
    h->budget.cap = (size_t)h->opt.mem_cap_mb << 20;
    g_budget = &h->budget;
  }
  ~BudgetScope() { g_budget = prev; }
};

int fail(flapw_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_last_error = msg;
  return code;
}

int cuda_fail(flapw_ctx* h, cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? FLAPW_ERR_OOM : FLAPW_ERR_CUDA;
  return fail(h, code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, expr, what)                              \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return cuda_fail(h, _e, what); \
  } while (0)

int check_options(flapw_ctx* h, const flapw_options& o) {
  if (o.precision != FLAPW_PREC_FP64 && o.precision != FLAPW_PREC_EMU)
    return fail(h, FLAPW_ERR_ARG, "options.precision must be FLAPW_PREC_FP64 or FLAPW_PREC_EMU");
  if (o.n_slices != 0 && (o.n_slices < 4 || o.n_slices > 8))
    return fail(h, FLAPW_ERR_ARG, "options.n_slices must be 0 or in 4..8");
  if (o.layout != FLAPW_LAYOUT_LOWER_FULL && o.layout != FLAPW_LAYOUT_LOWER_PACKED)
    return fail(h, FLAPW_ERR_ARG, "options.layout is not a FLAPW_LAYOUT_* value");
  if (o.operands != FLAPW_OPERANDS_FROM_AB && o.operands != FLAPW_OPERANDS_FACTORED)
    return fail(h, FLAPW_ERR_ARG, "options.operands is not a FLAPW_OPERANDS_* value");
  if (o.tile_order < 0 || o.tile_order > kNumTileOrders)
    return fail(h, FLAPW_ERR_ARG, "options.tile_order must be in 0..6");
  if (o.s_method != FLAPW_S_CONTRACTION && o.s_method != FLAPW_S_LEGENDRE)
    return fail(h, FLAPW_ERR_ARG, "options.s_method is not a FLAPW_S_* value");
  if (o.s_method == FLAPW_S_LEGENDRE && o.operands != FLAPW_OPERANDS_FACTORED)
    return fail(h, FLAPW_ERR_ARG, "options.s_method FLAPW_S_LEGENDRE needs FLAPW_OPERANDS_FACTORED");
  if (o.h_method != FLAPW_H_FACTORED && o.h_method != FLAPW_H_ALG3 && o.h_method != FLAPW_H_SPHERICAL &&
      o.h_method != FLAPW_H_ALG1)
    return fail(h, FLAPW_ERR_ARG, "options.h_method is not a FLAPW_H_* value");
  if (o.h_method == FLAPW_H_SPHERICAL && o.operands != FLAPW_OPERANDS_FACTORED)
    return fail(h, FLAPW_ERR_ARG, "options.h_method FLAPW_H_SPHERICAL needs FLAPW_OPERANDS_FACTORED");
  if (o.pipeline < 0 || o.pipeline > 2) return fail(h, FLAPW_ERR_ARG, "options.pipeline must be in 0..2");
  if (o.tile_cover < 0 || o.tile_cover > 2) return fail(h, FLAPW_ERR_ARG, "options.tile_cover must be in 0..2");
  if (o.wait_us < 0) return fail(h, FLAPW_ERR_ARG, "options.wait_us must be >= 0");
  if (o.part_count < 0 || o.part_index < 0 || o.part_index >= std::max(1, o.part_count))
    return fail(h, FLAPW_ERR_ARG, "options.part_index must be in 0..part_count-1");
  if (o.mem_cap_mb < 0) return fail(h, FLAPW_ERR_ARG, "options.mem_cap_mb must be >= 0");
  return FLAPW_OK;
}

int slices_of(const flapw_ctx* h) { return h->opt.n_slices ? h->opt.n_slices : 7; }

int device_setup(flapw_ctx* h) {
  CK(h, cudaGetDevice(&h->device), "cudaGetDevice");
  CK(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device),
     "cudaDeviceGetAttribute");
  {
    cudaDeviceProp prop;
    CK(h, cudaGetDeviceProperties(&prop, h->device), "cudaGetDeviceProperties");
    h->device_name = prop.name;
    for (char& c : h->device_name)
      if (c == ' ' || c == '/') c = '_';
  }
  for (auto& e : h->ev) CK(h, cudaEventCreate(&e), "cudaEventCreate");
  CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  CK(h, cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  CK(h, cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming), "cudaEventCreate");
  for (auto& e : h->pin_ev) CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
  CK(h, opform_init(), "constant table upload");
  return FLAPW_OK;
}

template <class T>
int upload(flapw_ctx* h, DevBuf& d, const std::vector<T>& v) {
  CK(h, d.ensure(v.size() * sizeof(T)), "cudaMalloc");
  if (!v.empty()) CK(h, cudaMemcpy(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "cudaMemcpy");
  return FLAPW_OK;
}

// First column block of the second part of a split H contraction: the last
// ~20 % of the lower-triangle tiles lie right of column 0.55 N_G.  With the
// output going to host memory at ~190 GB/s, that part's run time (~20 % of
// the launch) covers the copy of the first part's columns (~80 % of the
// bytes) on config-2-like shapes.
int h_split_block(int ng) { return (int)(0.55 * ((ng + 63) / 64)); }

// A job split over part_count independent callers (one per GPU, no
// communication; the k-points and the output tiles are independent, Sec. 5's
// multi-device split of the BLAS-3 calls and Sec. 6's k-point loop): whole
// k-points when there are at least as many as parts and the largest-first
// assignment (by N_G^2, to the least loaded part, ties to the lower index)
// keeps every part within 10 % of the mean load; otherwise every part takes
// every part_count-th contraction tile of each k-point.  owner[k] is the part
// of k-point k, or -1 when the k-points are shared by tiles.
void partition_owner(int n_k, const int64_t* ng, int parts, std::vector<int>* owner) {
  owner->assign(n_k, parts <= 1 ? 0 : -1);
  if (parts <= 1 || n_k < parts) return;
  std::vector<int> idx(n_k);
  for (int k = 0; k < n_k; ++k) idx[k] = k;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return ng[a] > ng[b]; });
  std::vector<double> load(parts, 0.0);
  std::vector<int> own(n_k);
  double total = 0;
  for (int k : idx) {
    const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    own[k] = r;
    load[r] += (double)ng[k] * (double)ng[k];
    total += (double)ng[k] * (double)ng[k];
  }
  if (*std::max_element(load.begin(), load.end()) <= 1.1 * total / parts) *owner = own;
}

// Emulated contraction tiles (one per CTA pair: a 64-column strip against four
// 64-row blocks, the cyclic cover of tiles.cuh) and FP64 tiles (64 x 64) of the
// lower triangles of problems [p0, p1).  The order of the emulated tiles
// decides which operand rows the ~75 concurrently running tiles share in L2:
// order 0 strip by strip; orders 1..5 bands of 4/8/16/32/64 row blocks of 64,
// strip by strip within a band.  cover_opt is the cyclic or the aligned cover
// (tiles.cuh), one for every problem of the handle (one kernel instantiation
// per launch).  part 0 takes every tile; 1 the strips below
// h_split_block(N_G), 2 the rest (an H contraction in two launches, so that the
// first part's columns can go to host memory while the second part runs; the
// cover is then cut at that strip, so the first part writes exactly the
// columns below it).  per_prob[p] counts the whole tiles of problem p.
void make_tiles(const std::vector<Prob>& probs, int p0, int p1, int order, int cover_opt, int pairs,
                std::vector<EmuTile>* emu, std::vector<F64Tile>* f64, int* n_split_ids,
                std::vector<int>* per_prob, const PartFilter& pf, int part = 0) {
  const size_t emu0 = emu->size();
  const int band = cover::order_band(order);
  for (int p = p0; p < p1; ++p) {
    if (pf.on && !(*pf.on)[p]) continue;
    const int ng = probs[p].n_g;
    const int ncb = (ng + 63) / 64;
    const int j1 = h_split_block(ng);
    const int s0 = (part == 2) ? j1 : 0, s1 = (part == 1) ? j1 : ncb;
    std::vector<EmuTile> pt;
    auto emit = [&](int jb, int mask, int r0, int r1, int r2, int r3) {
      pt.push_back(EmuTile{p, jb, 0, mask, {r0, r1, r2, r3}});
    };
    if (cover_opt == cover::kCoverCyclic)
      cover::for_each_tile(ncb, part ? j1 : ncb, s0, s1, emit);
    else
      cover::for_each_aligned_tile(ncb, s0, s1, emit);
    if (band > 0)
      std::stable_sort(pt.begin(), pt.end(), [band](const EmuTile& x, const EmuTile& y) {
        const int bx = x.rb[0] / band, by = y.rb[0] / band;
        return bx != by ? bx < by : x.jb < y.jb;
      });
    if (pf.stride > 1) {
      size_t w = 0;
      for (size_t i = 0; i < pt.size(); ++i)
        if ((int)(i % pf.stride) == pf.index) pt[w++] = pt[i];
      pt.resize(w);
    }
    if (per_prob) (*per_prob)[p] += (int)pt.size();
    emu->insert(emu->end(), pt.begin(), pt.end());
    const int nb = (ng + 63) / 64;
    int i64 = 0;
    for (int ib = 0; ib < nb; ++ib)
      for (int jb = 0; jb <= ib; ++jb)
        if (part == 0 || (part == 1) == (jb < j1))
          if (i64++ % pf.stride == pf.index) f64->push_back(F64Tile{p, ib, jb, 0});
  }
  // The pairs take the tiles round-robin, so the last rem = n mod pairs tiles
  // form a partly empty last wave.  Each of them becomes f K parts (f pairs
  // share it), so the last wave lasts 1/f of a tile.
  *n_split_ids = 0;
  const int n = (int)(emu->size() - emu0);
  if (pairs < 2 || n <= pairs) return;
  const int rem = n % pairs;
  const int f = rem ? std::min(kMaxSplit, pairs / rem) : 1;
  if (f < 2) return;
  std::vector<EmuTile> last(emu->end() - rem, emu->end());
  emu->resize(emu->size() - rem);
  for (int t = 0; t < rem; ++t)
    for (int part = 0; part < f; ++part) {
      EmuTile x = last[t];
      x.split = make_split(f, part, t);
      emu->push_back(x);
    }
  *n_split_ids = rem;
}

// Output pointers: device pointers are used in place; host pointers get a
// device staging area and a copy back after the contraction.
struct OutPlan {
  std::vector<double2*> dev;
  std::vector<void*> host;
  std::vector<size_t> bytes;
  std::vector<size_t> stage_off;
  size_t stage_bytes = 0;
};

// Width of the column blocks in which a full-layout output goes to host
// memory.  Each block is one 2D copy from the block's first diagonal element
// down, so nb blocks move the lower triangle plus the small triangles above
// the diagonal inside the blocks: about (1 + 1/nb) N_G^2 / 2 elements.  (The
// link to pinned host memory runs at ~190 GB/s on this part with 2D copies of
// such rows and with contiguous ones alike.)  Every copy takes an entry of the
// device's work queue, which holds about a thousand operations before an
// enqueueing call blocks until the GPU has drained some: with many host
// outputs in one call the blocks widen, so that a call enqueues at most about
// kCopyOps copies and two calls in flight still fit (32 blocks per matrix for
// one k-point, 5 for 32 k-points).
constexpr int kCopyOps = 320;
int64_t copy_block_cols(int64_t ng, int n_host) {
  const int nb = std::max(2, std::min(32, kCopyOps / std::max(1, n_host)));
  return std::max<int64_t>(64, (ng + nb - 1) / nb);
}

// Device-to-host copy of columns [c0, c1) of one output's lower triangle: the
// packed layout as one contiguous range, the full layout (ld = ng) in blocks
// of w columns (copy_block_cols).  Adds the copies and bytes to *ops, *bytes.
cudaError_t copy_out(void* dst, const double2* src, int64_t ng, int layout, int64_t c0, int64_t c1,
                     int64_t w, cudaStream_t st, int* ops, int64_t* bytes) {
  if (c1 <= c0) return cudaSuccess;
  char* d = static_cast<char*>(dst);
  const char* s = reinterpret_cast<const char*>(src);
  if (layout == FLAPW_LAYOUT_LOWER_PACKED) {
    const size_t o0 = (size_t)(c0 * ng - c0 * (c0 - 1) / 2) * 16;
    const size_t o1 = (size_t)(c1 * ng - c1 * (c1 - 1) / 2) * 16;
    *ops += 1;
    *bytes += (int64_t)(o1 - o0);
    return cudaMemcpyAsync(d + o0, s + o0, o1 - o0, cudaMemcpyDeviceToHost, st);
  }
  for (int64_t j0 = c0; j0 < c1; j0 += w) {
    const size_t off = (size_t)(j0 * ng + j0) * 16;
    const int64_t cols = std::min(w, c1 - j0);
    const cudaError_t e = cudaMemcpy2DAsync(d + off, (size_t)ng * 16, s + off, (size_t)ng * 16,
                                            (size_t)(ng - j0) * 16, (size_t)cols,
                                            cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    *ops += 1;
    *bytes += (ng - j0) * cols * 16;
  }
  return cudaSuccess;
}

size_t out_bytes(int layout, int64_t ng) {
  return (layout == FLAPW_LAYOUT_LOWER_PACKED) ? (size_t)(ng * (ng + 1) / 2) * 16
                                               : (size_t)(ng * ng) * 16;
}

// One half of the work: problems [p0, p1), operand rows [row0, row0 + nrows),
// tiles [t0, t0 + nt) of the uploaded lists.
struct Half {
  int64_t row0, nrows;
  int emu_t0, emu_nt, f64_t0, f64_nt;
};

// Bound of the tensor-core kernels' abortable device waits: options.wait_us,
// or 0 for the kernels' default (4 s).
unsigned long long wait_ns(const flapw_ctx* h) { return (unsigned long long)h->opt.wait_us * 1000ull; }

// The contraction's pipeline shape: the option, or by size.
bool use_deep_pipe(const flapw_ctx* h) {
  if (h->opt.autotune && h->pipe_choice) return h->pipe_choice == 2;
  return h->opt.pipeline == 2 || (h->opt.pipeline == 0 && h->deep_pipe);
}

// Split-tile scratch of the handle; its counts are zeroed on `st` first.
int split_scratch(flapw_ctx* h, cudaStream_t st, SplitScratch* out) {
  const size_t counts = (size_t)std::max(1, h->split_ids) * 2 * 8 * 4;
  const size_t total = split_scratch_bytes(std::max(1, h->split_ids));
  out->partial = h->d_split.as<long long>();
  out->count = reinterpret_cast<int*>(h->d_split.as<char>() + (total - counts));
  CK(h, cudaMemsetAsync(out->count, 0, counts, st), "cudaMemsetAsync");
  return FLAPW_OK;
}

// Slices (emulated precision; not if `presliced`, the slices being written
// already) and contracts one half beside concurrent work that holds busy_sms
// SMs.  Records ev_sl (if >= 0) after the slicer and ev_k after the contraction.
int enqueue_contraction(flapw_ctx* h, const Half& hf, int busy_sms, cudaStream_t st, int ev_sl,
                        int ev_k, bool presliced = false) {
  const int s = slices_of(h);
  const int64_t rows = h->rows;
  if (h->opt.precision == FLAPW_PREC_EMU) {
    if (!presliced)
      CK(h, launch_slicer(h->d_Z.as<double2>(), h->k_alloc, h->d_probs.as<Prob>(), h->d_rowprob.as<int>(),
                          0, rows, hf.row0, hf.nrows, s, h->d_SL.as<__half>(), h->d_rexp.as<int>(), st),
         "slicer launch");
    if (ev_sl >= 0) CK(h, cudaEventRecord(h->ev[ev_sl], st), "cudaEventRecord");
    SplitScratch sp{};
    if (int rc = split_scratch(h, st, &sp)) return rc;
    CK(h, launch_herk_emu(h->tmap, h->d_probs.as<Prob>(), h->d_emu_tiles.as<EmuTile>() + hf.emu_t0,
                          hf.emu_nt, h->d_rexp.as<int>(), s, fixed_frac_bits(h->k_terms),
                          h->d_cnt.as<int>() + 2, busy_sms, sp, use_deep_pipe(h),
                          h->tiles_cover == cover::kCoverCyclic, wait_ns(h), st),
       "emulated contraction launch");
  } else {
    if (ev_sl >= 0) CK(h, cudaEventRecord(h->ev[ev_sl], st), "cudaEventRecord");
    CK(h, launch_herk_f64(h->d_Z.as<double2>(), h->k_alloc, h->d_probs.as<Prob>(),
                          h->d_f64_tiles.as<F64Tile>() + hf.f64_t0, hf.f64_nt, st),
       "FP64 contraction launch");
  }
  CK(h, cudaEventRecord(h->ev[ev_k], st), "cudaEventRecord");
  return FLAPW_OK;
}

// Slice workspace and its tensor map (host-side; never inside stream capture).
int ensure_slices(flapw_ctx* h) {
  if (h->opt.precision != FLAPW_PREC_EMU) return FLAPW_OK;
  CK(h, herk_emu_init(), "contraction kernel setup");
  const int s = slices_of(h);
  CK(h, h->d_SL.ensure((size_t)s * 2 * h->rows * h->k_alloc * 2), "slice workspace");
  if (h->tmap_base != h->d_SL.p || h->tmap_k != h->k_alloc || h->tmap_rows != h->rows ||
      h->tmap_s != s) {
    std::string e;
    if (!make_slice_tmaps(&h->tmap, h->d_SL.p, h->k_alloc, h->rows, s, &e)) return fail(h, FLAPW_ERR_CUDA, e);
    h->tmap_base = h->d_SL.p;
    h->tmap_k = h->k_alloc;
    h->tmap_rows = h->rows;
    h->tmap_s = s;
  }
  return FLAPW_OK;
}

// Tile lists of problems [0, n_first) then [n_first, n_prob), the first half
// contracted beside busy_first busy SMs, the second beside busy_second.  With
// split_first the first half is two lists (make_tiles parts 1 and 2):
// *first, then *first_b.
int ensure_tiles(flapw_ctx* h, const std::vector<Prob>& probs, int n_first, int64_t key,
                 Half* first, Half* second, int busy_first = 0, int busy_second = 0,
                 bool split_first = false, Half* first_b = nullptr) {
  const int order = h->tile_order;
  int max_ng = 0;
  for (const Prob& p : probs) max_ng = std::max(max_ng, p.n_g);
  const int cover_opt = cover::cover_for(h->tile_cover, max_ng);
  int pf = 0, ps = 0;
  if (h->opt.precision == FLAPW_PREC_EMU) {
    CK(h, herk_emu_init(), "contraction kernel setup");
    pf = herk_emu_pairs(busy_first);
    ps = herk_emu_pairs(busy_second);
  }
  if (h->tiles_rows_key != key || h->tiles_order != order || h->tiles_cover != cover_opt ||
      h->tiles_pairs != pf * 1024 + ps || h->tiles_split != split_first || h->tiles_part != h->part_key) {
    std::vector<EmuTile> emu;
    std::vector<F64Tile> f64;
    int ids_first = 0, ids_second = 0, ids_b = 0;
    std::vector<int>* pp = &h->emu_tiles_per_prob;
    pp->assign(probs.size(), 0);
    make_tiles(probs, 0, n_first, order, cover_opt, pf, &emu, &f64, &ids_first, pp, h->part_filter,
               split_first ? 1 : 0);
    h->split_emu_b = (int)emu.size();
    h->split_f64_b = (int)f64.size();
    if (split_first)
      make_tiles(probs, 0, n_first, order, cover_opt, pf, &emu, &f64, &ids_b, pp, h->part_filter, 2);
    ids_first = std::max(ids_first, ids_b);
    h->split_emu = (int)emu.size();
    h->split_f64 = (int)f64.size();
    make_tiles(probs, n_first, (int)probs.size(), order, cover_opt, ps, &emu, &f64, &ids_second, pp,
               h->part_filter);
    h->n_emu_tiles = (int)emu.size();
    h->n_f64_tiles = (int)f64.size();
    if (int rc_up = upload(h, h->d_emu_tiles, emu)) return rc_up;
    if (int rc_up = upload(h, h->d_f64_tiles, f64)) return rc_up;
    // the halves run one after the other on one stream: they share the scratch
    h->split_ids = std::max(ids_first, ids_second);
    CK(h, h->d_split.ensure(split_scratch_bytes(std::max(1, h->split_ids))), "split-tile scratch");
    h->tiles_rows_key = key;
    h->tiles_order = order;
    h->tiles_cover = cover_opt;
    h->tiles_part = h->part_key;
    h->tiles_pairs = pf * 1024 + ps;
    h->tiles_split = split_first;
  }
  first->emu_t0 = 0;
  first->emu_nt = h->split_emu_b;
  first->f64_t0 = 0;
  first->f64_nt = h->split_f64_b;
  if (first_b) {
    first_b->emu_t0 = h->split_emu_b;
    first_b->emu_nt = h->split_emu - h->split_emu_b;
    first_b->f64_t0 = h->split_f64_b;
    first_b->f64_nt = h->split_f64 - h->split_f64_b;
  }
  second->emu_t0 = h->split_emu;
  second->emu_nt = h->n_emu_tiles - h->split_emu;
  second->f64_t0 = h->split_f64;
  second->f64_nt = h->n_f64_tiles - h->split_f64;
  return FLAPW_OK;
}

// Library default tile order for the handle's cover and largest N_G (tiles.cuh).
int default_tile_order(const flapw_ctx* h) { return cover::default_order(h->tile_cover, h->max_ng); }

// The tile order in use unless the autotuner picks it: the forced one, else
// the default for the cover.
void set_tile_order(flapw_ctx* h) {
  if (h->opt.tile_order > 0 && !h->opt.autotune) h->tile_order = h->opt.tile_order - 1;
  else h->tile_order = default_tile_order(h);
}

// Autotuner choices by problem shape: kept for the process and, if the
// environment variable FLAPW_AUTOTUNE_CACHE names a file, read from it once
// and appended to it, one line "shape cover order pipeline" per shape.
struct Tuned {
  int cover, order, pipe;
};
std::mutex g_tune_mutex;
std::map<std::string, Tuned> g_tuned;
bool g_tune_file_read = false;

const char* tune_file() {
  const char* f = std::getenv("FLAPW_AUTOTUNE_CACHE");
  return (f && *f) ? f : nullptr;
}

// The shape key: GPU, slice count, H and S methods, K of the H contraction
// and every problem's N_G (hashed).
std::string shape_key(const flapw_ctx* h, const std::vector<Prob>& probs) {
  uint64_t x = 1469598103934665603ull;  // FNV-1a over the N_G list
  for (const Prob& p : probs) {
    x ^= (uint64_t)p.n_g;
    x *= 1099511628211ull;
  }
  std::ostringstream o;
  o << h->device_name << "/sm" << h->num_sms << "/s" << slices_of(h) << "/h" << h->opt.h_method << "/s"
    << h->opt.s_method << "/k" << h->k_terms << "/p" << probs.size() << "/" << std::hex << x;
  return o.str();
}

bool tuned_lookup(const std::string& key, Tuned* t) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  if (!g_tune_file_read) {
    g_tune_file_read = true;
    if (const char* f = tune_file()) {
      std::ifstream in(f);
      std::string k;
      Tuned v;
      while (in >> k >> v.cover >> v.order >> v.pipe)
        if (v.cover >= 1 && v.cover <= 2 && v.order >= 0 && v.order < kNumTileOrders && v.pipe >= 1 &&
            v.pipe <= 2)
          g_tuned[k] = v;
    }
  }
  auto it = g_tuned.find(key);
  if (it == g_tuned.end()) return false;
  *t = it->second;
  return true;
}

void tuned_store(const std::string& key, const Tuned& t) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tuned[key] = t;
  if (const char* f = tune_file()) {
    std::ofstream out(f, std::ios::app);
    out << key << " " << t.cover << " " << t.order << " " << t.pipe << "\n";
  }
}

void apply_tuned(flapw_ctx* h, const Tuned& t) {
  h->tile_cover = t.cover;
  h->tile_order = t.order;
  h->pipe_choice = t.pipe;
}

// Times the emulated contraction (both halves) on the slices the last build
// left in place, the outputs rewritten with the same values, and picks the
// tile cover, the tile order and the load pipeline by coordinate descent from
// the size-based defaults: the pipeline, then the other cover (with its default
// order), then every order.
int autotune_tiles(flapw_ctx* h, const std::vector<Prob>& probs, int n_first, int64_t key,
                   int n_slots, const std::string& shape, cudaStream_t st) {
  CK(h, cudaStreamSynchronize(st), "cudaStreamSynchronize");
  CK(h, cudaStreamSynchronize(h->aux_stream), "cudaStreamSynchronize");
  const int s = slices_of(h);
  int max_ng = 0;
  for (const Prob& p : probs) max_ng = std::max(max_ng, p.n_g);
  auto time_cfg = [&](const Tuned& c, float* out) -> int {
    apply_tuned(h, c);
    Half a, b;
    if (int rc = ensure_tiles(h, probs, n_first, key, &a, &b, 0, n_slots)) return rc;
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      CK(h, cudaEventRecord(h->ev[14], st), "cudaEventRecord");
      for (const Half* hf : {&b, &a}) {
        SplitScratch sp{};
        if (int rc = split_scratch(h, st, &sp)) return rc;
        CK(h, launch_herk_emu(h->tmap, h->d_probs.as<Prob>(), h->d_emu_tiles.as<EmuTile>() + hf->emu_t0,
                              hf->emu_nt, h->d_rexp.as<int>(), s, fixed_frac_bits(h->k_terms),
                              h->d_cnt.as<int>() + 2, 0, sp, use_deep_pipe(h),
                              h->tiles_cover == cover::kCoverCyclic, wait_ns(h), st),
           "emulated contraction launch");
      }
      CK(h, cudaEventRecord(h->ev[15], st), "cudaEventRecord");
      CK(h, cudaEventSynchronize(h->ev[15]), "cudaEventSynchronize");
      float ms = 0.f;
      CK(h, cudaEventElapsedTime(&ms, h->ev[14], h->ev[15]), "cudaEventElapsedTime");
      best = std::min(best, ms);
      if (ms > 200.f) break;  // long launches: one repetition is enough
    }
    *out = best;
    return FLAPW_OK;
  };
  const int cov0 = cover::cover_for(cover::kCoverAuto, max_ng);
  Tuned cur{cov0, cover::default_order(cov0, max_ng), herk_emu_deep(max_ng) ? 2 : 1};
  float t_cur = 0.f;
  if (int rc = time_cfg(cur, &t_cur)) return rc;
  auto try_cfg = [&](Tuned c) -> int {
    float t = 0.f;
    if (int rc = time_cfg(c, &t)) return rc;
    if (t < t_cur) {
      t_cur = t;
      cur = c;
    }
    return FLAPW_OK;
  };
  if (int rc = try_cfg(Tuned{cur.cover, cur.order, 3 - cur.pipe})) return rc;
  if (int rc = try_cfg(Tuned{3 - cur.cover, cover::default_order(3 - cur.cover, max_ng), cur.pipe})) return rc;
  const int o0 = cur.order;
  for (int o = 0; o < kNumTileOrders; ++o)
    if (o != o0)
      if (int rc = try_cfg(Tuned{cur.cover, o, cur.pipe})) return rc;
  apply_tuned(h, cur);
  Half a, b;
  if (int rc = ensure_tiles(h, probs, n_first, key, &a, &b, 0, n_slots)) return rc;
  tuned_store(shape, cur);
  h->tuned_shape = shape;
  return FLAPW_OK;
}

}  // namespace

extern "C" {

void flapw_default_options(flapw_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = FLAPW_PREC_EMU;
  opt->n_slices = 7;
  opt->layout = FLAPW_LAYOUT_LOWER_FULL;
  opt->operands = FLAPW_OPERANDS_FROM_AB;
  opt->use_graph = 0;
  opt->autotune = 0;
}

int flapw_enumerate_g(const double lattice[9], const double k_frac[3], double kmax, int max_g,
                      int* n3, int* n_g) {
  if (!lattice || !k_frac || !n_g) return fail(nullptr, FLAPW_ERR_ARG, "NULL argument");
  std::vector<int> v;
  const int n = enumerate_g(lattice, k_frac, kmax, &v);
  if (n < 0) return fail(nullptr, FLAPW_ERR_ARG, "singular lattice or kmax <= 0");
  *n_g = n;
  if (n3) std::memcpy(n3, v.data(), sizeof(int) * 3 * (size_t)std::min(n, std::max(max_g, 0)));
  return FLAPW_OK;
}

int flapw_set_spherical_T(flapw_handle h, const double* t_sph, int n_slots) {
  if (!h) return fail(h, FLAPW_ERR_ARG, "NULL handle");
  if (h->engine_only) return fail(h, FLAPW_ERR_STATE, "handle has no crystal");
  if (!t_sph || n_slots < 1) {
    h->tsph.clear();
    h->tsph_slots = 0;
    h->tsph_lmax = -1;
    return FLAPW_OK;
  }
  const size_t n = (size_t)n_slots * (h->lmax + 1) * 4;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(t_sph[i])) return fail(h, FLAPW_ERR_ARG, "t_sph entries must be finite");
  h->tsph.assign(t_sph, t_sph + n);
  h->tsph_slots = n_slots;
  h->tsph_lmax = h->lmax;
  return FLAPW_OK;
}

int flapw_partition(int n_k, const int* n_g, int part_count, int* owner) {
  if (n_k < 0 || (n_k > 0 && (!n_g || !owner)) || part_count < 1)
    return fail(nullptr, FLAPW_ERR_ARG, "need n_k >= 0, n_g and owner, part_count >= 1");
  std::vector<int64_t> ng(n_g, n_g + n_k);
  std::vector<int> own;
  partition_owner(n_k, ng.data(), part_count, &own);
  std::copy(own.begin(), own.end(), owner);
  return FLAPW_OK;
}

int flapw_engine_create(const flapw_options* opt, flapw_handle* out) {
  if (!out) return fail(nullptr, FLAPW_ERR_ARG, "NULL out");
  std::unique_ptr<flapw_ctx> h(new flapw_ctx);
  flapw_default_options(&h->opt);
  if (opt) h->opt = *opt;
  if (check_options(nullptr, h->opt)) return FLAPW_ERR_ARG;
  h->tile_cover = h->opt.tile_cover;
  set_tile_order(h.get());
  h->engine_only = true;
  if (int rc = device_setup(h.get())) {
    g_last_error = h->err;
    return rc;
  }
  *out = h.release();
  return FLAPW_OK;
}

int flapw_hs_create(const double lattice[9], int n_atoms, const double* pos_frac,
                    const int* atom_type, int n_types, const double* mt_radius, int lmax,
                    int n_k, const double* k_frac, const double* kmax,
                    const flapw_options* opt, flapw_handle* out) {
  if (!out || !lattice || !pos_frac || !atom_type || !mt_radius || !k_frac || !kmax)
    return fail(nullptr, FLAPW_ERR_ARG, "NULL argument");
  if (n_atoms < 1 || n_types < 1 || n_k < 1) return fail(nullptr, FLAPW_ERR_ARG, "n_atoms, n_types and n_k must be >= 1");
  if (lmax < 0 || lmax > kMaxLmax) return fail(nullptr, FLAPW_ERR_UNSUPPORTED, "lmax must be in 0..12");
  for (int a = 0; a < n_atoms; ++a)
    if (atom_type[a] < 0 || atom_type[a] >= n_types) return fail(nullptr, FLAPW_ERR_ARG, "atom_type out of range");
  for (int t = 0; t < n_types; ++t)
    if (!(mt_radius[t] > 0)) return fail(nullptr, FLAPW_ERR_ARG, "mt_radius must be > 0");
  std::unique_ptr<flapw_ctx> h(new flapw_ctx);
  flapw_default_options(&h->opt);
  if (opt) h->opt = *opt;
  if (check_options(nullptr, h->opt)) return FLAPW_ERR_ARG;
  h->tile_cover = h->opt.tile_cover;
  std::memcpy(h->lat, lattice, sizeof(h->lat));
  double det;
  reciprocal(h->lat, h->rec, &det);
  if (!(std::fabs(det) > 0)) return fail(nullptr, FLAPW_ERR_ARG, "singular lattice");
  h->volume = std::fabs(det);
  h->n_atoms = n_atoms;
  h->n_types = n_types;
  h->lmax = lmax;
  h->n_L = (lmax + 1) * (lmax + 1);
  h->n_k = n_k;
  h->pos.assign(pos_frac, pos_frac + 3 * n_atoms);
  h->type.assign(atom_type, atom_type + n_atoms);
  h->radius.assign(mt_radius, mt_radius + n_types);
  h->kfrac.assign(k_frac, k_frac + 3 * n_k);
  h->kmax.assign(kmax, kmax + n_k);
  h->n3.resize(n_k);
  h->goff.assign(n_k + 1, 0);
  for (int k = 0; k < n_k; ++k) {
    const int ng = enumerate_g(h->lat, &h->kfrac[3 * k], h->kmax[k], &h->n3[k]);
    if (ng < 0) return fail(nullptr, FLAPW_ERR_ARG, "kmax must be > 0");
    if (ng == 0) return fail(nullptr, FLAPW_ERR_ARG, "a k-point has no plane wave below kmax");
    h->goff[k + 1] = h->goff[k] + ng;
  }
  h->g_total = h->goff[n_k];
  if (h->g_total > (int64_t)1 << 30) return fail(nullptr, FLAPW_ERR_UNSUPPORTED, "too many plane waves");
  int64_t max_ng = 0;
  for (int k = 0; k < n_k; ++k) max_ng = std::max<int64_t>(max_ng, h->goff[k + 1] - h->goff[k]);
  h->max_ng = max_ng;
  h->deep_pipe = herk_emu_deep(max_ng);
  set_tile_order(h.get());
  h->ktau.resize((size_t)n_k * n_atoms);
  for (int k = 0; k < n_k; ++k)
    for (int a = 0; a < n_atoms; ++a)
      h->ktau[(size_t)k * n_atoms + a] = h->kfrac[3 * k] * h->pos[3 * a] +
                                         h->kfrac[3 * k + 1] * h->pos[3 * a + 1] +
                                         h->kfrac[3 * k + 2] * h->pos[3 * a + 2];
  for (int k = 0; k < n_k; ++k) {
    const int ng = (int)(h->goff[k + 1] - h->goff[k]);
    for (int g0 = 0; g0 < ng; g0 += 128) {
      h->gt128.push_back(k);
      h->gt128.push_back(g0);
    }
    for (int g0 = 0; g0 < ng; g0 += 64) {
      h->gt64.push_back(k);
      h->gt64.push_back(g0);
    }
  }
  if (int rc = device_setup(h.get())) {
    g_last_error = h->err;
    return rc;
  }
  // geometry to the device
  std::vector<double> rec(h->rec, h->rec + 9);
  std::vector<int> n3all, gk;
  n3all.reserve(3 * h->g_total);
  gk.reserve(h->g_total);
  for (int k = 0; k < n_k; ++k) {
    n3all.insert(n3all.end(), h->n3[k].begin(), h->n3[k].end());
    gk.insert(gk.end(), h->n3[k].size() / 3, k);
  }
  // normalised-Legendre recurrence coefficients, index 2*(l(l+1)/2 + m)
  std::vector<double> coef((size_t)(lmax + 2) * (lmax + 3), 0.0);
  for (int l = 0; l <= lmax; ++l)
    for (int m = 0; m <= l; ++m) {
      const size_t i = 2 * ((size_t)l * (l + 1) / 2 + m);
      if (l == m) {
        coef[i] = (m > 0) ? std::sqrt((2.0 * m + 1.0) / (2.0 * m)) : 0.0;
      } else if (l == m + 1) {
        coef[i] = std::sqrt(2.0 * m + 3.0);
      } else {
        coef[i] = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        coef[i + 1] = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) /
                                (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      }
    }
  flapw_ctx* hp = h.get();
  if (upload(hp, h->d_rec, rec) || upload(hp, h->d_pos, h->pos) || upload(hp, h->d_type, h->type) ||
      upload(hp, h->d_radius, h->radius) || upload(hp, h->d_kfrac, h->kfrac) ||
      upload(hp, h->d_ktau, h->ktau) || upload(hp, h->d_n3, n3all) || upload(hp, h->d_gk, gk) ||
      upload(hp, h->d_goff, h->goff) || upload(hp, h->d_coef, coef) ||
      upload(hp, h->d_gt128, h->gt128) || upload(hp, h->d_gt64, h->gt64)) {
    g_last_error = h->err;
    return FLAPW_ERR_CUDA;
  }
  *out = h.release();
  return FLAPW_OK;
}

int flapw_set_options(flapw_handle h, const flapw_options* opt) {
  if (!h || !opt) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  if (int rc = check_options(h, *opt)) return rc;
  h->opt = *opt;
  if (!opt->autotune) {
    h->tile_cover = opt->tile_cover;
    h->pipe_choice = 0;
    h->tuned_shape.clear();
    set_tile_order(h);
  }
  return FLAPW_OK;
}

int flapw_num_g(flapw_handle h, int k, int* n_g) {
  if (!h || !n_g) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  if (h->engine_only) return fail(h, FLAPW_ERR_STATE, "handle has no crystal");
  if (k < 0 || k >= h->n_k) return fail(h, FLAPW_ERR_ARG, "k out of range");
  *n_g = (int)(h->goff[k + 1] - h->goff[k]);
  return FLAPW_OK;
}

int flapw_get_gvectors(flapw_handle h, int k, int* n3) {
  if (!h || !n3) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  if (h->engine_only) return fail(h, FLAPW_ERR_STATE, "handle has no crystal");
  if (k < 0 || k >= h->n_k) return fail(h, FLAPW_ERR_ARG, "k out of range");
  std::memcpy(n3, h->n3[k].data(), sizeof(int) * h->n3[k].size());
  return FLAPW_OK;
}

int flapw_ab_offset(flapw_handle h, int k, int64_t* offset) {
  if (!h || !offset) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  if (h->engine_only) return fail(h, FLAPW_ERR_STATE, "handle has no crystal");
  if (k < 0 || k > h->n_k) return fail(h, FLAPW_ERR_ARG, "k out of range");
  *offset = (int64_t)h->n_atoms * h->n_L * h->goff[k];
  return FLAPW_OK;
}

static int prepare_prep(flapw_ctx* h, cudaStream_t st) {
  const int64_t G = h->g_total;
  CK(h, h->d_Yc.ensure((size_t)h->n_L * G * 16), "workspace");
  CK(h, h->d_al.ensure((size_t)h->n_types * (h->lmax + 1) * G * 8), "workspace");
  CK(h, h->d_bl.ensure((size_t)h->n_types * (h->lmax + 1) * G * 8), "workspace");
  CK(h, h->d_ph.ensure((size_t)h->n_atoms * G * 16), "workspace");
  Geom geo{h->n_atoms, h->n_types, h->lmax, h->n_L, h->n_k, G,
           h->d_rec.as<double>(), h->d_pos.as<double>(), h->d_type.as<int>(),
           h->d_radius.as<double>(), h->d_kfrac.as<double>(), h->d_ktau.as<double>(),
           4.0 * M_PI / std::sqrt(h->volume)};
  GData gd{h->d_n3.as<int>(), h->d_gk.as<int>(), h->d_goff.as<int64_t>()};
  CK(h, launch_ab_prep(geo, gd, h->d_radial.as<double>(), h->d_coef.as<double>(),
                       h->d_Yc.as<double2>(), h->d_al.as<double>(), h->d_bl.as<double>(),
                       h->d_ph.as<double2>(), st),
     "A/B preparation launch");
  h->prep_valid = true;
  return FLAPW_OK;
}

int flapw_build_AB(flapw_handle h, const double* radial, void* A, void* B, void* stream) {
  (void)cudaGetLastError();  // a stale error of unrelated code must not fail our launch checks
  if (!h || !radial || !A || !B) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  BudgetScope budget_scope(h);
  if (h->engine_only) return fail(h, FLAPW_ERR_STATE, "handle has no crystal");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nrad = (size_t)h->n_types * (h->lmax + 1) * 4;
  for (size_t i = 0; i < nrad; i += 4) {
    const double D = radial[i] * radial[i + 3] - radial[i + 1] * radial[i + 2];
    if (!(D != 0.0) || !std::isfinite(D))
      return fail(h, FLAPW_ERR_ARG, "radial data: u udot' - u' udot must be finite and nonzero");
  }
  h->radial.assign(radial, radial + nrad);
  h->have_radial = true;
  CK(h, h->d_radial.ensure(nrad * 8), "workspace");
  CK(h, cudaMemcpyAsync(h->d_radial.p, h->radial.data(), nrad * 8, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
  CK(h, cudaEventRecord(h->ev[6], st), "cudaEventRecord");
  if (int rc = prepare_prep(h, st)) return rc;
  const size_t total = (size_t)h->n_atoms * h->n_L * h->g_total;
  const bool devA = is_device_ptr(A), devB = is_device_ptr(B);
  double2* dA = static_cast<double2*>(A);
  double2* dB = static_cast<double2*>(B);
  if (!devA) {
    CK(h, h->d_stageA.ensure(total * 16), "staging");
    dA = h->d_stageA.as<double2>();
  }
  if (!devB) {
    CK(h, h->d_stageB.ensure(total * 16), "staging");
    dB = h->d_stageB.as<double2>();
  }
  Geom geo{h->n_atoms, h->n_types, h->lmax, h->n_L, h->n_k, h->g_total,
           h->d_rec.as<double>(), h->d_pos.as<double>(), h->d_type.as<int>(),
           h->d_radius.as<double>(), h->d_kfrac.as<double>(), h->d_ktau.as<double>(),
           4.0 * M_PI / std::sqrt(h->volume)};
  CK(h, cudaEventRecord(h->ev[17], st), "cudaEventRecord");
  CK(h, launch_ab_assemble_tiles(geo, h->d_gt128.as<int>(), (int)(h->gt128.size() / 2),
                                 h->d_goff.as<int64_t>(), h->d_Yc.as<double2>(), h->d_al.as<double>(),
                                 h->d_bl.as<double>(), h->d_ph.as<double2>(), dA, dB, st),
     "A/B assembly launch");
  CK(h, cudaEventRecord(h->ev[7], st), "cudaEventRecord");
  h->ev_ab = true;
  if (!devA) CK(h, cudaMemcpyAsync(A, dA, total * 16, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  if (!devB) CK(h, cudaMemcpyAsync(B, dB, total * 16, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  h->last_stream = st;
  return FLAPW_OK;
}

int flapw_build_HS(flapw_handle h, const double* T, int n_slots, const int* atom_slot,
                   const double* U, const void* A, const void* B, void* const* H,
                   void* const* S, void* stream) {
  (void)cudaGetLastError();  // a stale error of unrelated code must not fail our launch checks
  if (!h || !T || !atom_slot || !U || !H || !S) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  BudgetScope budget_scope(h);
  if (h->engine_only) return fail(h, FLAPW_ERR_STATE, "handle has no crystal");
  const bool factored = h->opt.operands == FLAPW_OPERANDS_FACTORED;
  if (!factored && (!A || !B)) return fail(h, FLAPW_ERR_ARG, "A and B are required with FLAPW_OPERANDS_FROM_AB");
  if (factored && !h->have_radial)
    return fail(h, FLAPW_ERR_STATE, "FLAPW_OPERANDS_FACTORED needs a previous flapw_build_AB");
  if (n_slots < 1) return fail(h, FLAPW_ERR_ARG, "n_slots must be >= 1");
  for (int a = 0; a < h->n_atoms; ++a)
    if (atom_slot[a] < 0 || atom_slot[a] >= n_slots) return fail(h, FLAPW_ERR_ARG, "atom_slot out of range");
  // this caller's part of a partitioned job: whole k-points, or every P-th tile
  {
    const int parts = std::max(1, h->opt.part_count);
    std::vector<int64_t> ngk(h->n_k);
    for (int k = 0; k < h->n_k; ++k) ngk[k] = h->goff[k + 1] - h->goff[k];
    std::vector<int> owner;
    partition_owner(h->n_k, ngk.data(), parts, &owner);
    const bool by_tiles = parts > 1 && h->n_k > 0 && owner[0] < 0;
    h->part_on.assign(2 * h->n_k, 1);
    for (int k = 0; k < h->n_k; ++k)
      h->part_on[k] = h->part_on[h->n_k + k] = (parts == 1 || by_tiles || owner[k] == h->opt.part_index);
    h->part_filter.on = &h->part_on;
    h->part_filter.stride = by_tiles ? parts : 1;
    h->part_filter.index = by_tiles ? h->opt.part_index : 0;
    h->part_key = std::to_string(parts) + "/" + std::to_string(h->opt.part_index);
  }
  for (int k = 0; k < h->n_k; ++k)
    if (h->part_on[k] && (!H[k] || !S[k])) return fail(h, FLAPW_ERR_ARG, "NULL H[k] or S[k]");
  cudaStream_t user_st = static_cast<cudaStream_t>(stream);
  const int n = 2 * h->n_L;
  const int nlp = h->lmax + 1;
  const int nk = h->n_k;
  const int64_t K = (int64_t)h->n_atoms * n;
  // H by the paper's Alg. 3: L^H R over 3 N_A N_L rows, no factorisation
  // Alg. 1 is Alg. 3's stacked contraction with C^H in place of T^AA where the
  // Cholesky factorisation of T^AA succeeds (alg3.cuh)
  const bool alg1 = h->opt.h_method == FLAPW_H_ALG1;
  const bool alg3 = h->opt.h_method == FLAPW_H_ALG3 || alg1;
  // H from the spherical part of T by the addition theorem plus the contraction
  // of the rest (which is skipped when the rest is zero)
  const bool h_sph = h->opt.h_method == FLAPW_H_SPHERICAL;
  bool h_zero = false;
  if (h_sph && (h->tsph_slots != n_slots || h->tsph_lmax != h->lmax))
    return fail(h, FLAPW_ERR_STATE, "FLAPW_H_SPHERICAL needs flapw_set_spherical_T for these n_slots");
  const size_t tsph_bytes = h_sph ? h->tsph.size() * sizeof(double) : 0;
  const int64_t K_H = alg3 ? (int64_t)h->n_atoms * 3 * h->n_L : K;
  if (K_H >= ((int64_t)1 << 17))
    return fail(h, FLAPW_ERR_UNSUPPORTED, "the H contraction's K (2 N_A N_L, or 3 N_A N_L for Alg. 3) must be below 131072");
  const int layout = h->opt.layout;

  // ---- host-side preparation (never captured) ----
  const size_t t_bytes = (size_t)n_slots * n * n * 16;
  const size_t slot_bytes = (size_t)h->n_atoms * 4;
  const size_t u_bytes = (size_t)h->n_types * nlp * 8;
  // factored operands: (slot, type) pairs and their atoms
  std::vector<int> combo_slot, combo_type, combo_atoms, combo_start{0};
  if (factored) {
    std::map<std::pair<int, int>, std::vector<int>> cmb;
    for (int a = 0; a < h->n_atoms; ++a) cmb[{atom_slot[a], h->type[a]}].push_back(a);
    for (auto& kv : cmb) {
      combo_slot.push_back(kv.first.first);
      combo_type.push_back(kv.first.second);
      combo_atoms.insert(combo_atoms.end(), kv.second.begin(), kv.second.end());
      combo_start.push_back((int)combo_atoms.size());
    }
  }
  const int n_combo = (int)combo_slot.size();
  const size_t cmb_ints = combo_slot.size() * 2 + combo_atoms.size() + combo_start.size();

  // outputs: problem k = H of k-point k, problem nk + k = S of k-point k
  OutPlan op;
  op.dev.resize(2 * nk);
  op.host.assign(2 * nk, nullptr);
  op.bytes.resize(2 * nk);
  op.stage_off.resize(2 * nk);
  for (int w = 0; w < 2; ++w)
    for (int k = 0; k < nk; ++k) {
      const int64_t ng = h->goff[k + 1] - h->goff[k];
      void* ptr = w ? S[k] : H[k];
      const int idx = w * nk + k;
      op.bytes[idx] = out_bytes(layout, ng);
      if (!h->part_on[idx]) {  // another part's k-point: nothing written or copied
        op.dev[idx] = nullptr;
        continue;
      }
      if (is_device_ptr(ptr)) {
        op.dev[idx] = static_cast<double2*>(ptr);
      } else {
        op.host[idx] = ptr;
        op.stage_off[idx] = op.stage_bytes;
        op.stage_bytes += round_up((int64_t)op.bytes[idx], 256);
      }
    }
  if (op.stage_bytes) {
    CK(h, h->d_stageOut.ensure(op.stage_bytes), "staging");
    for (int i = 0; i < 2 * nk; ++i)
      if (op.host[i]) op.dev[i] = reinterpret_cast<double2*>(h->d_stageOut.as<char>() + op.stage_off[i]);
  }
  // A/B in host memory are staged through the device
  const size_t ab_total = (size_t)h->n_atoms * h->n_L * h->g_total;
  const double2* dA = static_cast<const double2*>(A);
  const double2* dB = static_cast<const double2*>(B);
  bool stage_ab = false;
  if (!factored && (!is_device_ptr(A) || !is_device_ptr(B))) {
    CK(h, h->d_stageA.ensure(ab_total * 16), "staging");
    CK(h, h->d_stageB.ensure(ab_total * 16), "staging");
    stage_ab = true;
    dA = h->d_stageA.as<double2>();
    dB = h->d_stageB.as<double2>();
  }
  // problems: H rows are [0, G_total), S rows [G_total, 2 G_total); with Alg. 3
  // the H rows hold L, rows [G_total, 2 G_total) R, and S follows at 2 G_total.
  // The H problems' K split (sigma = +1 / -1) comes from the factorisation.
  const int64_t s_row0 = alg3 ? 2 * h->g_total : h->g_total;
  std::vector<Prob> probs(2 * nk);
  for (int k = 0; k < nk; ++k) {
    const int ng = (int)(h->goff[k + 1] - h->goff[k]);
    const int hb = (int)h->goff[k], sb = (int)(s_row0 + h->goff[k]);
    probs[k] = Prob{hb, ng, alg3 ? (int)K_H : 0, 0, layout, alg3 ? (int)(h->g_total + hb) : hb, ng, op.dev[k]};
    probs[nk + k] = Prob{sb, ng, (int)K, 0, layout, sb, ng, op.dev[nk + k]};
  }
  h->rows = alg3 ? 3 * h->g_total : 2 * h->g_total;
  h->k_alloc = alg3 ? round_up(K_H, kChunk) : round_up(K, kChunk) + kChunk;
  h->k_terms = K_H;
  CK(h, h->d_T.ensure(t_bytes), "workspace");
  CK(h, h->d_work.ensure(t_bytes), "workspace");
  CK(h, h->d_CH.ensure(t_bytes), "workspace");
  CK(h, h->d_hpd.ensure(sizeof(int) * (size_t)std::max(n_slots, 1)), "workspace");
  // S by the addition theorem: Khat of every plane wave and the atoms grouped
  // by type, both fixed by the crystal (computed once)
  const bool s_legendre = h->opt.s_method == FLAPW_S_LEGENDRE;
  if (h_sph) CK(h, h->d_tsph.ensure(tsph_bytes), "workspace");
  if ((s_legendre || h_sph) && !h->khat_valid) {
    std::vector<int> ta;
    std::vector<int> start{0};
    for (int t = 0; t < h->n_types; ++t) {
      for (int a = 0; a < h->n_atoms; ++a)
        if (h->type[a] == t) ta.push_back(a);
      start.push_back((int)ta.size());
    }
    ta.insert(ta.end(), start.begin(), start.end());
    if (int rc_up = upload(h, h->d_typeatoms, ta)) return rc_up;
    CK(h, h->d_khat.ensure((size_t)h->g_total * 3 * 8), "workspace");
    Geom geo{h->n_atoms, h->n_types, h->lmax, h->n_L, h->n_k, h->g_total,
             h->d_rec.as<double>(), h->d_pos.as<double>(), h->d_type.as<int>(),
             h->d_radius.as<double>(), h->d_kfrac.as<double>(), h->d_ktau.as<double>(),
             4.0 * M_PI / std::sqrt(h->volume)};
    GData gd{h->d_n3.as<int>(), h->d_gk.as<int>(), h->d_goff.as<int64_t>()};
    CK(h, launch_khat(geo, gd, h->d_khat.as<double>(), nullptr), "Khat launch");
    CK(h, cudaDeviceSynchronize(), "Khat");
    h->khat_valid = true;
  }
  if (s_legendre && h->opt.precision == FLAPW_PREC_EMU)
    CK(h, h->d_sdf.ensure(slegendre_df_floats2(h->n_types, h->lmax, h->n_atoms, h->g_total) * 8),
       "workspace");
  if (h_sph && h->opt.precision == FLAPW_PREC_EMU)
    CK(h, h->d_hdf.ensure(slegendre_df_floats2(h->n_types, h->lmax, h->n_atoms, h->g_total) * 8),
       "workspace");
  // emulated path with factored operands: the H operands come from the
  // tensor-core product of conj(C^H) and W (opgemm.cu)
  // (for Alg. 3 the product of M = [[T^BA, T^BB/2], [T^AA, 0]] and W)
  const bool tc_ops = factored && h->opt.precision == FLAPW_PREC_EMU;
  const int op_kp = round_up(n, kChunk);
  const int64_t op_rows_a = (int64_t)n_slots * n, op_rows_b = (int64_t)h->n_types * h->g_total;
  if (tc_ops) {
    CK(h, opgemm_init(), "operand kernel setup");
    CK(h, h->d_opA.ensure((size_t)op_rows_a * op_kp * 16), "operand workspace");
    CK(h, h->d_opB.ensure((size_t)op_rows_b * op_kp * 16), "operand workspace");
    CK(h, h->d_opSLA.ensure((size_t)kOpSlices * 2 * op_rows_a * op_kp * 2), "operand workspace");
    CK(h, h->d_opSLB.ensure((size_t)kOpSlices * 2 * op_rows_b * op_kp * 2), "operand workspace");
    CK(h, h->d_oprexp.ensure((size_t)(op_rows_a + op_rows_b) * 4), "workspace");
    CK(h, h->d_opP.ensure((size_t)n_combo * h->g_total * n * 16), "operand workspace");
    std::vector<OpTile> tl;
    const int nrb = (n + 127) / 128;
    const int64_t ngb = (h->g_total + 63) / 64;
    for (int c = 0; c < n_combo; ++c)
      for (int64_t gb = 0; gb < ngb; ++gb)
        for (int rb = 0; rb < nrb; ++rb) tl.push_back(OpTile{c, rb, (int)gb, 0});
    if (tl.size() != h->optiles.size() || !std::equal(tl.begin(), tl.end(), h->optiles.begin(),
                                                       [](const OpTile& x, const OpTile& y) {
                                                         return x.combo == y.combo && x.rb == y.rb && x.gb == y.gb;
                                                       })) {
      if (int rc_up = upload(h, h->d_optiles, tl)) return rc_up;
      h->optiles = tl;
    }
    if (h->opmap_a_base != h->d_opSLA.p || h->opmap_a_rows != op_rows_a || h->opmap_kp != op_kp ||
        h->opmap_b_base != h->d_opSLB.p || h->opmap_b_rows != op_rows_b) {
      std::string e;
      if (!make_tmap_4d(&h->opmap_a, h->d_opSLA.p, op_kp, op_rows_a, kOpSlices, 128, 1, &e) ||
          !make_tmap_4d(&h->opmap_b, h->d_opSLB.p, op_kp, op_rows_b, kOpSlices, 64, 2, &e))
        return fail(h, FLAPW_ERR_CUDA, e);
      h->opmap_a_base = h->d_opSLA.p;
      h->opmap_b_base = h->d_opSLB.p;
      h->opmap_a_rows = op_rows_a;
      h->opmap_b_rows = op_rows_b;
      h->opmap_kp = op_kp;
    }
  }
  CK(h, h->d_fac.ensure(sizeof(int) * 2 * (size_t)n_slots * n), "workspace");
  CK(h, h->d_cnt.ensure(sizeof(int) * (8 + 2 * (size_t)n_slots)), "workspace");
  CK(h, h->d_slot.ensure(slot_bytes + cmb_ints * 4 + 64), "workspace");
  CK(h, h->d_U.ensure(u_bytes), "workspace");
  CK(h, h->d_off.ensure(sizeof(int) * (2 * (size_t)h->n_atoms + 8)), "workspace");
  CK(h, h->d_probs.ensure(sizeof(Prob) * probs.size()), "workspace");
  // FP64 operand rows: none on the emulated path with factored operands and
  // factored H, where each half is formed and sliced in one pass
  if (!(tc_ops && !alg3)) CK(h, h->d_Z.ensure((size_t)h->rows * h->k_alloc * 16), "operand workspace");
  CK(h, h->d_rexp.ensure((size_t)h->rows * 4), "workspace");
  if (h->tiles_rows_key != h->rows) {
    std::vector<int> rp(h->rows);
    for (int q = 0; q < (int)probs.size(); ++q)
      for (int g = 0; g < probs[q].n_g; ++g) {
        rp[probs[q].row_base + g] = q;
        rp[probs[q].col_base + g] = q;
      }
    if (int rc_up = upload(h, h->d_rowprob, rp)) return rc_up;
  }
  // H to host memory: the H contraction in two launches split by columns, the
  // first part's columns copied while the second runs (not with the autotuner,
  // which times whole halves)
  bool h_host = false;
  for (int k = 0; k < nk; ++k) h_host = h_host || op.host[k] != nullptr;
  // autotuner: a shape seen before runs with its choice; a new one runs with
  // the size-based defaults and is tuned after the enqueue below
  const bool tune = h->opt.autotune && h->opt.precision == FLAPW_PREC_EMU;
  std::string shape;
  if (tune) {
    shape = shape_key(h, probs);
    Tuned t;
    if (h->tuned_shape != shape) {
      if (tuned_lookup(shape, &t)) {
        apply_tuned(h, t);
        h->tuned_shape = shape;
      } else {
        h->tile_cover = h->opt.tile_cover;
        h->tile_order = default_tile_order(h);
        h->pipe_choice = 0;
      }
    }
  }
  // (the call that tunes times whole halves: no split there)
  const bool h_split = h_host && !(tune && h->tuned_shape != shape);
  Half hH, hHb, hS;
  if (int rc = ensure_tiles(h, probs, nk, h->rows, &hH, &hS, 0, n_slots, h_split, &hHb)) return rc;
  hH.row0 = 0;
  hH.nrows = alg3 ? 2 * h->g_total : h->g_total;
  hS.row0 = s_row0;
  hS.nrows = h->g_total;
  if (int rc = ensure_slices(h)) return rc;
  if (factored && !h->prep_valid) {
    if (int rc = prepare_prep(h, user_st)) return rc;
  }

  // pinned inputs: a slot whose copies (enqueued two calls back) have run,
  // so that the call returns after enqueueing; a graph replays the copies
  // from slot 0, so that path waits for the previous call instead
  int slot = 0;
  if (h->opt.use_graph) {
    if (h->last_stream) CK(h, cudaStreamSynchronize(h->last_stream), "cudaStreamSynchronize");
    CK(h, cudaStreamSynchronize(h->aux_stream), "cudaStreamSynchronize");
  } else {
    slot = h->pin_slot;
    h->pin_slot ^= 1;
    if (h->pin_ev_used[slot]) CK(h, cudaEventSynchronize(h->pin_ev[slot]), "cudaEventSynchronize");
  }
  PinBuf& pin_in = h->pin_ring[slot];
  PinBuf& pin_probs = h->pin_probs_ring[slot];
  CK(h, pin_in.ensure(t_bytes + slot_bytes + u_bytes + cmb_ints * 4 + tsph_bytes + 256), "cudaMallocHost");
  CK(h, pin_probs.ensure(sizeof(Prob) * probs.size()), "cudaMallocHost");
  char* pin = static_cast<char*>(pin_in.p);
  std::memcpy(pin, T, t_bytes);
  std::memcpy(pin + t_bytes, atom_slot, slot_bytes);
  std::memcpy(pin + t_bytes + slot_bytes, U, u_bytes);
  int* pc = reinterpret_cast<int*>(pin + t_bytes + slot_bytes + u_bytes);
  std::memcpy(pc, combo_slot.data(), combo_slot.size() * 4);
  std::memcpy(pc + n_combo, combo_type.data(), combo_type.size() * 4);
  std::memcpy(pc + 2 * n_combo, combo_atoms.data(), combo_atoms.size() * 4);
  std::memcpy(pc + 2 * n_combo + combo_atoms.size(), combo_start.data(), combo_start.size() * 4);
  if (h_sph) {
    // the rest of T after its spherical part: t^AA_l, t^BB_l and t^BA_l come
    // off the diagonals of the blocks (t^AB_l = conj t^BA_l off T^AB)
    std::memcpy(pin + t_bytes + slot_bytes + u_bytes + cmb_ints * 4, h->tsph.data(), tsph_bytes);
    double* Tr = reinterpret_cast<double*>(pin);
    const int nl = h->n_L;
    for (int sl = 0; sl < n_slots; ++sl)
      for (int l = 0; l <= h->lmax; ++l) {
        const double* c = &h->tsph[((size_t)sl * (h->lmax + 1) + l) * 4];
        for (int L = l * l; L < (l + 1) * (l + 1); ++L) {
          double* blk = Tr + (size_t)sl * n * n * 2;
          blk[2 * ((size_t)L * n + L)] -= c[0];
          blk[2 * ((size_t)(nl + L) * n + nl + L)] -= c[1];
          blk[2 * ((size_t)(nl + L) * n + L)] -= c[2];
          blk[2 * ((size_t)(nl + L) * n + L) + 1] -= c[3];
          blk[2 * ((size_t)L * n + nl + L)] -= c[2];
          blk[2 * ((size_t)L * n + nl + L) + 1] += c[3];
        }
      }
    // a remainder that is exactly zero (on and below the diagonal) needs no contraction
    h_zero = true;
    for (int sl = 0; sl < n_slots && h_zero; ++sl)
      for (int r = 0; r < n && h_zero; ++r)
        for (int c = 0; c <= r; ++c) {
          const double* e = Tr + ((size_t)sl * n * n + (size_t)r * n + c) * 2;
          if (e[0] != 0.0 || e[1] != 0.0) {
            h_zero = false;
            break;
          }
        }
  }
  h->last_h_zero = h_zero;
  std::memcpy(pin_probs.p, probs.data(), sizeof(Prob) * probs.size());
  h->last_n_slots = n_slots;
  h->last_alg3 = alg3;
  h->last_alg1 = alg1;

  // ---- the enqueued sequence (graph-capturable) ----
  // S needs no factorisation: its operands, slices and contraction run on the
  // caller's stream while the T blocks are factorised on the auxiliary
  // stream; the H work joins both.
  auto enqueue = [&](cudaStream_t st) -> int {
    CK(h, cudaEventRecord(h->ev[0], st), "cudaEventRecord");
    CK(h, cudaMemcpyAsync(h->d_T.p, pin, t_bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    CK(h, cudaMemcpyAsync(h->d_slot.p, pin + t_bytes, slot_bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    CK(h, cudaMemcpyAsync(h->d_slot.as<char>() + slot_bytes, pc, cmb_ints * 4, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    CK(h, cudaMemcpyAsync(h->d_U.p, pin + t_bytes + slot_bytes, u_bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    if (h_sph)
      CK(h, cudaMemcpyAsync(h->d_tsph.p, pin + t_bytes + slot_bytes + u_bytes + cmb_ints * 4, tsph_bytes,
                            cudaMemcpyHostToDevice, st),
         "cudaMemcpyAsync");
    CK(h, cudaMemcpyAsync(h->d_probs.p, pin_probs.p, sizeof(Prob) * probs.size(), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    if (!h->opt.use_graph) {
      CK(h, cudaEventRecord(h->pin_ev[slot], st), "cudaEventRecord");
      h->pin_ev_used[slot] = true;
    }
    if (stage_ab) {
      CK(h, cudaMemcpyAsync(h->d_stageA.p, A, ab_total * 16, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
      CK(h, cudaMemcpyAsync(h->d_stageB.p, B, ab_total * 16, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    }
    int* cnt = h->d_cnt.as<int>();  // [0] 2x2 pivots, [2] error flag, [8..] npos, nneg
    CK(h, cudaMemsetAsync(cnt, 0, sizeof(int) * 8, st), "cudaMemsetAsync");
    // tiles split over parts: host-memory outputs get zeros where other parts' blocks are
    if (h->part_filter.stride > 1)
      for (int i = 0; i < 2 * nk; ++i)
        if (op.host[i]) CK(h, cudaMemsetAsync(op.dev[i], 0, op.bytes[i], st), "cudaMemsetAsync");
    int* npos = cnt + 8;
    int* nneg = cnt + 8 + n_slots;
    int* pos_off = h->d_off.as<int>();
    int* neg_off = pos_off + h->n_atoms;
    int* kpk = neg_off + h->n_atoms;
    int* perm = h->d_fac.as<int>();
    int* outrow = perm + (size_t)n_slots * n;
    OpformArgs oa{};
    oa.n_atoms = h->n_atoms;
    oa.n_L = h->n_L;
    oa.n = n;
    oa.n_k = nk;
    oa.atom_slot = h->d_slot.as<int>();
    oa.atom_type = h->d_type.as<int>();
    oa.CH = h->d_CH.as<double2>();
    oa.perm = perm;
    oa.outrow = outrow;
    oa.npos = npos;
    oa.nneg = nneg;
    oa.pos_off = pos_off;
    oa.neg_off = neg_off;
    oa.kpk = kpk;
    oa.U = h->d_U.as<double>();
    oa.lmax = h->lmax;
    oa.k_alloc = h->k_alloc;
    oa.Z = h->d_Z.as<double2>();
    oa.gtiles = h->d_gt64.as<int>();
    oa.n_gtiles = (int)(h->gt64.size() / 2);
    oa.goff = h->d_goff.as<int64_t>();
    oa.g_total = h->g_total;
    oa.h_row0 = 0;
    oa.s_row0 = s_row0;
    oa.r_row0 = h->g_total;
    oa.T = h->d_T.as<double2>();
    oa.M = h->d_CH.as<double2>();
    oa.hpd = alg1 ? h->d_hpd.as<int>() : nullptr;
    oa.A = dA;
    oa.B = dB;
    oa.Yc = h->d_Yc.as<double2>();
    oa.al = h->d_al.as<double>();
    oa.bl = h->d_bl.as<double>();
    oa.ph = h->d_ph.as<double2>();
    oa.n_types = h->n_types;
    const int* dc = reinterpret_cast<const int*>(h->d_slot.as<char>() + slot_bytes);
    oa.combo_slot = dc;
    oa.combo_type = dc + n_combo;
    oa.combo_atoms = dc + 2 * n_combo;
    oa.combo_start = dc + 2 * n_combo + combo_atoms.size();
    oa.n_combo = n_combo;
    // fork: factorisation on the auxiliary stream
    CK(h, cudaEventRecord(h->ev[13], st), "cudaEventRecord");
    CK(h, cudaStreamWaitEvent(h->aux_stream, h->ev[13], 0), "cudaStreamWaitEvent");
    int* oprexp_a = h->d_oprexp.as<int>();
    int* oprexp_b = oprexp_a + op_rows_a;
    if (!alg3 && !h_zero) {
      // beside the S contraction one CTA per slot; with S by the addition
      // theorem the factorisation leads the critical path: a cluster per slot
      CK(h, launch_tfactor(h->d_T.as<double2>(), n, n_slots, h->d_work.as<double2>(), h->d_CH.as<double2>(),
                           perm, outrow, npos, nneg, cnt, cnt + 2, s_legendre, h->aux_stream),
         "T factorisation launch");
      CK(h, launch_layout(npos, nneg, h->d_slot.as<int>(), h->n_atoms, nk, pos_off, neg_off, kpk,
                          h->d_probs.as<Prob>(), (int)K, h->aux_stream),
         "layout launch");
    }
    if (alg3) {
      // the operand matrix of Alg. 3, or of Alg. 1 with the Cholesky factors of T^AA
      CK(h, launch_alg_m(h->d_T.as<double2>(), n, h->n_L, n_slots, alg1, h->d_CH.as<double2>(),
                         h->d_work.as<double2>(), h->d_hpd.as<int>(), h->aux_stream),
         "operand matrix launch");
    }
    CK(h, cudaEventRecord(h->ev[1], h->aux_stream), "cudaEventRecord");
    if (tc_ops && alg3) {
      CK(h, launch_opgemm_build_alg3(h->d_CH.as<double2>(), n_slots, n, h->n_L, op_kp, h->d_opA.as<double2>(),
                                     h->aux_stream),
         "operand factor launch");
    } else if (tc_ops && !h_zero) {
      CK(h, launch_opgemm_build(h->d_CH.as<double2>(), perm, n_slots, n, op_kp, nullptr, nullptr, nullptr,
                                h->n_L, h->lmax, h->n_types, h->g_total, h->d_opA.as<double2>(), nullptr,
                                h->aux_stream, true),
         "operand factor launch");
    }
    if (tc_ops && !h_zero) {
      CK(h, launch_slicer_rows(h->d_opA.as<double2>(), op_kp, op_rows_a, kOpSlices, h->d_opSLA.as<__half>(),
                               oprexp_a, h->aux_stream),
         "operand factor slicer launch");
    }
    CK(h, cudaEventRecord(h->ev[16], h->aux_stream), "cudaEventRecord");
    // S on the caller's stream, beside the factorisation (which holds n_slots SMs)
    CK(h, cudaEventRecord(h->ev[9], st), "cudaEventRecord");
    if (tc_ops) {
      // the W factor of the H operands needs no factorisation: formed and sliced
      // here, it is done before the S contraction claims the SMs
      CK(h, launch_opgemm_build(nullptr, nullptr, 0, n, op_kp, h->d_Yc.as<double2>(), h->d_al.as<double>(),
                                h->d_bl.as<double>(), h->n_L, h->lmax, h->n_types, h->g_total, nullptr,
                                h->d_opB.as<double2>(), st, false),
         "operand factor launch");
      CK(h, launch_slicer_rows(h->d_opB.as<double2>(), op_kp, op_rows_b, kOpSlices, h->d_opSLB.as<__half>(),
                               oprexp_b, st),
         "operand factor slicer launch");
    }
    if (s_legendre) {
      // S by the addition theorem: no S operands, slices or contraction
      CK(h, cudaEventRecord(h->ev[2], st), "cudaEventRecord");
      CK(h, cudaEventRecord(h->ev[3], st), "cudaEventRecord");
      SLegArgs la{};
      la.probs = h->d_probs.as<Prob>();
      la.s_row0 = s_row0;
      la.g_total = h->g_total;
      la.lmax = h->lmax;
      la.n_types = h->n_types;
      la.khat = h->d_khat.as<double>();
      la.al = h->d_al.as<double>();
      la.bl = h->d_bl.as<double>();
      la.U = h->d_U.as<double>();
      la.ph = h->d_ph.as<double2>();
      la.type_atoms = h->d_typeatoms.as<int>();
      la.type_start = h->d_typeatoms.as<int>() + h->n_atoms;
      la.scale = 4.0 * M_PI / h->volume;
      la.n_atoms = h->n_atoms;
      la.dfw = (h->opt.precision == FLAPW_PREC_EMU) ? h->d_sdf.as<float2>() : nullptr;
      CK(h, launch_slegendre(la, h->d_f64_tiles.as<F64Tile>() + hS.f64_t0, hS.f64_nt, st),
         "S (addition theorem) launch");
      CK(h, cudaEventRecord(h->ev[4], st), "cudaEventRecord");
    } else if (tc_ops) {
      // S rows formed from W and sliced in one pass: no FP64 S operand
      CK(h, cudaEventRecord(h->ev[2], st), "cudaEventRecord");
      SopArgs sa{};
      sa.n = n;
      sa.n_L = h->n_L;
      sa.lmax = h->lmax;
      sa.n_atoms = h->n_atoms;
      sa.G = h->g_total;
      sa.W = h->d_opB.as<double2>();
      sa.kpw = op_kp;
      sa.U = h->d_U.as<double>();
      sa.ph = h->d_ph.as<double2>();
      sa.combo_type = oa.combo_type;
      sa.combo_atoms = oa.combo_atoms;
      sa.combo_start = oa.combo_start;
      sa.n_combo = n_combo;
      sa.s_row0 = s_row0;
      sa.k_alloc = h->k_alloc;
      CK(h, launch_sop_slice(sa, slices_of(h), h->d_SL.as<__half>(), h->rows, h->d_rexp.as<int>(), st),
         "S operand slice launch");
      if (int rc = enqueue_contraction(h, hS, n_slots, st, 3, 4, true)) return rc;
    } else {
      CK(h, launch_opform_S(oa, factored, st), "S operand launch");
      CK(h, cudaEventRecord(h->ev[2], st), "cudaEventRecord");
      if (int rc = enqueue_contraction(h, hS, n_slots, st, 3, 4)) return rc;
    }
    // join, then H
    CK(h, cudaStreamWaitEvent(st, h->ev[16], 0), "cudaStreamWaitEvent");
    CK(h, cudaEventRecord(h->ev[8], st), "cudaEventRecord");
    HLegArgs hl{};
    if (h_sph) {
      hl.probs = h->d_probs.as<Prob>();
      hl.h_row0 = 0;
      hl.g_total = h->g_total;
      hl.lmax = h->lmax;
      hl.khat = h->d_khat.as<double>();
      hl.al = h->d_al.as<double>();
      hl.bl = h->d_bl.as<double>();
      hl.ph = h->d_ph.as<double2>();
      hl.tsph = h->d_tsph.as<double>();
      hl.combo_slot = oa.combo_slot;
      hl.combo_type = oa.combo_type;
      hl.combo_atoms = oa.combo_atoms;
      hl.combo_start = oa.combo_start;
      hl.n_combo = n_combo;
      hl.scale = 4.0 * M_PI / h->volume;
      hl.n_atoms = h->n_atoms;
      hl.n_types = h->n_types;
      hl.dfw = (h->opt.precision == FLAPW_PREC_EMU) ? h->d_hdf.as<float2>() : nullptr;
    }
    if (h_zero) {
      // T is its spherical part: no factorisation, operands or contraction for H
      // (with H in host memory in two launches split by column, as the contraction)
      CK(h, cudaEventRecord(h->ev[10], st), "cudaEventRecord");
      CK(h, cudaEventRecord(h->ev[11], st), "cudaEventRecord");
      CK(h, launch_hlegendre(hl, h->d_f64_tiles.as<F64Tile>() + hH.f64_t0, hH.f64_nt, false, st),
         "H (addition theorem) launch");
      if (h_split) {
        CK(h, cudaEventRecord(h->ev[18], st), "cudaEventRecord");
        CK(h, launch_hlegendre(hl, h->d_f64_tiles.as<F64Tile>() + hHb.f64_t0, hHb.f64_nt, false, st, hH.f64_nt > 0),
           "H (addition theorem) launch");
      }
      CK(h, cudaEventRecord(h->ev[12], st), "cudaEventRecord");
    } else if (tc_ops) {
      OpGemmArgs ga{};
      ga.n = n;
      ga.kchunks = op_kp / kChunk;
      ga.G = h->g_total;
      ga.combo_slot = oa.combo_slot;
      ga.combo_type = oa.combo_type;
      ga.combo_atoms = oa.combo_atoms;
      ga.combo_start = oa.combo_start;
      ga.outrow = outrow;
      ga.npos = npos;
      ga.nneg = nneg;
      ga.pos_off = pos_off;
      ga.neg_off = neg_off;
      ga.kpk = kpk;
      ga.rexp_a = oprexp_a;
      ga.rexp_b = oprexp_b;
      ga.ph = h->d_ph.as<double2>();
      ga.P = h->d_opP.as<longlong2>();
      ga.Z = h->d_Z.as<double2>();
      ga.k_alloc = h->k_alloc;
      ga.h_row0 = 0;
      ga.alg3_nl = alg3 ? h->n_L : 0;
      ga.hpd = alg1 ? h->d_hpd.as<int>() : nullptr;
      ga.r_row0 = h->g_total;
      CK(h, launch_opgemm(h->opmap_a, h->opmap_b, ga, h->d_optiles.as<OpTile>(), (int)h->optiles.size(),
                          cnt + 2, h->num_sms, wait_ns(h), st),
         "H operand launch");
      if (alg3) {
        CK(h, launch_opgemm_phase(ga, n_combo, st), "H operand phase launch");
        CK(h, launch_opform_alg3(oa, factored, false, st), "H operand (Alg. 3) copy launch");
      } else {
        // the atom phases applied and the rows sliced in one pass: no FP64 H operand
        CK(h, cudaEventRecord(h->ev[10], st), "cudaEventRecord");
        CK(h, launch_opgemm_slice(ga, n_combo, slices_of(h), h->d_SL.as<__half>(), h->rows,
                                  h->d_rexp.as<int>(), st),
           "H operand slice launch");
      }
    } else if (alg3) {
      CK(h, launch_opform_alg3(oa, factored, true, st), "H operand (Alg. 3) launch");
    } else {
      CK(h, launch_opform_H(oa, factored, st), "H operand launch");
    }
    if (!h_zero) {
      const bool h_presliced = tc_ops && !alg3;
      if (!h_presliced) CK(h, cudaEventRecord(h->ev[10], st), "cudaEventRecord");
      // with FLAPW_H_SPHERICAL the spherical part of T by the addition theorem is
      // added to each part's columns after the contraction of the rest
      const int ev_first = h_split ? 18 : 12;
      if (int rc = enqueue_contraction(h, hH, 0, st, 11, ev_first, h_presliced)) return rc;
      if (h_sph) {
        CK(h, launch_hlegendre(hl, h->d_f64_tiles.as<F64Tile>() + hH.f64_t0, hH.f64_nt, true, st),
           "H (addition theorem) launch");
        CK(h, cudaEventRecord(h->ev[ev_first], st), "cudaEventRecord");
      }
      if (h_split) {
        if (int rc = enqueue_contraction(h, hHb, 0, st, -1, 12, true)) return rc;
        if (h_sph) {
          CK(h, launch_hlegendre(hl, h->d_f64_tiles.as<F64Tile>() + hHb.f64_t0, hHb.f64_nt, true, st, hH.f64_nt > 0),
             "H (addition theorem) launch");
          CK(h, cudaEventRecord(h->ev[12], st), "cudaEventRecord");
        }
      }
    }
    // Host-memory outputs go back on the copy stream: S beside the H work; with
    // the split H contraction, columns [0, c1) of H while its second part runs,
    // the rest after it.  Every copy is enqueued after all the compute, so that
    // a long copy queue (many k-points) cannot hold the host back from
    // enqueueing the H work; each waits for the contraction that writes it.
    bool s_host = false;
    int n_host = 0, copy_ops = 0;
    int64_t copy_bytes = 0;
    for (int i = 0; i < 2 * nk; ++i) n_host += op.host[i] != nullptr;
    for (int i = nk; i < 2 * nk; ++i) s_host = s_host || op.host[i] != nullptr;
    auto ng_of = [&](int k) -> int64_t { return h->goff[k + 1] - h->goff[k]; };
    auto copy = [&](int i, int k, int64_t c0, int64_t c1) -> cudaError_t {
      return copy_out(op.host[i], op.dev[i], ng_of(k), layout, c0, c1, copy_block_cols(ng_of(k), n_host),
                      h->copy_stream, &copy_ops, &copy_bytes);
    };
    if (s_host) {
      CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev[4], 0), "cudaStreamWaitEvent");
      for (int i = nk; i < 2 * nk; ++i)
        if (op.host[i]) CK(h, copy(i, i - nk, 0, ng_of(i - nk)), "cudaMemcpy2DAsync");
    }
    auto h_c1 = [&](int k) -> int64_t {
      return h_split ? std::min<int64_t>(ng_of(k), 64 * (int64_t)h_split_block((int)ng_of(k))) : 0;
    };
    if (h_split) {
      CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev[18], 0), "cudaStreamWaitEvent");
      for (int k = 0; k < nk; ++k)
        if (op.host[k]) CK(h, copy(k, k, 0, h_c1(k)), "cudaMemcpy2DAsync");
    }
    if (h_host) CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev[12], 0), "cudaStreamWaitEvent");
    for (int k = 0; k < nk; ++k)
      if (op.host[k]) CK(h, copy(k, k, h_c1(k), ng_of(k)), "cudaMemcpy2DAsync");
    h->stats.copy_ops = copy_ops;
    h->stats.bytes_d2h = copy_bytes;
    if (s_host || h_host) {
      CK(h, cudaEventRecord(h->ev_copy, h->copy_stream), "cudaEventRecord");
      CK(h, cudaStreamWaitEvent(st, h->ev_copy, 0), "cudaStreamWaitEvent");
    }
    CK(h, cudaEventRecord(h->ev[5], st), "cudaEventRecord");
    return FLAPW_OK;
  };

  h->ev_recorded = true;
  h->ev_engine = false;
  h->last_stream = user_st;
  if (!h->opt.use_graph) {
    if (int rc = enqueue(user_st)) return rc;
    if (tune && h->tuned_shape != shape) return autotune_tiles(h, probs, nk, h->rows, n_slots, shape, user_st);
    return FLAPW_OK;
  }

  // graph replay, keyed on everything the captured sequence bakes in
  std::vector<uintptr_t> key{(uintptr_t)A, (uintptr_t)B, (uintptr_t)n_slots, (uintptr_t)h->opt.precision,
                             (uintptr_t)h_zero, (uintptr_t)h->d_tsph.p,
                             (uintptr_t)h->opt.s_method, (uintptr_t)h->opt.h_method,
                             (uintptr_t)layout, (uintptr_t)h->opt.operands, (uintptr_t)slices_of(h),
                             (uintptr_t)h->d_Z.p, (uintptr_t)h->d_SL.p, (uintptr_t)h->pin_ring[0].p,
                             (uintptr_t)h->d_T.p, (uintptr_t)h->d_stageOut.p, (uintptr_t)h->d_emu_tiles.p,
                             (uintptr_t)h->d_opA.p, (uintptr_t)h->d_opB.p, (uintptr_t)h->d_opSLA.p,
                             (uintptr_t)h->d_opSLB.p, (uintptr_t)h->d_oprexp.p, (uintptr_t)h->d_optiles.p,
                             (uintptr_t)h->d_opP.p, (uintptr_t)h->d_split.p, (uintptr_t)h->d_sdf.p,
                             (uintptr_t)h->d_hdf.p};
  for (int k = 0; k < nk; ++k) {
    key.push_back((uintptr_t)H[k]);
    key.push_back((uintptr_t)S[k]);
  }
  if (!h->gexec || key != h->gkey) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    const int rc = enqueue(h->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    CK(h, e2, "cudaStreamEndCapture");
    const cudaError_t e3 = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    CK(h, e3, "cudaGraphInstantiate");
    h->gkey = key;
  } else {
    ++h->stats.graph_replays;
  }
  CK(h, cudaGraphLaunch(h->gexec, user_st), "cudaGraphLaunch");
  return FLAPW_OK;
}

int flapw_herk(flapw_handle h, const void* Z, int64_t ldz, int K, int N, const int* sigma,
               void* H, int64_t ldh, void* stream) {
  (void)cudaGetLastError();  // a stale error of unrelated code must not fail our launch checks
  if (!h || !Z || !H) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  BudgetScope budget_scope(h);
  if (K < 1 || N < 1 || ldz < K) return fail(h, FLAPW_ERR_ARG, "need K >= 1, N >= 1, ldz >= K");
  if (K >= (1 << 17)) return fail(h, FLAPW_ERR_UNSUPPORTED, "K must be below 131072");
  if (h->opt.layout == FLAPW_LAYOUT_LOWER_FULL && ldh < N) return fail(h, FLAPW_ERR_ARG, "ldh < N");
  if (!is_device_ptr(Z)) return fail(h, FLAPW_ERR_ARG, "Z must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int> pos, neg;
  for (int k = 0; k < K; ++k) {
    const int sg = sigma ? sigma[k] : 1;
    if (sg != 1 && sg != -1) return fail(h, FLAPW_ERR_ARG, "sigma entries must be +1 or -1");
    (sg > 0 ? pos : neg).push_back(k);
  }
  const int64_t kp_pad = neg_base((int)pos.size());
  const int64_t k_alloc = std::max<int64_t>((int64_t)k_chunks((int)pos.size(), (int)neg.size()) * kChunk, kChunk);
  std::vector<int> kmap(k_alloc, -1);
  for (size_t i = 0; i < pos.size(); ++i) kmap[i] = pos[i];
  for (size_t i = 0; i < neg.size(); ++i) kmap[kp_pad + i] = neg[i];
  const bool devH = is_device_ptr(H);
  const size_t ob = out_bytes(h->opt.layout, N);
  double2* dH = static_cast<double2*>(H);
  if (!devH) {
    CK(h, h->d_stageOut.ensure(ob), "staging");
    dH = h->d_stageOut.as<double2>();
  }
  if (h->last_stream) CK(h, cudaStreamSynchronize(h->last_stream), "cudaStreamSynchronize");
  std::vector<Prob> probs{Prob{0, N, (int)pos.size(), (int)neg.size(), h->opt.layout, /*col_base*/ 0,
                               h->opt.layout == FLAPW_LAYOUT_LOWER_FULL ? ldh : N, dH}};
  h->rows = N;
  h->k_alloc = k_alloc;
  h->k_terms = K;
  h->deep_pipe = herk_emu_deep(N);
  h->max_ng = N;
  set_tile_order(h);
  h->part_filter = PartFilter{};  // the contraction step alone is never split
  h->part_key.clear();
  if (int rc_up = upload(h, h->d_kmap, kmap) || upload(h, h->d_probs, probs)) return rc_up;
  std::vector<int> rp(N, 0);
  if (int rc_up = upload(h, h->d_rowprob, rp)) return rc_up;
  Half hf, none;
  h->tiles_rows_key = -1;
  if (int rc = ensure_tiles(h, probs, 1, -2 - (int64_t)N, &hf, &none)) return rc;
  h->tiles_rows_key = -1;  // a later build_HS rebuilds its own lists
  hf.row0 = 0;
  hf.nrows = N;
  CK(h, h->d_Z.ensure((size_t)N * k_alloc * 16), "operand workspace");
  CK(h, h->d_rexp.ensure((size_t)N * 4), "workspace");
  CK(h, h->d_cnt.ensure(sizeof(int) * 16), "workspace");
  if (int rc = ensure_slices(h)) return rc;
  CK(h, cudaMemsetAsync(h->d_cnt.p, 0, sizeof(int) * 8, st), "cudaMemsetAsync");
  CK(h, cudaEventRecord(h->ev[0], st), "cudaEventRecord");
  CK(h, launch_gather_Z(static_cast<const double2*>(Z), ldz, K, N, h->d_kmap.as<int>(), k_alloc,
                        h->d_Z.as<double2>(), st),
     "gather launch");
  CK(h, cudaEventRecord(h->ev[2], st), "cudaEventRecord");
  if (int rc = enqueue_contraction(h, hf, 0, st, 3, 4)) return rc;
  if (!devH) CK(h, cudaMemcpyAsync(H, dH, ob, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  h->stats.copy_ops = devH ? 0 : 1;
  h->stats.bytes_d2h = devH ? 0 : (int64_t)ob;
  CK(h, cudaEventRecord(h->ev[5], st), "cudaEventRecord");
  h->ev_recorded = true;
  h->ev_engine = true;
  h->last_stream = st;
  h->gkey.clear();
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return FLAPW_OK;
}

int flapw_sync(flapw_handle h) {
  if (!h) return fail(h, FLAPW_ERR_ARG, "NULL handle");
  CK(h, cudaStreamSynchronize(h->last_stream), "cudaStreamSynchronize");
  CK(h, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if (h->d_cnt.p) {
    int c[8];
    CK(h, cudaMemcpy(c, h->d_cnt.p, sizeof(c), cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (c[2] == FLAPW_ERR_TIMEOUT)
      return fail(h, FLAPW_ERR_TIMEOUT, "a bounded device wait expired in the contraction");
    if (c[2] == FLAPW_ERR_FACTOR)
      return fail(h, FLAPW_ERR_FACTOR, "a T block has a singular 2x2 pivot");
    if (c[2] != 0) return fail(h, FLAPW_ERR_CUDA, "device error flag " + std::to_string(c[2]));
  }
  return FLAPW_OK;
}

int flapw_get_stats(flapw_handle h, flapw_stats* st) {
  if (!h || !st) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  auto el = [&](int a, int b) -> double {
    float ms = 0.f;
    if (cudaEventQuery(h->ev[b]) != cudaSuccess) {
      (void)cudaGetLastError();
      return -1.0;
    }
    if (cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) != cudaSuccess) {
      (void)cudaGetLastError();
      return -1.0;
    }
    return ms;
  };
  flapw_stats s = h->stats;
  if (h->ev_ab) {
    s.ms_ab = el(6, 7);
    s.ms_ab_assemble = el(17, 7);
  }
  if (h->ev_recorded && h->ev_engine) {
    s.ms_factor = 0.0;
    s.ms_operands = el(0, 2);
    s.ms_slice = (h->opt.precision == FLAPW_PREC_EMU) ? el(2, 3) : 0.0;
    s.ms_contract = el(3, 4);
    s.ms_hs_total = el(0, 5);
  } else if (h->ev_recorded) {
    s.ms_factor = el(0, 1);
    s.ms_operands = el(9, 2) + el(8, 10);
    s.ms_slice = (h->opt.precision == FLAPW_PREC_EMU) ? el(2, 3) + el(10, 11) : 0.0;
    s.ms_contract = el(3, 4) + el(11, 12);
    s.ms_s = el(3, 4);
    s.ms_hs_total = el(0, 5);
  }
  s.n_slices = slices_of(h);
  s.n_tiles = (h->opt.precision == FLAPW_PREC_EMU) ? h->n_emu_tiles : h->n_f64_tiles;
  s.tile_order = h->tiles_order;
  {
    int64_t max_ng = 0;
    for (int k = 0; k < h->n_k; ++k) max_ng = std::max<int64_t>(max_ng, h->goff[k + 1] - h->goff[k]);
    if (h->engine_only) max_ng = h->rows;
    s.tile_cover = h->tiles_cover >= 0 ? h->tiles_cover : cover::cover_for(h->tile_cover, max_ng);
    s.pipeline = use_deep_pipe(h) ? 2 : 1;
  }
  if (!h->engine_only) {
    s.k_total = (int64_t)h->n_atoms * (h->last_alg3 ? 3 : 2) * h->n_L;
    double ng2 = 0;
    for (int k = 0; k < h->n_k; ++k) {
      const double ng = (double)(h->goff[k + 1] - h->goff[k]);
      ng2 += ng * ng;
    }
    s.flops_herk = 16.0 * h->n_atoms * h->n_L * ng2;
  }
  const bool done = h->ev_recorded && cudaEventQuery(h->ev[5]) == cudaSuccess;
  (void)cudaGetLastError();
  if (h->d_cnt.p && h->d_off.p && done && !h->engine_only) {
    int c[8];
    int kpk[3] = {0, 0, 0};
    if (cudaMemcpy(c, h->d_cnt.p, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemcpy(kpk, h->d_off.as<int>() + 2 * h->n_atoms, sizeof(kpk), cudaMemcpyDeviceToHost) == cudaSuccess) {
      if (h->last_alg3) {  // no factorisation: every H row has sigma = +1
        kpk[1] = (int)s.k_total;
        kpk[2] = 0;
        c[0] = 0;
      }
      if (h->last_alg1 && h->last_n_slots > 0) {
        std::vector<int> hpd(h->last_n_slots, 0);
        if (cudaMemcpy(hpd.data(), h->d_hpd.p, sizeof(int) * hpd.size(), cudaMemcpyDeviceToHost) == cudaSuccess)
          for (int v : hpd) s.n_chol += v;
      }
      if (h->last_h_zero) {  // T was its spherical part: no H contraction
        kpk[1] = kpk[2] = 0;
        c[0] = 0;
      }
      s.n_pivot2 = c[0];
      s.n_pos = kpk[1];
      s.n_neg = kpk[2];
      // tensor flops executed: per tile, slice pair and 16-wide K step of
      // the 64-wide chunks (the sigma = -1 block from the next multiple of 16
      // after the sigma = +1 one, the end padded to a whole chunk), an R and an
      // I pass of M = 256, N = 128, K = 16 MMAs
      const int S_ = slices_of(h);
      const double pairs = S_ * (S_ + 1) / 2.0;
      const double ksH = 4.0 * k_chunks(kpk[1], kpk[2]);
      const double ksS = (h->opt.s_method == FLAPW_S_LEGENDRE)
                             ? 0.0
                             : 4.0 * std::ceil((double)h->n_atoms * 2 * h->n_L / 64.0);
      double tf = 0;
      const int nk = h->n_k;
      if ((int)h->emu_tiles_per_prob.size() == 2 * nk)
        for (int k = 0; k < nk; ++k)
          tf += pairs * 2.0 * (2.0 * 256 * 128 * 16) *
                (h->emu_tiles_per_prob[k] * ksH + h->emu_tiles_per_prob[nk + k] * ksS);
      s.flops_tensor = tf;
    } else {
      (void)cudaGetLastError();
    }
  }
  *st = s;
  return FLAPW_OK;
}

int flapw_get_factor(flapw_handle h, int slot, double* CH, int* n_pos, int* n_neg) {
  if (!h || !CH || !n_pos || !n_neg) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  if (slot < 0 || slot >= h->last_n_slots) return fail(h, FLAPW_ERR_ARG, "slot out of range");
  if (h->last_alg3) return fail(h, FLAPW_ERR_STATE, "the last build_HS used FLAPW_H_ALG3: no factorisation");
  const int n = 2 * h->n_L;
  CK(h, cudaStreamSynchronize(h->last_stream), "cudaStreamSynchronize");
  CK(h, cudaStreamSynchronize(h->aux_stream), "cudaStreamSynchronize");
  std::vector<double2> M((size_t)n * n);
  std::vector<int> perm(n), outrow(n);
  CK(h, cudaMemcpy(M.data(), h->d_CH.as<double2>() + (size_t)slot * n * n, (size_t)n * n * 16, cudaMemcpyDeviceToHost), "cudaMemcpy");
  const int* fac = h->d_fac.as<int>();
  CK(h, cudaMemcpy(perm.data(), fac + (size_t)slot * n, n * 4, cudaMemcpyDeviceToHost), "cudaMemcpy");
  CK(h, cudaMemcpy(outrow.data(), fac + (size_t)h->last_n_slots * n + (size_t)slot * n, n * 4, cudaMemcpyDeviceToHost), "cudaMemcpy");
  int* cnt = h->d_cnt.as<int>();
  CK(h, cudaMemcpy(n_pos, cnt + 8 + slot, 4, cudaMemcpyDeviceToHost), "cudaMemcpy");
  CK(h, cudaMemcpy(n_neg, cnt + 8 + h->last_n_slots + slot, 4, cudaMemcpyDeviceToHost), "cudaMemcpy");
  // C^H = M P^T, rows moved to their sigma-grouped places
  std::memset(CH, 0, sizeof(double) * 2 * (size_t)n * n);
  for (int r = 0; r < n; ++r) {
    if (outrow[r] < 0) continue;
    for (int i = 0; i < n; ++i) {
      const size_t o = ((size_t)outrow[r] * n + perm[i]) * 2;
      CH[o] = M[(size_t)r * n + i].x;
      CH[o + 1] = M[(size_t)r * n + i].y;
    }
  }
  return FLAPW_OK;
}

int flapw_eigh(flapw_handle h, int n, void* H, int64_t ldh, void* S, int64_t lds, double* w, int vectors,
               void* stream) {
  (void)cudaGetLastError();
  if (!h || !H || !S || !w) return fail(h, FLAPW_ERR_ARG, "NULL argument");
  if (n < 1 || ldh < n || lds < n) return fail(h, FLAPW_ERR_ARG, "need n >= 1, ldh >= n, lds >= n");
  if (!is_device_ptr(H) || !is_device_ptr(S)) return fail(h, FLAPW_ERR_ARG, "H and S must be device memory");
  if (ldh > INT32_MAX || lds > INT32_MAX) return fail(h, FLAPW_ERR_UNSUPPORTED, "ldh and lds must fit in int");
  BudgetScope budget_scope(h);
  Solver& sv = solver_lib();
  if (!sv.ok) return fail(h, FLAPW_ERR_UNSUPPORTED, sv.why.c_str());
  if (!h->solver) {
    cusolverDnHandle_t sh = nullptr;
    if (sv.create(&sh) != CUSOLVER_STATUS_SUCCESS) return fail(h, FLAPW_ERR_CUDA, "cusolverDnCreate failed");
    h->solver = sh;
  }
  cusolverDnHandle_t sh = static_cast<cusolverDnHandle_t>(h->solver);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sv.set_stream(sh, st) != CUSOLVER_STATUS_SUCCESS) return fail(h, FLAPW_ERR_CUDA, "cusolverDnSetStream failed");
  const cusolverEigMode_t jobz = vectors ? CUSOLVER_EIG_MODE_VECTOR : CUSOLVER_EIG_MODE_NOVECTOR;
  cuDoubleComplex* A = static_cast<cuDoubleComplex*>(H);
  cuDoubleComplex* B = static_cast<cuDoubleComplex*>(S);
  CK(h, h->d_eig_w.ensure((size_t)n * 8 + 16), "eigensolver workspace");
  double* dw = h->d_eig_w.as<double>();
  int* dinfo = reinterpret_cast<int*>(dw + n);
  int lwork = 0;
  if (sv.zhegvd_buffer(sh, CUSOLVER_EIG_TYPE_1, jobz, CUBLAS_FILL_MODE_LOWER, n, A, (int)ldh, B, (int)lds, dw,
                       &lwork) != CUSOLVER_STATUS_SUCCESS)
    return fail(h, FLAPW_ERR_CUDA, "cusolverDnZhegvd_bufferSize failed");
  CK(h, h->d_eig_work.ensure((size_t)std::max(lwork, 1) * sizeof(cuDoubleComplex)), "eigensolver workspace");
  if (sv.zhegvd(sh, CUSOLVER_EIG_TYPE_1, jobz, CUBLAS_FILL_MODE_LOWER, n, A, (int)ldh, B, (int)lds, dw,
                h->d_eig_work.as<cuDoubleComplex>(), lwork, dinfo) != CUSOLVER_STATUS_SUCCESS)
    return fail(h, FLAPW_ERR_CUDA, "cusolverDnZhegvd failed");
  int info = 0;
  CK(h, cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  CK(h, cudaMemcpyAsync(w, dw, (size_t)n * 8, is_device_ptr(w) ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault, st),
     "cudaMemcpyAsync");
  CK(h, cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (info > n) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "S is not positive definite (its leading minor of order %d): the muffin-tin S alone is "
                  "singular when 2 N_A N_L < N_G", info - n);
    return fail(h, FLAPW_ERR_FACTOR, msg);
  }
  if (info > 0) return fail(h, FLAPW_ERR_FACTOR, "the Hermitian eigensolver did not converge");
  if (info < 0) return fail(h, FLAPW_ERR_ARG, "the eigensolver rejected an argument");
  return FLAPW_OK;
}

const char* flapw_last_error(flapw_handle h) {
  return h ? h->err.c_str() : g_last_error.c_str();
}

int flapw_destroy(flapw_handle h) {
  if (!h) return fail(nullptr, FLAPW_ERR_ARG, "NULL handle");
  cudaStreamSynchronize(h->last_stream);
  if (h->aux_stream) cudaStreamSynchronize(h->aux_stream);
  (void)cudaGetLastError();
  delete h;
  return FLAPW_OK;
}

}  // extern "C"
