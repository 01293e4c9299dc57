// flapw_herk_noalloc: the emulated lower-triangle contraction Z^H diag(sigma) Z
// for callers that must not allocate device memory.
//
// Every workspace the emulated contraction needs (the sigma-grouped copy of
// Z, its fp16 slices, per-row exponents, the tile list and the problem
// record) lives in one file-scope __device__ array of kScratchBytes.  The
// array is part of the library image: every GPU that loads the library
// holds it until the process exits.  Nothing here calls cudaMalloc,
// cudaFree or any allocating routine; the work is the existing gather,
// slicer and tcgen05 contraction kernels pointed at regions of the array.
// The host data a call needs (sigma, the problem record) travels in kernel
// arguments, so no copy reads the caller's host memory after the call returns.
//
// The array's name in host code is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, once per device, on the
// first call made with that device current.  That first call should come
// before any stream capture.  All calls share the array and it keeps the
// previous call's contents: what must start at zero is cleared on the stream,
// and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "flapw_internal.h"
#include "tiles.cuh"

namespace flapw {
namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// sigma as bits (bit k set: sigma_k = -1), passed by value in the setup
// kernel's arguments; K is below 2^17 as in the other contraction entry points.
constexpr int kMaxK = 1 << 17;
struct SigmaBits {
  uint32_t w[kMaxK / 32];
};

// One CTA of 256 threads writes, into the scratch array: the problem record;
// kmap[k'] = original row of operand column k' (sigma = +1 rows, then from
// kp_pad the sigma = -1 rows, -1 in the padding); and the tile list of the
// cyclic lower-triangle cover (tiles.cuh), strip by strip, toff[] holding each
// strip's first tile.
__global__ void __launch_bounds__(256)
    noalloc_setup_kernel(const __grid_constant__ SigmaBits sb, int K, int kp_pad, int k_alloc, Prob P,
                         Prob* prob, int* kmap, int ncb, int* toff, EmuTile* tiles) {
  __shared__ int scan[256];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *prob = P;
  for (int i = tid; i < k_alloc; i += nt) kmap[i] = -1;
  // each thread takes a run of sigma words: count its -1 rows, scan, place
  const int nw = (K + 31) / 32, per = (nw + nt - 1) / nt;
  const int w0 = min(nw, tid * per), w1 = min(nw, w0 + per);
  int negs = 0;
  for (int w = w0; w < w1; ++w) negs += __popc(sb.w[w]);
  scan[tid] = negs;
  __syncthreads();  // also orders the kmap padding before the placements
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < nt; ++t) {
      const int v = scan[t];
      scan[t] = acc;
      acc += v;
    }
    int off = 0;
    for (int a = 0; a < ncb;) {
      const int e = cover::seg_end(a, ncb, ncb);
      for (int j = a; j < e; ++j) {
        toff[j] = off;
        off += cover::strip_tiles(a, e, ncb, j);
      }
      a = e;
    }
    toff[ncb] = off;
  }
  __syncthreads();
  int q = scan[tid], p = w0 * 32 - q;
  for (int w = w0; w < w1; ++w)
    for (int b = 0; b < 32 && w * 32 + b < K; ++b) {
      const int k = w * 32 + b;
      if ((sb.w[w] >> b) & 1u) kmap[kp_pad + q++] = k;
      else kmap[p++] = k;
    }
  for (int j = tid; j < ncb; j += nt) {
    int a, e;
    cover::segment_of(ncb, ncb, j, a, e);
    const int n = cover::strip_tiles(a, e, ncb, j);
    for (int t = 0; t < n; ++t) {
      EmuTile T{0, j, 0, 0, {0, 0, 0, 0}};
      T.wmask = cover::strip_tile(a, e, ncb, j, t, T.rb);
      tiles[toff[j] + t] = T;
    }
  }
}

int count_tiles(int ncb) {
  int n = 0;
  for (int a = 0; a < ncb;) {
    const int e = cover::seg_end(a, ncb, ncb);
    for (int j = a; j < e; ++j) n += cover::strip_tiles(a, e, ncb, j);
    a = e;
  }
  return n;
}

// Errors: the return code, and the calling thread's message for
// flapw_last_error(NULL) (this entry point keeps no handle).
int fail(int code, const char* why) {
  set_thread_error(why);
  return code;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace flapw

using namespace flapw;

extern "C" int flapw_herk_noalloc(const void* Z, int64_t ldz, int K, int N, const int* sigma,
                                  void* H, int64_t ldh, int layout, int n_slices, void* stream) {
  (void)cudaGetLastError();
  if (!Z || !H) return fail(FLAPW_ERR_ARG, "NULL Z or H");
  if (K < 1 || N < 1 || ldz < K) return fail(FLAPW_ERR_ARG, "need K >= 1, N >= 1, ldz >= K");
  if (K >= kMaxK) return fail(FLAPW_ERR_UNSUPPORTED, "K must be below 131072");
  if (layout != FLAPW_LAYOUT_LOWER_FULL && layout != FLAPW_LAYOUT_LOWER_PACKED)
    return fail(FLAPW_ERR_ARG, "layout is not a FLAPW_LAYOUT_* value");
  if (layout == FLAPW_LAYOUT_LOWER_FULL && ldh < N) return fail(FLAPW_ERR_ARG, "ldh < N");
  const int s = n_slices ? n_slices : 7;
  if (s < 4 || s > 8) return fail(FLAPW_ERR_ARG, "n_slices must be 0 or in 4..8");
  if (!on_device(Z) || !on_device(H)) return fail(FLAPW_ERR_ARG, "Z and H must be device memory");
  SigmaBits sb;
  std::memset(sb.w, 0, sizeof(sb.w));
  int kp = 0, kn = 0;
  for (int k = 0; k < K; ++k) {
    const int v = sigma ? sigma[k] : 1;
    if (v != 1 && v != -1) return fail(FLAPW_ERR_ARG, "sigma entries must be +1 or -1");
    if (v > 0) {
      ++kp;
    } else {
      ++kn;
      sb.w[k >> 5] |= 1u << (k & 31);
    }
  }
  const int64_t kp_pad = neg_base(kp);
  int64_t k_alloc = (int64_t)k_chunks(kp, kn) * kChunk;
  if (k_alloc < kChunk) k_alloc = kChunk;
  const int ncb = (N + 63) / 64;
  const int n_tiles = count_tiles(ncb);

  // carve the scratch array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_err = take(8 * sizeof(int));
  const size_t o_kmap = take((size_t)k_alloc * sizeof(int));
  const size_t o_prob = take(sizeof(Prob));
  const size_t o_rowp = take((size_t)N * sizeof(int));
  const size_t o_rexp = take((size_t)N * sizeof(int));
  const size_t o_toff = take((size_t)(ncb + 1) * sizeof(int));
  const size_t o_tile = take((size_t)n_tiles * sizeof(EmuTile));
  const size_t o_z = take((size_t)N * k_alloc * 16);
  const size_t o_sl = take((size_t)s * 2 * N * k_alloc * 2);
  if (off > kScratchBytes) return fail(FLAPW_ERR_UNSUPPORTED, "problem larger than the scratch array");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(FLAPW_ERR_CUDA, "cudaGetDevice failed or device ordinal too large");
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) return fail(FLAPW_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      g_scratch_dev[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_dev[dev]);
  }

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = reinterpret_cast<int*>(base + o_err);
  int* kmap = reinterpret_cast<int*>(base + o_kmap);
  Prob* prob = reinterpret_cast<Prob*>(base + o_prob);
  int* rowp = reinterpret_cast<int*>(base + o_rowp);
  int* rexp = reinterpret_cast<int*>(base + o_rexp);
  int* toff = reinterpret_cast<int*>(base + o_toff);
  EmuTile* tiles = reinterpret_cast<EmuTile*>(base + o_tile);
  double2* Zs = reinterpret_cast<double2*>(base + o_z);
  __half* SL = reinterpret_cast<__half*>(base + o_sl);

  const Prob P{0, N, kp, kn, layout, /*col_base*/ 0, layout == FLAPW_LAYOUT_LOWER_FULL ? ldh : N,
               static_cast<double2*>(H)};
  SliceMaps tmap;
  std::string terr;
  if (!make_slice_tmaps(&tmap, SL, k_alloc, N, s, &terr)) return fail(FLAPW_ERR_CUDA, "tensor map encoding failed");
  if (herk_emu_init() != cudaSuccess) return fail(FLAPW_ERR_CUDA, "contraction kernel setup failed");
  cudaError_t e = cudaMemsetAsync(err, 0, 8 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(rowp, 0, (size_t)N * sizeof(int), st);
  if (e != cudaSuccess) return fail(FLAPW_ERR_CUDA, cudaGetErrorString(e));
  noalloc_setup_kernel<<<1, 256, 0, st>>>(sb, K, (int)kp_pad, (int)k_alloc, P, prob, kmap, ncb, toff, tiles);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_gather_Z(static_cast<const double2*>(Z), ldz, K, N, kmap, k_alloc, Zs, st);
  if (e == cudaSuccess) e = launch_slicer(Zs, k_alloc, prob, rowp, 0, N, 0, N, s, SL, rexp, st);
  if (e == cudaSuccess)
    e = launch_herk_emu(tmap, prob, tiles, n_tiles, rexp, s, fixed_frac_bits(K), err, 0,
                        SplitScratch{nullptr, nullptr}, herk_emu_deep(N), /*cyclic*/ true, 0, st);
  if (e != cudaSuccess) return fail(FLAPW_ERR_CUDA, cudaGetErrorString(e));
  return FLAPW_OK;
}
