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
//
// The array's name in host code is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, once per device, on the
// first call made with that device current.  That first call should come
// before any stream capture.  All calls share the array and it keeps the
// previous call's contents: what must start at zero is cleared on the stream,
// and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.
#include <cstdio>
#include <mutex>

#include "flapw_internal.h"

namespace flapw {
namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// kmap[k'] = original row of operand column k' (sigma = +1 rows, then from
// kp_pad the sigma = -1 rows), -1 in the padding.  One thread: K is small.
__global__ void noalloc_kmap_kernel(const int* sigma, int K, int kp_pad, int k_alloc, int* kmap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < k_alloc; ++i) kmap[i] = -1;
  int p = 0, q = 0;
  for (int k = 0; k < K; ++k) {
    const int s = sigma ? sigma[k] : 1;
    if (s > 0) kmap[p++] = k;
    else kmap[kp_pad + q++] = k;
  }
}

// Lower-triangle tiles (256 x 64) in bands of 2 row blocks, column by column.
__global__ void noalloc_tiles_kernel(int N, EmuTile* tiles) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nib = (N + 255) / 256, njb = (N + 63) / 64;
  int t = 0;
  for (int i0 = 0; i0 < nib; i0 += 2)
    for (int jb = 0; jb < njb; ++jb)
      for (int ib = i0; ib < min(nib, i0 + 2); ++ib)
        if (jb * 64 <= ib * 256 + 255) tiles[t++] = EmuTile{0, ib, jb, 0};
}

int count_tiles(int N) {
  const int nib = (N + 255) / 256, njb = (N + 63) / 64;
  int t = 0;
  for (int ib = 0; ib < nib; ++ib)
    for (int jb = 0; jb < njb; ++jb)
      if (jb * 64 <= ib * 256 + 255) ++t;
  return t;
}

// Errors are reported by return code only (this entry point keeps no handle).
int fail(int code, const char* /*why*/) { return code; }

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
  if (layout != FLAPW_LAYOUT_LOWER_FULL && layout != FLAPW_LAYOUT_LOWER_PACKED)
    return fail(FLAPW_ERR_ARG, "layout is not a FLAPW_LAYOUT_* value");
  if (layout == FLAPW_LAYOUT_LOWER_FULL && ldh < N) return fail(FLAPW_ERR_ARG, "ldh < N");
  const int s = n_slices ? n_slices : 7;
  if (s < 4 || s > 8) return fail(FLAPW_ERR_ARG, "n_slices must be 0 or in 4..8");
  if (!on_device(Z) || !on_device(H)) return fail(FLAPW_ERR_ARG, "Z and H must be device memory");
  int kp = 0, kn = 0;
  for (int k = 0; k < K; ++k) {
    const int v = sigma ? sigma[k] : 1;
    if (v != 1 && v != -1) return fail(FLAPW_ERR_ARG, "sigma entries must be +1 or -1");
    (v > 0 ? kp : kn)++;
  }
  const int64_t kp_pad = (kp + kChunk - 1) / kChunk * kChunk;
  int64_t k_alloc = kp_pad + (kn + kChunk - 1) / kChunk * kChunk;
  if (k_alloc < kChunk) k_alloc = kChunk;
  const int n_tiles = count_tiles(N);

  // carve the scratch array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_err = take(8 * sizeof(int));
  const size_t o_sig = take((size_t)K * sizeof(int));
  const size_t o_kmap = take((size_t)k_alloc * sizeof(int));
  const size_t o_prob = take(sizeof(Prob));
  const size_t o_rowp = take((size_t)N * sizeof(int));
  const size_t o_rexp = take((size_t)N * sizeof(int));
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
  int* dsig = reinterpret_cast<int*>(base + o_sig);
  int* kmap = reinterpret_cast<int*>(base + o_kmap);
  Prob* prob = reinterpret_cast<Prob*>(base + o_prob);
  int* rowp = reinterpret_cast<int*>(base + o_rowp);
  int* rexp = reinterpret_cast<int*>(base + o_rexp);
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
  if (e == cudaSuccess && sigma)
    e = cudaMemcpyAsync(dsig, sigma, (size_t)K * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(prob, &P, sizeof(Prob), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(FLAPW_ERR_CUDA, cudaGetErrorString(e));
  noalloc_kmap_kernel<<<1, 32, 0, st>>>(sigma ? dsig : nullptr, K, (int)kp_pad, (int)k_alloc, kmap);
  noalloc_tiles_kernel<<<1, 32, 0, st>>>(N, tiles);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_gather_Z(static_cast<const double2*>(Z), ldz, K, N, kmap, k_alloc, Zs, st);
  if (e == cudaSuccess) e = launch_slicer(Zs, k_alloc, prob, rowp, 0, N, 0, N, s, SL, rexp, st);
  if (e == cudaSuccess)
    e = launch_herk_emu(tmap, prob, tiles, n_tiles, rexp, s, fixed_frac_bits(K), err, 0,
                        SplitScratch{nullptr, nullptr}, herk_emu_deep(N), st);
  if (e != cudaSuccess) return fail(FLAPW_ERR_CUDA, cudaGetErrorString(e));
  return FLAPW_OK;
}
