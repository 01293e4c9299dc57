// Device helpers shared by the tcgen05 kernels: shared-memory addresses,
// mbarriers with bounded waits, TMA tile loads, UMMA shared-memory
// descriptors, TMEM loads and the FP32 -> 64-bit fixed-point drain.
#pragma once

#include <cstdint>

#include "flapw_internal.h"

namespace flapw {
namespace tc {

// Default bound of the abortable waits (4 s; a kernel argument, settable per
// handle) and fixed bound of the teardown waits, which wait for work that
// was already issued.
constexpr unsigned long long kWaitNs = 4000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Arrive on a barrier given by its cluster address (any CTA of the cluster).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cbar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Abort flag of a CTA, and optionally the cluster address of its peer's flag.
// A role that gives up raises both.
struct Abort {
  volatile int* local;
  uint32_t peer;
  bool has_peer;
  unsigned long long limit_ns;  // bound of each abortable wait
  __device__ void raise() const {
    *local = 1;
    if (has_peer) asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer), "r"(1) : "memory");
  }
};

// Bounded wait.  Returns false if the wall-clock limit passed or another role
// aborted; the first role to time out raises the abort flags.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const Abort& ab) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*ab.local) return false;
      if (global_ns() - t0 > ab.limit_ns) {
        ab.raise();
        return false;
      }
    }
  }
}
// After an abort, copies that one CTA of a pair issued may complete on its
// peer's barrier, which nobody waits for: every thread of an aborted CTA
// lets 20 us pass (far longer than a tile copy takes) before the pair's
// closing barrier, so that nothing is still landing in shared memory when
// the CTAs exit.
__device__ __forceinline__ void settle_after_abort(const Abort& ab) {
  if (!*ab.local) return;
  const unsigned long long t0 = global_ns();
  while (global_ns() - t0 < 20000ull) {
  }
}
// Wait that ignores the abort flags (teardown), still bounded.
__device__ __forceinline__ void mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitNs) break;
}

// K-major, 128-byte-swizzled operand: 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// tcgen05.wait::ld that also marks the loaded registers as written here, so
// the compiler cannot read them before the wait.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

// acc[o + n] += f(v_n) for the integer values v_n of NC consecutive TMEM
// columns from tb (this thread's lane), n < NC.  The next 8 columns load while
// the current 8 are converted.
template <int NC, int NA, class F>
__device__ __forceinline__ void drain_cols(uint32_t tb, long long (&acc)[NA], int o, F f) {
  static_assert(NC % 16 == 0, "column count");
  uint32_t xa[8], xb[8];
  tmem_ld8(tb, xa);
  tmem_wait_ld_regs(xa);
#pragma unroll
  for (int cb = 0; cb < NC / 8; ++cb) {
    if (cb & 1) {
      if (cb + 1 < NC / 8) tmem_ld8(tb + 8u * (cb + 1), xa);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[o + 8 * cb + e] += f(__float2int_rn(__uint_as_float(xb[e])));
      if (cb + 1 < NC / 8) tmem_wait_ld_regs(xa);
    } else {
      if (cb + 1 < NC / 8) tmem_ld8(tb + 8u * (cb + 1), xb);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[o + 8 * cb + e] += f(__float2int_rn(__uint_as_float(xa[e])));
      if (cb + 1 < NC / 8) tmem_wait_ld_regs(xb);
    }
  }
}

// Adds sign * v * 2^sh (rounded half up below the fixed point) for the NC
// integer-valued FP32 columns from tb to acc[o..o+NC).  |v| <= 2^24 and
// sh <= 36: one 32 x 32 -> 64-bit multiply-add per value where sh >= 0.
template <int NC, int NA>
__device__ __forceinline__ void drain_fixed(uint32_t tb, long long (&acc)[NA], int o, int sh,
                                            bool sub) {
  if (sh >= 0) {
    const int pre = sh > 30 ? sh - 30 : 0;
    const int mul = sub ? -(1 << (sh - pre)) : (1 << (sh - pre));
    if (pre == 0) drain_cols<NC>(tb, acc, o, [=](int v) { return (long long)v * mul; });
    else drain_cols<NC>(tb, acc, o, [=](int v) { return (long long)(v << pre) * mul; });
  } else {
    const int rs = -sh, half = 1 << (-sh - 1);
    drain_cols<NC>(tb, acc, o, [=](int v) { return (long long)(((sub ? -v : v) + half) >> rs); });
  }
}

}  // namespace tc
}  // namespace flapw
