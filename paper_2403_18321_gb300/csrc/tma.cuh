// tma.cuh -- mbarrier and TMA (cp.async.bulk) helpers shared by the
// streaming kernels.  Every wait is bounded: after one second of
// globaltimer it raises *abort (shared) and reports failure, so that no
// role can wait forever on a copy or an arrival that never comes.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace gbpca {

constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s bound on every wait

// A position in a ring of n stages -- the stage and the parity of its current
// phase -- advanced one slot at a time (no division in the per-chunk loops).
struct Ring {
  int n, idx;
  uint32_t phase;
  __device__ explicit Ring(int n_) : n(n_), idx(0), phase(0u) {}
  __device__ __forceinline__ void next() {
    if (++idx == n) { idx = 0; phase ^= 1u; }
  }
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same test, but a thread whose phase is not complete is suspended until it
// completes or `ns` nanoseconds pass, instead of returning at once: a waiting
// warp then takes no issue slots from the warps doing the work.
__device__ __forceinline__ bool mbar_try_suspend(uint64_t* b, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait; false on time-out or when another role already aborted.  The
// first test is inline (the common case of a phase already complete costs no
// call); the loop is out of line.
static __device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t parity, int* abort) {
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try_suspend(b, parity, 1000000u)) return true;
    if (*(volatile int*)abort) return false;
    if (gtimer() - t0 > kWaitNs) {
      atomicExch(abort, 1);
      return false;
    }
  }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* abort) {
  return mbar_try(b, parity) || mbar_wait_slow(b, parity, abort);
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}
// 2-D tiled copy of box (x, y) of a tensor map into shared memory.  x times the
// element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace gbpca
