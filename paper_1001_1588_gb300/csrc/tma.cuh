// Bulk asynchronous copies global -> shared (the TMA's 1-D bulk path) completed
// on an mbarrier, with bounded waits.
//
// One thread arms a barrier with the number of bytes it expects and issues the
// copies; the CTA then waits for the barrier's phase.  The wait is bounded by
// the global timer: if the copies have not landed after kWaitNs the waiting
// thread records kStatusTimeout in the plan's status word, waits once more
// (again bounded) so that no copy is still writing into shared memory, and the
// whole CTA returns.  Copies need 16-byte aligned addresses and sizes that are
// multiples of 16 bytes.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace fftenkf {

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async (copy) proxy
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// Tensor load global -> shared of one 3-D box (coordinates innermost first, the
// innermost one a multiple of 16 bytes), completed on an mbarrier like bulk_g2s.
// The shared destination must be 128-byte aligned.
__device__ __forceinline__ void tensor_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// CTA-wide wait for `parity` of `bar`, observed by thread 0.  Returns false
// (for every thread) after a timeout; the caller must then return.  expire
// (a test setting) makes the wait give up at once, as an expired one does:
// the timeout is recorded and the copies in flight are drained before the
// CTA leaves.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, int* status, int* flag, bool expire = false) {
  if (threadIdx.x == 0) {
    bool ok = !expire && mbar_wait_bounded(bar, parity);
    if (!ok) {
      atomicOr(status, kStatusTimeout);
      mbar_wait_bounded(bar, parity);  // let copies in flight land before leaving
    }
    *flag = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag != 0;
}

}  // namespace fftenkf
