// Tensor memory (TMEM) as per-thread storage.
//
// Each SM has 128 lanes x 512 columns of 32-bit tensor memory next to its tensor
// cores.  Nothing on this path multiplies matrices, but a kernel can allocate the
// columns and keep per-thread tables there: a warp reads and writes only the 32
// lanes of its quadrant (warp mod 4), thread l of the warp lane 32 (warp mod 4) + l,
// and tcgen05.ld / tcgen05.st move runs of consecutive columns of that lane to and
// from registers without touching shared memory.  The column passes keep their
// per-wavenumber covariance accumulators and gains there (160 KB for a 4096-point
// column of 4 blocks), leaving shared memory to the bulk-copy stages and the FFT
// exchanges.
//
// Every load here waits for its data in the same asm statement, so no register is
// read early (tm_ld2: two loads, then one wait, in one statement).  Stores
// are asynchronous: a caller that reads columns it stored earlier calls
// tm_wait_st() first (once, before a batch of loads).
#pragma once
#include <stdint.h>

#include "tma.cuh"

namespace fftenkf {

// allocate ncols (a power of two >= 32) columns for the CTA; the whole warp calls it,
// and the TMEM address is written to *slot (shared memory)
__device__ __forceinline__ void tm_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// free them (the warp that allocated, after every thread's last access and a CTA barrier)
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// this thread's lane, column col0 of the allocation at base
__device__ __forceinline__ uint32_t tm_addr(uint32_t base, int col0) {
  const uint32_t warp = threadIdx.x >> 5;
  return base + (((warp & 3u) * 32u) << 16) + (uint32_t)col0;
}

__device__ __forceinline__ void tm_ld8(uint32_t a, float* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
      : "r"(a)
      : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t a, const float* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(a),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7])
      : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t a, float* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(a)
      : "memory");
}
__device__ __forceinline__ void tm_st16(uint32_t a, const float* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(a),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]),
      "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
      : "memory");
}
// wait for this thread's earlier stores
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 consecutive columns, one wait
__device__ __forceinline__ void tm_ld32(uint32_t a, float* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]), "=f"(r[16]),
        "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]), "=f"(r[24]),
        "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31])
      : "r"(a)
      : "memory");
}
__device__ __forceinline__ void tm_st32(uint32_t a, const float* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(a),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]),
      "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15]), "f"(r[16]), "f"(r[17]), "f"(r[18]),
      "f"(r[19]), "f"(r[20]), "f"(r[21]), "f"(r[22]), "f"(r[23]), "f"(r[24]), "f"(r[25]), "f"(r[26]), "f"(r[27]),
      "f"(r[28]), "f"(r[29]), "f"(r[30]), "f"(r[31])
      : "memory");
}

// n consecutive columns (n a multiple of 8, known at compile time)
template <int n>
__device__ __forceinline__ void tm_ld(uint32_t a, float* r) {
  static_assert(n % 8 == 0, "multiples of 8 columns");
#pragma unroll
  for (int c = 0; c < n;) {
    if (n - c >= 32) {
      tm_ld32(a + c, r + c);
      c += 32;
    } else if (n - c >= 16) {
      tm_ld16(a + c, r + c);
      c += 16;
    } else {
      tm_ld8(a + c, r + c);
      c += 8;
    }
  }
}
template <int n>
__device__ __forceinline__ void tm_st(uint32_t a, const float* r) {
  static_assert(n % 8 == 0, "multiples of 8 columns");
#pragma unroll
  for (int c = 0; c < n;) {
    if (n - c >= 32) {
      tm_st32(a + c, r + c);
      c += 32;
    } else if (n - c >= 16) {
      tm_st16(a + c, r + c);
      c += 16;
    } else {
      tm_st8(a + c, r + c);
      c += 8;
    }
  }
}

// two loads and one wait in one asm statement: 16 + 32 or 32 + 32 columns
__device__ __forceinline__ void tm_ld16_32(uint32_t a1, float* r, uint32_t a2, float* q) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%49];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]),
        "=f"(q[0]), "=f"(q[1]), "=f"(q[2]), "=f"(q[3]), "=f"(q[4]), "=f"(q[5]), "=f"(q[6]), "=f"(q[7]), "=f"(q[8]),
        "=f"(q[9]), "=f"(q[10]), "=f"(q[11]), "=f"(q[12]), "=f"(q[13]), "=f"(q[14]), "=f"(q[15]), "=f"(q[16]),
        "=f"(q[17]), "=f"(q[18]), "=f"(q[19]), "=f"(q[20]), "=f"(q[21]), "=f"(q[22]), "=f"(q[23]), "=f"(q[24]),
        "=f"(q[25]), "=f"(q[26]), "=f"(q[27]), "=f"(q[28]), "=f"(q[29]), "=f"(q[30]), "=f"(q[31])
      : "r"(a1), "r"(a2)
      : "memory");
}
__device__ __forceinline__ void tm_ld32_32(uint32_t a1, float* r, uint32_t a2, float* q) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]), "=f"(r[16]),
        "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]), "=f"(r[24]),
        "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31]),
        "=f"(q[0]), "=f"(q[1]), "=f"(q[2]), "=f"(q[3]), "=f"(q[4]), "=f"(q[5]), "=f"(q[6]), "=f"(q[7]), "=f"(q[8]),
        "=f"(q[9]), "=f"(q[10]), "=f"(q[11]), "=f"(q[12]), "=f"(q[13]), "=f"(q[14]), "=f"(q[15]), "=f"(q[16]),
        "=f"(q[17]), "=f"(q[18]), "=f"(q[19]), "=f"(q[20]), "=f"(q[21]), "=f"(q[22]), "=f"(q[23]), "=f"(q[24]),
        "=f"(q[25]), "=f"(q[26]), "=f"(q[27]), "=f"(q[28]), "=f"(q[29]), "=f"(q[30]), "=f"(q[31])
      : "r"(a1), "r"(a2)
      : "memory");
}
// n1 columns at a1 and n2 at a2, one wait for both where a single statement covers the pair
// (16 + 32, 32 + 32); otherwise two waited loads
template <int n1, int n2>
__device__ __forceinline__ void tm_ld2(uint32_t a1, float* r1, uint32_t a2, float* r2) {
  if constexpr (n1 == 16 && n2 == 32) {
    tm_ld16_32(a1, r1, a2, r2);
  } else if constexpr (n1 == 32 && n2 == 32) {
    tm_ld32_32(a1, r1, a2, r2);
  } else {
    tm_ld<n1>(a1, r1);
    tm_ld<n2>(a2, r2);
  }
}

}  // namespace fftenkf
