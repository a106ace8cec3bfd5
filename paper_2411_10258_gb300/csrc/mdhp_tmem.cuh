// Tensor memory (TMEM) as a per-thread feature store.
//
// Each SM of sm_100-class parts has 256 KB of tensor memory: 128 lanes x 512
// columns of 32 bits, allocated per CTA in columns.  A warp may touch only
// the 32 lanes of its quarter (warp index mod 4), and with the 32x32b access
// shape thread i of the warp reads or writes lane 32 * (warp % 4) + i.  So a
// thread can keep a private row of up to 512 floats there and read it back
// with one instruction per 32 (or 16) floats, beside its registers and the
// CTA's shared memory.  The decoupled fit keeps the first feature steps of
// every thread there instead of re-reading them from the global scratch at
// every iteration.
//
// All accesses are warp-collective (.sync.aligned): every thread of a warp
// must execute them together, with the same address operand pattern.  Loads
// are issued together with their wait, so their results cannot be consumed
// before they arrive.
#pragma once

#include <cstdint>

namespace mdhp {

__device__ __forceinline__ void tm_alloc(uint32_t dst_saddr, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_saddr),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tm_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tm_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

#define MDHP_U(v) "r"(__float_as_uint(v))

// Store NQ float4 (4 NQ consecutive columns of this thread's lane), NQ = 4 or 8.
template <int NQ>
__device__ __forceinline__ void tm_st(uint32_t taddr, const float4 (&x)[NQ]) {
  static_assert(NQ == 4 || NQ == 8, "16 or 32 columns");
  if constexpr (NQ == 8) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        MDHP_U(x[0].x), MDHP_U(x[0].y), MDHP_U(x[0].z), MDHP_U(x[0].w), MDHP_U(x[1].x),
        MDHP_U(x[1].y), MDHP_U(x[1].z), MDHP_U(x[1].w), MDHP_U(x[2].x), MDHP_U(x[2].y),
        MDHP_U(x[2].z), MDHP_U(x[2].w), MDHP_U(x[3].x), MDHP_U(x[3].y), MDHP_U(x[3].z),
        MDHP_U(x[3].w), MDHP_U(x[4].x), MDHP_U(x[4].y), MDHP_U(x[4].z), MDHP_U(x[4].w),
        MDHP_U(x[5].x), MDHP_U(x[5].y), MDHP_U(x[5].z), MDHP_U(x[5].w), MDHP_U(x[6].x),
        MDHP_U(x[6].y), MDHP_U(x[6].z), MDHP_U(x[6].w), MDHP_U(x[7].x), MDHP_U(x[7].y),
        MDHP_U(x[7].z), MDHP_U(x[7].w)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        MDHP_U(x[0].x), MDHP_U(x[0].y), MDHP_U(x[0].z), MDHP_U(x[0].w), MDHP_U(x[1].x),
        MDHP_U(x[1].y), MDHP_U(x[1].z), MDHP_U(x[1].w), MDHP_U(x[2].x), MDHP_U(x[2].y),
        MDHP_U(x[2].z), MDHP_U(x[2].w), MDHP_U(x[3].x), MDHP_U(x[3].y), MDHP_U(x[3].z),
        MDHP_U(x[3].w)
        : "memory");
  }
}
#undef MDHP_U

// Load NQ float4 from this thread's lane and wait for them (one asm block:
// the registers are defined only after the wait).
template <int NQ>
__device__ __forceinline__ void tm_ld(uint32_t taddr, float4 (&x)[NQ]) {
  static_assert(NQ == 4 || NQ == 8, "16 or 32 columns");
  uint32_t r[4 * NQ];
  if constexpr (NQ == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    x[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                       __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
}

}  // namespace mdhp
