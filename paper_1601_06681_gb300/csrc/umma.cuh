// tcgen05 helpers shared by the tensor-core sweeps: shared-memory matrix
// descriptors for the canonical K-major layout without swizzle, element
// offsets in that layout, bounded mbarrier waits and TMEM loads.
//
// K-major, no swizzle: 8-row x 16-byte core matrices; core matrices adjacent
// along K are 128 bytes apart (leading byte offset) and 8-row groups are
// (K bytes / 16) * 128 bytes apart (stride byte offset).
#pragma once

#include <cstdint>

namespace ehdg {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                    // descriptor version of sm_100-family MMA
  return d;                                  // base offset 0, no swizzle
}

// byte offset of element (row, k) in the K-major no-swizzle layout
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int kbyte, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(kbyte >> 4) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(kbyte & 15);
}

// Instruction descriptor of kind::f16 / kind::tf32 with FP32 accumulation,
// K-major A and B: fmt 1 = BF16, 2 = TF32.
__host__ __device__ __forceinline__ uint32_t umma_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Poll an mbarrier phase at most `limit` times; false if it never completed.
__device__ __forceinline__ bool mbar_wait_bounded(const uint64_t* bar, uint32_t parity,
                                                  uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
        " selp.u32 %0, 1, 0, w;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 8 consecutive 32-bit TMEM columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                 "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

// 2 consecutive 32-bit TMEM columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(v[0]), "=r"(v[1])
               : "r"(taddr));
}

}  // namespace ehdg
