// Fifth-generation tensor-core building blocks (tcgen05) shared by the split-BF16 contractions: shared-memory
// matrix descriptors for the no-swizzle K-major canonical layout, the BF16 MMA with FP32 accumulation in
// tensor memory, and the 32-lane tensor-memory load.
//
// Canonical layout (no swizzle, K-major): 8-row x 16-byte core matrices stored contiguously, core (rb, kb) at
// (rb * K/8 + kb) * 128 bytes; a descriptor's leading-dimension offset (between cores along K) is then 128
// bytes and its stride-dimension offset (between 8-row groups) 16 K bytes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dhk {

// Offset in elements of (row, k) in a [rows][K] bf16 operand in the canonical layout above.
__host__ __device__ __forceinline__ int umma_off(int row, int k, int K) {
    return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;                 // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an FP32 accumulator, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D (tensor memory) = A B (+ D when accumulate != 0), issued by one thread.
__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive on the mbarrier once every MMA this thread issued has completed.
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

// Sixteen consecutive 32-bit columns of this warp's 32 tensor-memory lanes, one lane per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(v[i]);
}

// Allocate / free `cols` tensor-memory columns (a power of two >= 32); called by one whole warp.  The
// allocated address is written to the shared-memory word `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols));
}

}  // namespace dhk
