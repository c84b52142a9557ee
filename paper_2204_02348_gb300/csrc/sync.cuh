// Bounded waits on shared-memory mbarriers, shared by every kernel that waits on one.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dhk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Wait until the mbarrier at shared address `mbar` completes the phase with the given parity, trying at most
// `limit` times (each try may itself suspend briefly).  Returns false when the limit ran out.
__device__ __forceinline__ bool bounded_mbar_wait(uint32_t mbar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

}  // namespace dhk
