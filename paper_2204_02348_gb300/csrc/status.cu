// Device status readback and the bounded-wait self-check.
#include <cuda_runtime.h>

#include "runtime.hpp"
#include "sync.cuh"

namespace dhk {

// One thread waits on an mbarrier that nothing ever arrives on, with the same bounded wait the kernels use,
// and reports whether the limit ran out (1) or the barrier completed (0).
__global__ void k_wait_selfcheck(long limit, int* expired) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        const bool ok = bounded_mbar_wait(smem_u32(&mbar), 0, limit);
        *expired = ok ? 0 : 1;
    }
}

}  // namespace dhk

using namespace dh;

extern "C" int dh_get_device_status(dh_handle h, int* status) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    if (!status) return fail(DH_ERROR_NULLPOINTER, "status is null");
    std::lock_guard<std::mutex> lk(H->mu);
    *status = 0;
    if (!H->d_blob || !H->plan.status) return DH_SUCCESS;
    cudaError_t e = cudaMemcpy(status, H->plan.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status readback");
    const int zero = 0;
    e = cudaMemcpy(H->plan.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "status clear");
    return DH_SUCCESS;
}

extern "C" int dh_check_bounded_wait(long long limit, int* expired) {
    if (!expired) return fail(DH_ERROR_NULLPOINTER, "expired is null");
    if (limit < 1) return fail(DH_ERROR_INVALIDARGUMENT, "limit must be >= 1");
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return fail(DH_ERROR_MEMORYALLOCATION, "self-check flag");
    dhk::k_wait_selfcheck<<<1, 32>>>((long)limit, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(expired, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-check");
    return DH_SUCCESS;
}
