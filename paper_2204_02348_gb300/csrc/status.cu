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

// One thread guards an access one element past the end of a four-element extent: the bounds-checked build refuses
// it and records site kSiteProbe; the guarded block is empty, so neither build touches memory here.
__global__ void k_bounds_probe(int* status) {
    if (threadIdx.x == 0 && DH_IN(status, 4, 4, kSiteProbe)) {
    }
}

}  // namespace dhk

using namespace dh;

// Read and clear `words` ints of a status block; a null block reads as zero.
static int read_clear(const int* blk, int* out, int words) {
    for (int i = 0; i < words; ++i) out[i] = 0;
    if (!blk) return DH_SUCCESS;
    cudaError_t e = cudaMemcpy(out, blk, sizeof(int) * words, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status readback");
    const int zero[4] = {0, 0, 0, 0};
    e = cudaMemcpy(const_cast<int*>(blk), zero, sizeof(int) * words, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "status clear");
    return DH_SUCCESS;
}

static int* current_noalloc_block() {
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess ? noalloc_status_block(dev) : nullptr;
}

extern "C" int dh_get_device_status(dh_handle h, int* status) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    if (!status) return fail(DH_ERROR_NULLPOINTER, "status is null");
    std::lock_guard<std::mutex> lk(H->mu);
    *status = 0;
    int a = 0, b = 0;
    int rc = read_clear(H->d_blob ? H->plan.status : nullptr, &a, 1);
    if (rc) return rc;
    rc = read_clear(current_noalloc_block(), &b, 1);
    if (rc) return rc;
    *status = a | b;
    return DH_SUCCESS;
}

extern "C" int dh_get_check_record(dh_handle h, int* site, int* offset, int* extent) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    if (!site || !offset || !extent) return fail(DH_ERROR_NULLPOINTER, "site, offset or extent is null");
    std::lock_guard<std::mutex> lk(H->mu);
    *site = *offset = *extent = 0;
    int rec[3], rec_na[3];
    int rc = read_clear(H->d_blob && H->plan.status ? H->plan.status + 1 : nullptr, rec, 3);
    if (rc) return rc;
    const int* na = current_noalloc_block();
    rc = read_clear(na ? na + 1 : nullptr, rec_na, 3);
    if (rc) return rc;
    const int* r = rec[0] ? rec : rec_na;
    *site = r[0];
    *offset = r[1];
    *extent = r[2];
    return DH_SUCCESS;
}

extern "C" int dh_checked_build(int* checked) {
    if (!checked) return fail(DH_ERROR_NULLPOINTER, "checked is null");
    *checked = dhk::kChecked ? 1 : 0;
    return DH_SUCCESS;
}

extern "C" int dh_check_bounds_probe(dh_handle h) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    int rc = ensure_plan(H);
    if (rc) return rc;
    dhk::k_bounds_probe<<<1, 32>>>(H->plan.status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "bounds probe");
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
