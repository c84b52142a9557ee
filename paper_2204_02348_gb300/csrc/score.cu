// Alignment-candidate scoring: total captured power of every frame under every candidate setting (the
// quantity the guide's AutoAlign search maximises while it perturbs tilt, defocus and waist).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "runtime.hpp"

namespace dhk {

// power[b * count + s] = sum over pols and modes of |c|^2, summed in a fixed order by one warp per frame.
__global__ void k_power(const float2* __restrict__ coefs, int per_frame, int frames, float* __restrict__ power,
                        int count, int s) {
    const int b = blockIdx.x;
    if (b >= frames) return;
    const float2* c = coefs + (size_t)b * per_frame;
    float acc = 0.f;
    for (int k = threadIdx.x; k < per_frame; k += 32) acc = fmaf(c[k].x, c[k].x, fmaf(c[k].y, c[k].y, acc));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) power[(size_t)b * count + s] = acc;
}

}  // namespace dhk

using namespace dh;

extern "C" int dh_score_settings(dh_handle h, const void* d_frames, int dtype, int batch, const dh_setting* settings,
                                 int count, float* d_power, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    if (!d_frames || !settings || !d_power) return fail(DH_ERROR_NULLPOINTER, "null pointer");
    if (count < 1) return fail(DH_ERROR_INVALIDARGUMENT, "candidate count must be >= 1");
    if (dtype != DH_DTYPE_U16 && dtype != DH_DTYPE_F32) return fail(DH_ERROR_INVALIDARGUMENT, "bad dtype");
    if (batch < 1) batch = 1;
    int rc = ensure_plan(H);
    if (rc) return rc;
    if (H->plan.modes == 0) return fail(DH_ERROR_INVALIDARGUMENT, "scoring needs a basis (group count > 0)");
    cudaStream_t st = (cudaStream_t)stream;
    // candidate plans: geometry and tables of every candidate, validated before any work is queued
    std::vector<void*> blobs;
    std::vector<dhk::Plan> plans;
    auto cleanup = [&]() {
        if (!blobs.empty()) cudaStreamSynchronize(st);
        for (void* b : blobs) cudaFree(b);
    };
    for (int s = 0; s < count; ++s) {
        Geometry g;
        std::string why;
        rc = build_geometry_candidate(H->s, settings[s], &g, &why);
        if (rc) {
            cleanup();
            return fail(rc, "candidate " + std::to_string(s) + ": " + why);
        }
        Tables t;
        build_tables(H->s, g, &t);
        void* blob = nullptr;
        dhk::Plan P;
        rc = upload_plan(H->s, g, t, &blob, &P);
        if (rc) {
            cleanup();
            return rc;
        }
        blobs.push_back(blob);
        plans.push_back(P);
    }
    const dhk::Plan& P0 = H->plan;
    const int per_frame = P0.pols * P0.modes;
    const size_t per_frame_scratch = split_window_bytes(P0) * P0.pols;
    int chunk = (int)std::max<size_t>(1, kScratchTarget / per_frame_scratch);
    chunk = std::min(chunk, batch);
    const size_t coef_bytes = ((size_t)batch * per_frame * sizeof(float2) + 255) & ~(size_t)255;
    rc = ensure_scratch(H, per_frame_scratch * chunk + coef_bytes);
    if (rc) {
        cleanup();
        return rc;
    }
    float2* coefs = (float2*)((char*)H->d_scratch + per_frame_scratch * chunk);
    for (int s = 0; s < count; ++s) {
        rc = run_split(plans[s], H->d_scratch, per_frame_scratch * chunk, d_frames, dtype, batch, nullptr, nullptr,
                       coefs, st, H->timer());
        if (rc) {
            cleanup();
            return rc;
        }
        if (H->timer()) H->prof.start(st);
        dhk::k_power<<<batch, 32, 0, st>>>(coefs, per_frame, batch, d_power, count, s);
        if (H->timer()) H->prof.stop(st, "k_power");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "power");
        }
    }
    cleanup();
    return DH_SUCCESS;
}
