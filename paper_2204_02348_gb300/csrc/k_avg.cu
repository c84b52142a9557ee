// Batch averaging (user guide, digHoloSetBatchAvg and the "Averaging modes" module): the kept Fourier windows
// of the avg_count frames of one averaging group are rotated into phase with the group's first frame and
// averaged before the single inverse transform of the group.
//
// The averaging runs on the windows after their inverse transform along x (the scratch between k_xpass and
// the last kernel): that transform is linear, and unitary up to a factor that is the same for every frame and
// polarisation, so both the phase-aligned sum and the inner products <W_0, W_j> that set the phases carry
// over unchanged.  The phase of a frame is one number for all its polarisations (the reference drift is
// common to them), so the relative phase between the polarisations is kept.
//
//   k_avg_dot : partial inner products sum conj(W_0) W_j over fixed slices of the window elements, one block
//               per (slice, member j >= 1, group); fixed-order block reduction.
//   k_avg_sum : every block re-sums its group's partials in slice order, forms the unit phasors
//               a_j = conj(d_j) / |d_j| (a_0 = 1; 1 when d_j = 0) and writes (1/A) sum_j a_j W_j.
// Deterministic: no atomics, every sum in a fixed order independent of the launch shape.
#include <algorithm>

#include "kernels.cuh"

namespace dhk {

namespace {

constexpr int kAvgThreads = 256;
constexpr int kAvgSlice = 8192;   // window elements per k_avg_dot block

__global__ void __launch_bounds__(kAvgThreads) k_avg_dot(const float2* __restrict__ g, float2* __restrict__ part,
                                                         long long elems, int slices, int members,
                                                         long long mstride, long long gstride, AvgExtents X) {
    __shared__ float2 red[kAvgThreads / 32];
    const int s = blockIdx.x, j = blockIdx.y + 1, gi = blockIdx.z;
    const float2* w0 = g + (size_t)gi * gstride;
    const float2* wj = w0 + (size_t)j * mstride;
    const long long e0 = (long long)s * kAvgSlice;
    const long long e1 = e0 + kAvgSlice < elems ? e0 + kAvgSlice : elems;
    float2 acc = make_float2(0.f, 0.f);
    for (long long e = e0 + threadIdx.x; e < e1; e += kAvgThreads) {
        const long long o0 = (long long)gi * gstride + e, oj = o0 + (long long)j * mstride;
        if (!(DH_IN(X.status, o0, X.g_len, kSiteAvg) && DH_IN(X.status, oj, X.g_len, kSiteAvg))) continue;
        const float2 a = w0[e], b = wj[e];
        acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
        acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = red[0];
        for (int w = 1; w < kAvgThreads / 32; ++w) {
            t.x += red[w].x;
            t.y += red[w].y;
        }
        if (DH_IN(X.status, ((long long)gi * members + j) * slices + s, X.part_len, kSiteAvg))
            part[((size_t)gi * members + j) * slices + s] = t;
    }
}

__global__ void __launch_bounds__(kAvgThreads) k_avg_sum(const float2* __restrict__ g, const float2* __restrict__ part,
                                                         float2* __restrict__ out, long long elems, int slices,
                                                         int members, long long mstride, long long gstride, AvgExtents X) {
    extern __shared__ float2 phasor[];   // [members]
    const int gi = blockIdx.y;
    for (int j = threadIdx.x; j < members; j += kAvgThreads) {
        float2 a = make_float2(1.f, 0.f);
        if (j > 0) {
            float2 d = make_float2(0.f, 0.f);
            const float2* pj = part + ((size_t)gi * members + j) * slices;
            for (int s = 0; s < slices; ++s) {
                if (!DH_IN(X.status, ((long long)gi * members + j) * slices + s, X.part_len, kSiteAvg)) continue;
                d.x += pj[s].x;
                d.y += pj[s].y;
            }
            const float n2 = d.x * d.x + d.y * d.y;
            if (n2 > 0.f) {
                const float inv = 1.f / sqrtf(n2);
                a = make_float2(d.x * inv, -d.y * inv);
            }
        }
        phasor[j] = a;
    }
    __syncthreads();
    const float scale = 1.f / (float)members;
    const float2* base = g + (size_t)gi * gstride;
    float2* o = out + (size_t)gi * elems;
    for (long long e = (long long)blockIdx.x * kAvgThreads + threadIdx.x; e < elems;
         e += (long long)gridDim.x * kAvgThreads) {
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0; j < members; ++j) {
            if (!DH_IN(X.status, (long long)gi * gstride + (long long)j * mstride + e, X.g_len, kSiteAvg)) continue;
            const float2 a = phasor[j], w = base[(size_t)j * mstride + e];
            acc.x = fmaf(a.x, w.x, fmaf(-a.y, w.y, acc.x));
            acc.y = fmaf(a.x, w.y, fmaf(a.y, w.x, acc.y));
        }
        if (DH_IN(X.status, (long long)gi * elems + e, X.out_len, kSiteAvg)) o[e] = make_float2(acc.x * scale, acc.y * scale);
    }
}

}  // namespace

int avg_slices(long long elems) { return (int)((elems + kAvgSlice - 1) / kAvgSlice); }

cudaError_t launch_avg(const float2* g, float2* part, float2* out, int groups, int members, long long elems,
                       long long mstride, long long gstride, const AvgExtents& X, cudaStream_t st, StageTimer* tm) {
    if (groups < 1 || members < 1 || elems < 1) return cudaSuccess;
    if (groups > 65535 || members > DH_MAX_AVG_COUNT) return cudaErrorInvalidValue;
    const int slices = avg_slices(elems);
    if (members > 1) {
        if (tm) tm->start(st);
        k_avg_dot<<<dim3(slices, members - 1, groups), kAvgThreads, 0, st>>>(g, part, elems, slices, members,
                                                                             mstride, gstride, X);
        if (tm) tm->stop(st, "k_avg_dot");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long long per_block = (long long)kAvgThreads * 4;
    const int gx = (int)std::min<long long>((elems + per_block - 1) / per_block, 65535);
    if (tm) tm->start(st);
    k_avg_sum<<<dim3(gx, groups), kAvgThreads, (size_t)members * sizeof(float2), st>>>(g, part, out, elems, slices,
                                                                                      members, mstride, gstride, X);
    if (tm) tm->stop(st, "k_avg_sum");
    return cudaGetLastError();
}

}  // namespace dhk
