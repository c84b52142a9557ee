// Output-basis transform: LG or custom coefficients as a matrix applied to the HG coefficients (user guide,
// digHoloConfigSetBasisTypeLG / digHoloConfigSetBasisTypeCustom: the field is decomposed in the separable HG
// basis and the coefficients are then multiplied by a transform matrix).
//
// One block takes kVB coefficient vectors (frame, polarisation), stages them in shared memory, and every
// thread owns output modes k (strided by the block size): for each input mode l it reads T[k][l] from the
// transposed matrix (consecutive k in consecutive threads, so a warp reads one contiguous row segment) and
// accumulates it against the kVB staged inputs, which the warp reads as a broadcast.  The matrix is read once
// per block from L2; the sums run in ascending l, so results do not depend on the launch shape.
#include "kernels.cuh"

namespace dhk {

namespace {

constexpr int kVB = 16;          // coefficient vectors per block
constexpr int kThreads = 256;
constexpr int kMaxModesIn = DH_MAX_GROUPS * (DH_MAX_GROUPS + 1) / 2;

__device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}

__global__ void __launch_bounds__(kThreads) k_basis(const float2* __restrict__ hg, float2* __restrict__ out,
                                                    const float2* __restrict__ tt, int vectors, int modes_in,
                                                    int modes_out) {
    extern __shared__ float2 s_in[];   // [kVB][modes_in]
    const int v0 = blockIdx.x * kVB;
    const int nv = min(kVB, vectors - v0);
    for (int i = threadIdx.x; i < kVB * modes_in; i += kThreads) {
        const int v = i / modes_in;
        s_in[i] = v < nv ? hg[(size_t)v0 * modes_in + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < modes_out; k += kThreads) {
        float2 acc[kVB];
#pragma unroll
        for (int v = 0; v < kVB; ++v) acc[v] = make_float2(0.f, 0.f);
        for (int l = 0; l < modes_in; ++l) {
            const float2 t = __ldg(tt + (size_t)l * modes_out + k);
#pragma unroll
            for (int v = 0; v < kVB; ++v) acc[v] = cmac(acc[v], t, s_in[v * modes_in + l]);
        }
#pragma unroll
        for (int v = 0; v < kVB; ++v)
            if (v < nv) out[(size_t)(v0 + v) * modes_out + k] = acc[v];
    }
}

}  // namespace

cudaError_t basis_init() {
    return cudaFuncSetAttribute(k_basis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kVB * kMaxModesIn * sizeof(float2)));
}

cudaError_t launch_basis(const Plan& P, const float2* hg, float2* out, int vectors, cudaStream_t st,
                         StageTimer* timer) {
    if (vectors < 1 || P.modes < 1 || P.modes_out < 1 || !P.basis_tt) return cudaSuccess;
    if (P.modes > kMaxModesIn) return cudaErrorInvalidValue;
    const int blocks = (vectors + kVB - 1) / kVB;
    const size_t smem = (size_t)kVB * P.modes * sizeof(float2);
    if (timer) timer->start(st);
    k_basis<<<blocks, kThreads, smem, st>>>(hg, out, P.basis_tt, vectors, P.modes, P.modes_out);
    if (timer) timer->stop(st, "k_basis");
    return cudaGetLastError();
}

}  // namespace dhk
