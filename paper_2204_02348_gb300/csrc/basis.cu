// Output-basis transform: LG or custom coefficients as a matrix applied to the HG coefficients (user guide,
// digHoloConfigSetBasisTypeLG / digHoloConfigSetBasisTypeCustom: the field is decomposed in the separable HG
// basis and the coefficients are then multiplied by a transform matrix).
//
// One block takes kVB coefficient vectors (frame, polarisation) and stages them in shared memory; its threads
// take (vector, output mode) pairs, output mode fastest, and sum T[k][l] c[v][l] over the input modes l in
// ascending order, reading the transposed matrix T^T[l][k] (consecutive k in consecutive threads: one
// contiguous row segment per warp) and the staged inputs (a broadcast per vector).  The sums run in a fixed
// order, so results do not depend on the launch shape.
#include "kernels.cuh"

namespace dhk {

namespace {

constexpr int kVB = 8;           // coefficient vectors per block
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
    for (int t = threadIdx.x; t < nv * modes_out; t += kThreads) {
        const int v = t / modes_out, k = t - v * modes_out;
        const float2* in = s_in + v * modes_in;
        float2 acc = make_float2(0.f, 0.f);
        for (int l = 0; l < modes_in; ++l) acc = cmac(acc, __ldg(tt + (size_t)l * modes_out + k), in[l]);
        out[(size_t)(v0 + v) * modes_out + k] = acc;
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
