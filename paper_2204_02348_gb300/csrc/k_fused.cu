// Fused single-kernel path for 128 x 128 windows (field sizes 32, 48 and 64): one thread block reconstructs
// one (frame, polarisation) window entirely in shared memory, persistent over windows, two blocks per SM.
//
// Per window (the guide's pipeline steps 1-3 and digHoloProcessRemoveTilt):
//   y pass   pairs of adjacent real columns (x, x+1) packed as one complex column; radix-16 DIF pass straight
//            from global memory (coalesced 32-bit / 64-bit pixel-pair loads), radix-8 pass fused with the
//            separation of the two real spectra (Z(k), conj Z(-k)) and the selection of the M box rows;
//   x pass   radix-16 then radix-8 DIF along x on the M box rows, the second pass fused with the box-column
//            selection, the circular mask and the beam-centre phase;
//   inverse  M-point inverse transform along x (DIT, digit-reversed in / natural out) and along y (DIF,
//            natural in / digit-reversed out), in place;
//   epilogue residual tilt and defocus removal, field write (coalesced along x), and the separable HG
//            contraction: partial sums over y per thread group, then one warp per mode sums over x with a
//            fixed shuffle tree (deterministic, no atomics).
// Shared memory: r1[N][M+1] box rows (x-major, padded pitch) and one union region used in turn as the y-pass
// tile, the M x (M+1) window / field, and the overlap partials; twiddles and the digit-reversal table.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fft.cuh"
#include "runtime.hpp"

namespace dhk {

constexpr int kFN = 128;          // window size of this path
constexpr int kFThreads = 256;
constexpr int kFCY = 32;          // column pairs per y-pass chunk
constexpr int kFGMax = 16;        // largest group count of this path

struct FusedArgs {
    const void* src;              // frames [B][H][W]
    int frame0, count;
    int vec_ok;                   // 1 when pixel pairs can be loaded as one aligned vector
    float2* fields;               // nullable [B][pol][M][M]
    float2* coefs;                // nullable [B][pol][modes]
};

template <int M>
struct FusedLayout {
    static constexpr int PITCH = M + 1;
    static constexpr int R1 = kFN * PITCH;
    static constexpr int ZT = kFN * kFCY;
    static constexpr int WB = M * PITCH;
    static constexpr int UN = ZT > WB ? ZT : WB;
    static constexpr size_t bytes = (size_t)(R1 + UN + kFN + M) * sizeof(float2) + (size_t)M * sizeof(int);
};

__device__ __forceinline__ float2 load_pair(const uint16_t* p, bool vec) {
    if (vec) {
        const uint32_t u = __ldg(reinterpret_cast<const unsigned int*>(p));
        return make_float2((float)(u & 0xffffu), (float)(u >> 16));
    }
    return make_float2((float)__ldg(p), (float)__ldg(p + 1));
}

__device__ __forceinline__ float2 load_pair(const float* p, bool vec) {
    if (vec) return __ldg(reinterpret_cast<const float2*>(p));
    return make_float2(__ldg(p), __ldg(p + 1));
}

// Write the separated spectra of columns x and x+1 at frequency k (if k is a box row).
__device__ __forceinline__ void emit_pair(float2* r1, int pitch, int M, int kly, int x, int k, float2 zk, float2 zm) {
    int q = (k - kly) % kFN;
    if (q < 0) q += kFN;
    if (q < M) {
        r1[x * pitch + q] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        r1[(x + 1) * pitch + q] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
}

template <int M, int MR0, int MR1, typename T>
__global__ void __launch_bounds__(kFThreads, 2) k_fused128(const __grid_constant__ Plan P,
                                                           const __grid_constant__ FusedArgs A) {
    using L = FusedLayout<M>;
    constexpr int N = kFN, PITCH = L::PITCH, NT = kFThreads;
    extern __shared__ float2 smem[];
    float2* r1 = smem;
    float2* un = r1 + L::R1;
    float2* twN = un + L::UN;
    float2* twM = twN + N;
    int* posM = reinterpret_cast<int*>(twM + M);
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += NT) twN[i] = P.tw_fwd_n[i];
    for (int i = tid; i < M; i += NT) {
        twM[i] = P.tw_inv_m[i];
        posM[i] = P.pos_m[i];
    }
    __syncthreads();
    const int G = P.groups, modes = P.modes;
    const int total = A.count * P.pols;
    const bool vec = A.vec_ok != 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int b = w / P.pols, pol = w - b * P.pols;
        const int f = A.frame0 + b;
        const PolDev& pd = P.pol[pol];
        const T* fr = static_cast<const T*>(A.src) + (size_t)f * P.width * P.height + (size_t)pd.oy * P.width + pd.ox;

        // ---------------------------------------------------------------- y pass, two chunks of 32 column pairs
        for (int cc = 0; cc < 2; ++cc) {
            {
                const int c = tid & 31, j = tid >> 5;
                const int x = 2 * (c + kFCY * cc);
                float2 v[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = load_pair(fr + (size_t)(j + 8 * r) * P.width + x, vec);
                dft16<false>(v);
#pragma unroll
                for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twN[j * r]);
#pragma unroll
                for (int r = 0; r < 16; ++r) un[(j + 8 * r) * kFCY + c] = v[r];
            }
            __syncthreads();
            {
                const int c = tid & 31, u = tid >> 5;
                const int d1 = u, d2 = (u == 0) ? 8 : 16 - u;
                float2 z1[8], z2[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    z1[r] = un[(8 * d1 + r) * kFCY + c];
                    z2[r] = un[(8 * d2 + r) * kFCY + c];
                }
                dft8<false>(z1);
                dft8<false>(z2);
                const int x = 2 * (c + kFCY * cc);
                if (u != 0) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        emit_pair(r1, PITCH, M, pd.kly, x, d1 + 16 * r, z1[r], z2[7 - r]);
                        emit_pair(r1, PITCH, M, pd.kly, x, d2 + 16 * r, z2[r], z1[7 - r]);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        emit_pair(r1, PITCH, M, pd.kly, x, 16 * r, z1[r], z1[(8 - r) & 7]);
                        emit_pair(r1, PITCH, M, pd.kly, x, 8 + 16 * r, z2[r], z2[7 - r]);
                    }
                }
            }
            __syncthreads();
        }

        // ---------------------------------------------------------------- x pass on the M box rows
        spass<16, false, false, N, N, M, PITCH, 1, NT>(r1, twN, tid);
        __syncthreads();
        for (int t = tid; t < M * 16; t += NT) {
            const int q = t % M, d = t / M;
            float2 v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) v[r] = r1[(8 * d + r) * PITCH + q];
            dft8<false>(v);
            const int lo = __ldg(&pd.mask_lo[q]), hi = __ldg(&pd.mask_hi[q]);
            const float2 phy = __ldg(&pd.phase_y[q]);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                int p = (d + 16 * r - pd.klx) % N;
                if (p < 0) p += N;
                if (p < M) {
                    float2 val = make_float2(0.f, 0.f);
                    if (p >= lo && p <= hi) val = cmul(cmul(v[r], __ldg(&pd.phase_x[p])), phy);
                    un[posM[p] * PITCH + q] = val;
                }
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- inverse transforms
        spass<MR1, true, true, M, MR1, M, PITCH, 1, NT>(un, twM, tid);
        __syncthreads();
        spass<MR0, true, true, M, M, M, PITCH, 1, NT>(un, twM, tid);
        __syncthreads();
        spass<MR0, true, false, M, M, M, 1, PITCH, NT>(un, twM, tid);
        __syncthreads();
        spass<MR1, true, false, M, MR1, M, 1, PITCH, NT>(un, twM, tid);
        __syncthreads();

        // ---------------------------------------------------------------- correction and field
        float2* fld = A.fields ? A.fields + (size_t)(f * P.pols + pol) * M * M : nullptr;
        for (int t = tid; t < M * M; t += NT) {
            const int i = t % M, j = t / M;
            const int a = i * PITCH + posM[j];
            const float2 e = cmul(cmul(un[a], __ldg(&pd.corr_x[i])), __ldg(&pd.corr_y[j]));
            un[a] = e;
            if (fld) fld[t] = e;
        }
        __syncthreads();

        // ---------------------------------------------------------------- HG overlap
        if (A.coefs && G > 0) {
            constexpr int JQ = NT / M;                 // thread groups splitting the y sum
            constexpr int JL = (M + JQ - 1) / JQ;
            float2* part = r1;                         // [JQ][G][M]
            if (tid < JQ * M) {
                const int i = tid % M, jq = tid / M;
                const int j0 = jq * JL, j1 = min(M, j0 + JL);
                float2 acc[kFGMax];
#pragma unroll
                for (int n = 0; n < kFGMax; ++n) acc[n] = make_float2(0.f, 0.f);
                for (int j = j0; j < j1; ++j) {
                    const float2 e = un[i * PITCH + posM[j]];
#pragma unroll
                    for (int n = 0; n < kFGMax; ++n) {
                        if (n < G) {
                            const float u = __ldg(&pd.hg_y[n * M + j]);
                            acc[n].x = fmaf(u, e.x, acc[n].x);
                            acc[n].y = fmaf(u, e.y, acc[n].y);
                        }
                    }
                }
#pragma unroll
                for (int n = 0; n < kFGMax; ++n)
                    if (n < G) part[(jq * G + n) * M + i] = acc[n];
            }
            __syncthreads();
            const int warp = tid >> 5, lane = tid & 31;
            float2* cf = A.coefs + (size_t)(f * P.pols + pol) * modes;
            for (int k = warp; k < modes; k += NT / 32) {
                const int m = __ldg(&P.mode_m[k]), n = __ldg(&P.mode_n[k]);
                float2 s = make_float2(0.f, 0.f);
                for (int i = lane; i < M; i += 32) {
                    float2 tsum = part[n * M + i];
#pragma unroll
                    for (int jq = 1; jq < JQ; ++jq) {
                        const float2 v = part[(jq * G + n) * M + i];
                        tsum.x += v.x;
                        tsum.y += v.y;
                    }
                    const float u = __ldg(&pd.hg_x[m * M + i]);
                    s.x = fmaf(u, tsum.x, s.x);
                    s.y = fmaf(u, tsum.y, s.y);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
                }
                if (lane == 0) cf[k] = s;
            }
        }
        __syncthreads();
    }
}

template <int M, int MR0, int MR1>
static cudaError_t set_attr() {
    cudaError_t e;
    const int bytes = (int)FusedLayout<M>::bytes;
    if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    return cudaFuncSetAttribute(k_fused128<M, MR0, MR1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int M, int MR0, int MR1>
static void launch(const Plan& P, const FusedArgs& A, int dtype, int grid, cudaStream_t st) {
    const size_t bytes = FusedLayout<M>::bytes;
    if (dtype == DH_DTYPE_U16)
        k_fused128<M, MR0, MR1, uint16_t><<<grid, kFThreads, bytes, st>>>(P, A);
    else
        k_fused128<M, MR0, MR1, float><<<grid, kFThreads, bytes, st>>>(P, A);
}

}  // namespace dhk

namespace dh {

static int g_sm_count[64] = {0};

bool use_fused(const dhk::Plan& P) {
    if (P.n != dhk::kFN || P.groups > dhk::kFGMax || P.precision != DH_PRECISION_FP32) return false;
    return P.m == 32 || P.m == 48 || P.m == 64;
}

cudaError_t fused_init() {
    cudaError_t e;
    if ((e = dhk::set_attr<32, 8, 4>())) return e;
    if ((e = dhk::set_attr<48, 16, 3>())) return e;
    return dhk::set_attr<64, 8, 8>();
}

int launch_fused_path(Handle* H, const void* frames, int dtype, int batch, void* fields, void* coefs,
                      cudaStream_t st, dhk::StageTimer* tm) {
    const dhk::Plan& P = H->plan;
    int dev = H->device;
    if (dev < 0 || dev >= 64) return fail(DH_ERROR_ERROR, "device index out of range");
    if (!g_sm_count[dev]) {
        int n = 0;
        cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device attribute");
        g_sm_count[dev] = n;
    }
    dhk::FusedArgs A;
    A.src = frames;
    A.frame0 = 0;
    A.count = batch;
    const int esz = dtype == DH_DTYPE_U16 ? 2 : 4;
    bool ok = (P.width % 2 == 0) && (((uintptr_t)frames) % (2 * esz) == 0);
    for (int p = 0; p < P.pols; ++p) ok = ok && (P.pol[p].ox % 2 == 0);
    A.vec_ok = ok ? 1 : 0;
    A.fields = (float2*)fields;
    A.coefs = (float2*)coefs;
    const long long windows = (long long)batch * P.pols;
    const int grid = (int)std::min<long long>(windows, 2LL * g_sm_count[dev]);
    if (tm) tm->start(st);
    switch (P.m) {
        case 32: dhk::launch<32, 8, 4>(P, A, dtype, grid, st); break;
        case 48: dhk::launch<48, 16, 3>(P, A, dtype, grid, st); break;
        default: dhk::launch<64, 8, 8>(P, A, dtype, grid, st); break;
    }
    if (tm) tm->stop(st, "k_fused128");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DH_SUCCESS;
}

}  // namespace dh
