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
    // float2 region: r1, union, twiddles N and M, phase x / y, correction x / y
    static constexpr int F2 = R1 + UN + kFN + M + 4 * M;
    // float region: hg_x, hg_y [kFGMax][M]; int region: posM, mask lo / hi, mode m / n
    static constexpr int FL = 2 * kFGMax * M;
    static constexpr int IN = 3 * M + 2 * (kFGMax * (kFGMax + 1) / 2);
    static constexpr size_t bytes = (size_t)F2 * sizeof(float2) + (size_t)FL * sizeof(float) + (size_t)IN * sizeof(int);
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

// Raw pixel pair held between its load and its use: two uint16 in one word, or two floats.
template <typename T>
struct RawPair;
template <>
struct RawPair<uint16_t> {
    using type = uint32_t;
    static __device__ __forceinline__ uint32_t load(const uint16_t* p, bool vec) {
        if (vec) return __ldg(reinterpret_cast<const unsigned int*>(p));
        return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 16);
    }
    static __device__ __forceinline__ float2 value(uint32_t u) {
        return make_float2((float)(u & 0xffffu), (float)(u >> 16));
    }
};
template <>
struct RawPair<float> {
    using type = float2;
    static __device__ __forceinline__ float2 load(const float* p, bool vec) { return load_pair(p, vec); }
    static __device__ __forceinline__ float2 value(float2 v) { return v; }
};

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
    float2* phx = twM + M;
    float2* phy = phx + M;
    float2* cx = phy + M;
    float2* cy = cx + M;
    float* hgx = reinterpret_cast<float*>(cy + M);
    float* hgy = hgx + kFGMax * M;
    int* posM = reinterpret_cast<int*>(hgy + kFGMax * M);
    int* mlo = posM + M;
    int* mhi = mlo + M;
    int* mdm = mhi + M;
    int* mdn = mdm + kFGMax * (kFGMax + 1) / 2;
    const int tid = threadIdx.x;
    // every block serves one polarisation: its tables are staged once
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    const int G = P.groups, modes = P.modes;
    for (int i = tid; i < N; i += NT) twN[i] = P.tw_fwd_n[i];
    for (int i = tid; i < M; i += NT) {
        twM[i] = P.tw_inv_m[i];
        posM[i] = P.pos_m[i];
        phx[i] = pd.phase_x[i];
        phy[i] = pd.phase_y[i];
        cx[i] = pd.corr_x[i];
        cy[i] = pd.corr_y[i];
        mlo[i] = pd.mask_lo[i];
        mhi[i] = pd.mask_hi[i];
    }
    for (int i = tid; i < G * M; i += NT) {
        hgx[i] = pd.hg_x[i];
        hgy[i] = pd.hg_y[i];
    }
    for (int i = tid; i < modes; i += NT) {
        mdm[i] = P.mode_m[i];
        mdn[i] = P.mode_n[i];
    }
    __syncthreads();
    const bool vec = A.vec_ok != 0;
    const int fstride = gridDim.x / P.pols;
    for (int b = blockIdx.x / P.pols; b < A.count; b += fstride) {
        const int f = A.frame0 + b;
        const T* fr = static_cast<const T*>(A.src) + (size_t)f * P.width * P.height + (size_t)pd.oy * P.width + pd.ox;

        // ---------------------------------------------------------------- y pass, two chunks of 32 column pairs
        // (the second chunk's pixel pairs are loaded before the first chunk is transformed)
        using RP = RawPair<T>;
        typename RP::type pre[16];
        {
            const int c = tid & 31, j = tid >> 5;
#pragma unroll
            for (int r = 0; r < 16; ++r) pre[r] = RP::load(fr + (size_t)(j + 8 * r) * P.width + 2 * c, vec);
        }
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            {
                const int c = tid & 31, j = tid >> 5;
                float2 v[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = RP::value(pre[r]);
                if (cc == 0) {
#pragma unroll
                    for (int r = 0; r < 16; ++r)
                        pre[r] = RP::load(fr + (size_t)(j + 8 * r) * P.width + 2 * (c + kFCY), vec);
                }
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
            const int lo = mlo[q], hi = mhi[q];
            const float2 py = phy[q];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int p = (d + 16 * r - pd.klx) & (N - 1);
                if (p < M) {
                    float2 val = make_float2(0.f, 0.f);
                    if (p >= lo && p <= hi) val = cmul(cmul(v[r], phx[p]), py);
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
            const float2 e = cmul(cmul(un[a], cx[i]), cy[j]);
            un[a] = e;
            if (fld) fld[t] = e;
        }
        __syncthreads();

        // ---------------------------------------------------------------- HG overlap
        if (A.coefs && G > 0) {
            constexpr int JQ = NT / M;                 // thread groups splitting the y sum
            constexpr int JL = (M + JQ - 1) / JQ;
            float2* part = r1;                         // [JQ][G][M]
            float2* tsum = r1 + JQ * kFGMax * M;       // [G][M]
            if (tid < JQ * M) {
                const int i = tid % M, jq = tid / M;
                const int j0 = jq * JL, j1 = min(M, j0 + JL);
                float2 acc[kFGMax];
#pragma unroll
                for (int n = 0; n < kFGMax; ++n) acc[n] = make_float2(0.f, 0.f);
#pragma unroll
                for (int jj = 0; jj < JL; ++jj) {
                    const int j = j0 + jj;
                    if (j < j1) {
                        const float2 e = un[i * PITCH + posM[j]];
#pragma unroll
                        for (int n = 0; n < kFGMax; ++n) {
                            if (n < G) {
                                const float u = hgy[n * M + j];
                                acc[n].x = fmaf(u, e.x, acc[n].x);
                                acc[n].y = fmaf(u, e.y, acc[n].y);
                            }
                        }
                    }
                }
#pragma unroll
                for (int n = 0; n < kFGMax; ++n)
                    if (n < G) part[(jq * G + n) * M + i] = acc[n];
            }
            __syncthreads();
            // T[n][i]: the y partial sums added in a fixed order
            for (int t = tid; t < G * M; t += NT) {
                float2 v = part[t];
#pragma unroll
                for (int jq = 1; jq < JQ; ++jq) {
                    const float2 w = part[jq * G * M + t];
                    v.x += w.x;
                    v.y += w.y;
                }
                tsum[t] = v;
            }
            __syncthreads();
            // c_mn = sum_i u_m(x'_i) T[n][i]: one warp per mode, fixed shuffle tree
            const int warp = tid >> 5, lane = tid & 31;
            float2* cf = A.coefs + (size_t)(f * P.pols + pol) * modes;
            // modes k = warp + 8 (k0 + kk), groups of KW: independent products first, then interleaved
            // shuffle trees
            constexpr int KW = 4;
            for (int k0 = 0; warp + k0 * (NT / 32) < modes; k0 += KW) {
            float2 s[KW];
#pragma unroll
            for (int kk = 0; kk < KW; ++kk) {
                s[kk] = make_float2(0.f, 0.f);
                const int k = warp + (k0 + kk) * (NT / 32);
                if (k < modes) {
                    const float* um = hgx + mdm[k] * M;
                    const float2* tn = tsum + mdn[k] * M;
#pragma unroll
                    for (int i = lane; i < M; i += 32) {
                        const float u = um[i];
                        const float2 t = tn[i];
                        s[kk].x = fmaf(u, t.x, s[kk].x);
                        s[kk].y = fmaf(u, t.y, s[kk].y);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int kk = 0; kk < KW; ++kk) {
                    s[kk].x += __shfl_xor_sync(0xffffffffu, s[kk].x, o);
                    s[kk].y += __shfl_xor_sync(0xffffffffu, s[kk].y, o);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int kk = 0; kk < KW; ++kk) {
                    const int k = warp + (k0 + kk) * (NT / 32);
                    if (k < modes) cf[k] = s[kk];
                }
            }
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
    // blocks serve one polarisation each: the grid is a multiple of the polarisation count
    const long long per_pol = std::min<long long>(batch, (2LL * g_sm_count[dev]) / P.pols);
    const int grid = (int)std::max<long long>(1, per_pol) * P.pols;
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
