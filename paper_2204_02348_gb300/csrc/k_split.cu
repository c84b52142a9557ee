// Generic reconstruction path: three kernels joined by L2-sized scratch, for any window N (16..1024,
// power of two) and field size M (multiple of 16 with a 19-smooth odd part).
//
//   k_ypass : pipeline step 1, first half.  Pairs of real window columns (x, x + N/2) are packed into one
//             complex column, transformed along y (N-point DIF), and the M box rows (k_y in
//             [k0y - M/2, k0y + M/2) mod N) of both real columns are separated from the packed spectrum.
//             Writes r1[q][x] (M x N complex per window).
//   k_xpass : pipeline step 1, second half, and step 2 along x.  Each box row is transformed along x
//             (N-point DIF); the M box columns are selected, masked by the circular window and multiplied by
//             the beam-centre phase and 1/N, then inverse transformed along x (M-point DIT).  Writes g[q][i].
//   k_yinv  : step 2 along y, tilt/defocus removal and step 3.  Column chunks of g are inverse transformed
//             along y, multiplied by the separable correction, written as the field, and contracted with the
//             Hermite-Gaussian tables (first over y, on sums and differences of mirrored rows, then over x)
//             into per-mode accumulators held in registers, in a fixed order (deterministic, no atomics).
#include <algorithm>

#include "fft.cuh"
#include "kernels.cuh"

namespace dhk {

constexpr int kThreads = 256;
constexpr int kChunkI = 32;      // columns per k_yinv chunk
constexpr int kMaxSmem = 227 * 1024;

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_ypass(const __grid_constant__ Plan P, const __grid_constant__ Batch B,
                                                    int logc) {
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int C = 1 << logc;
    // columns: N_x (packed pairs x, x + N_x/2); transform length N_y along y; M_y box rows
    const int N = P.n, M = P.my, NY = P.ny, half = N / 2;
    const int pol = blockIdx.y;
    const PolDev& pd = P.pol[pol];
    const int x0 = blockIdx.x * C;
    for (int fb = blockIdx.z; fb < B.count; fb += gridDim.z) {
        const int f = B.frame0 + fb;
        const T* fr = (const T*)B.src + (size_t)f * P.width * P.height;
        for (int idx = tid; idx < NY * C; idx += nthr) {
            const int y = idx >> logc, c = idx & (C - 1);
            const long long po = (long long)(pd.oy + y) * P.width + pd.ox + x0 + c;
            const T* row = fr + po;
            float2 v = DH_IN(P.status, po + half, (long long)P.width * P.height, kSiteYpassFrame)
                           ? make_float2(to_f(row[0]), to_f(row[half])) : make_float2(0.f, 0.f);
            if (pd.cal) {
                const float* k = pd.cal + (size_t)y * N + x0 + c;
                v.x *= __ldg(k);
                v.y *= __ldg(k + half);
            }
            smem[idx] = v;
        }
        __syncthreads();
        fft_run<false>(smem, NY, P.rad_ny, P.nrad_ny, logc, C, P.tw_fwd_ny, tid, nthr);
        float2* r1 = B.r1 + (size_t)(fb * P.pols + pol) * M * N;
        for (int idx = tid; idx < M * C; idx += nthr) {
            const int q = idx >> logc, c = idx & (C - 1);
            int k = (pd.kly + q) % NY;
            if (k < 0) k += NY;
            const int km = (NY - k) & (NY - 1);
            const float2 za = smem[P.pos_ny[k] * C + c];
            const float2 zb = smem[P.pos_ny[km] * C + c];
            // column x: (Z(k) + conj Z(-k)) / 2 ; column x + N/2: (Z(k) - conj Z(-k)) / (2i)
            if (DH_IN(P.status, (long long)(fb * P.pols + pol) * M * N + (long long)q * N + x0 + c + half, B.r1_len, kSiteYpassR1)) {
                if (DH_IN(P.status, (long long)(fb * P.pols + pol) * M * N + (long long)q * N + x0 + c + half, B.r1_len, kSiteYpassR1)) {
                    r1[(size_t)q * N + x0 + c] = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
                    r1[(size_t)q * N + x0 + c + half] = make_float2(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x));
                }
            }
        }
        __syncthreads();
    }
}

// Four consecutive pixels as one load (8 bytes of uint16, 16 bytes of float32) and their values as float.
template <typename T>
struct Pix4;
template <>
struct Pix4<uint16_t> {
    using type = uint2;
    __device__ __forceinline__ static void unpack(uint2 w, float* p) {
        p[0] = (float)(w.x & 0xFFFFu);
        p[1] = (float)(w.x >> 16);
        p[2] = (float)(w.y & 0xFFFFu);
        p[3] = (float)(w.y >> 16);
    }
};
template <>
struct Pix4<float> {
    using type = float4;
    __device__ __forceinline__ static void unpack(float4 w, float* p) {
        p[0] = w.x;
        p[1] = w.y;
        p[2] = w.z;
        p[3] = w.w;
    }
};

// k_ypass for the power-of-two windows, with the host plan's radix sequence fixed at compile time (128: 16 x 8,
// 256: 16 x 16, 512: 8 x 8 x 8, 1024: 16 x 8 x 8): no runtime radix dispatch, twiddles staged in shared
// memory, 2^LOGC column pairs per block, three blocks per SM (four at N = 256, whose 16-pair tiles fit 64
// registers).  Same inputs, outputs and arithmetic order as k_ypass.
template <typename T, int N, int R0, int R1, int R2, int LOGC>
__global__ void __launch_bounds__(kThreads, (N == 256 && LOGC == 4) ? 4 : 3) k_ypass_s(const __grid_constant__ Plan P, const __grid_constant__ Batch B) {
    extern __shared__ float2 smem[];   // [N][C] tile, then the twiddles W_N^k
    constexpr int C = 1 << LOGC, half = N / 2;
    static_assert(R0 * R1 * R2 == N, "the radices multiply to N");
    float2* tw = smem + N * C;
    const int tid = threadIdx.x;
    const int M = P.m;
    const int pol = blockIdx.y;
    const PolDev& pd = P.pol[pol];
    const int x0 = blockIdx.x * C;
    for (int i = tid; i < N; i += kThreads) tw[i] = P.tw_fwd_n[i];
    static_assert((N * C) % (8 * kThreads) == 0, "whole load batches");
    const bool r1_16 = ((uintptr_t)B.r1 & 15) == 0;   // M N is even: every window's rows stay 16-byte aligned
    for (int fb = blockIdx.z; fb < B.count; fb += gridDim.z) {
        const int f = B.frame0 + fb;
        const T* fr = (const T*)B.src + (size_t)f * P.width * P.height;
        if (((pd.ox + x0) & 3) == 0 && (P.width & 3) == 0) {
            // the block's columns start on a 4-pixel boundary: four pixels of each column group per load, eight
            // (uint16) or four (float32) such load pairs in flight per thread
            using V4 = typename Pix4<T>::type;
            constexpr int LB = sizeof(T) == 2 ? 8 : 4, Q = C / 4;
            for (int i0 = tid; i0 < N * Q; i0 += LB * kThreads) {
                V4 a[LB], b[LB];
#pragma unroll
                for (int u = 0; u < LB; ++u) {
                    const int idx = i0 + u * kThreads;
                    if (idx < N * Q) {
                        const int y = idx / Q, c = (idx % Q) * 4;
                        const long long po = (long long)(pd.oy + y) * P.width + pd.ox + x0 + c;
                        const T* row = fr + po;
                        if (DH_IN(P.status, po + half + 3, (long long)P.width * P.height, kSiteYpassFrame)) {
                            a[u] = *reinterpret_cast<const V4*>(row);
                            b[u] = *reinterpret_cast<const V4*>(row + half);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < LB; ++u) {
                    const int idx = i0 + u * kThreads;
                    if (idx < N * Q) {
                        const int y = idx / Q, c = (idx % Q) * 4;
                        float pa[4], pb[4];
                        Pix4<T>::unpack(a[u], pa);
                        Pix4<T>::unpack(b[u], pb);
                        float2 v[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = make_float2(pa[e], pb[e]);
                        if (pd.cal) {
                            const float* k = pd.cal + (size_t)y * N + x0 + c;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                v[e].x *= __ldg(k + e);
                                v[e].y *= __ldg(k + half + e);
                            }
                        }
                        float4* d = reinterpret_cast<float4*>(smem + y * C + c);
                        d[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
                        d[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
                    }
                }
            }
        } else {
            // eight pixel pairs in flight per thread before their shared-memory stores
            for (int i0 = tid; i0 < N * C; i0 += 8 * kThreads) {
                T a[8], b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = i0 + u * kThreads;
                    const int y = idx >> LOGC, c = idx & (C - 1);
                    const long long po = (long long)(pd.oy + y) * P.width + pd.ox + x0 + c;
                    const T* row = fr + po;
                    if (DH_IN(P.status, po + half, (long long)P.width * P.height, kSiteYpassFrame)) {
                        a[u] = row[0];
                        b[u] = row[half];
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = i0 + u * kThreads;
                    float2 v = make_float2(to_f(a[u]), to_f(b[u]));
                    if (pd.cal) {
                        const int y = idx >> LOGC, c = idx & (C - 1);
                        const float* k = pd.cal + (size_t)y * N + x0 + c;
                        v.x *= __ldg(k);
                        v.y *= __ldg(k + half);
                    }
                    smem[idx] = v;
                }
            }
        }
        __syncthreads();
        spass<R0, false, false, N, N, C, C, 1, kThreads>(smem, tw, tid);
        __syncthreads();
        spass<R1, false, false, N, N / R0, C, C, 1, kThreads>(smem, tw, tid);
        __syncthreads();
        if constexpr (R2 > 1) {
            spass<R2, false, false, N, N / (R0 * R1), C, C, 1, kThreads>(smem, tw, tid);
            __syncthreads();
        }
        float2* r1 = B.r1 + (size_t)(fb * P.pols + pol) * M * N;
        if (r1_16) {
            // two adjacent column pairs per thread: 16-byte shared-memory reads and global writes
            for (int idx = tid; idx < M * C / 2; idx += kThreads) {
                const int q = idx / (C / 2), c = 2 * (idx % (C / 2));
                int k = (pd.kly + q) % N;
                if (k < 0) k += N;
                const int km = (N - k) & (N - 1);
                const float4 za = *reinterpret_cast<const float4*>(smem + dif_pos<R0, R1, R2>(k) * C + c);
                const float4 zb = *reinterpret_cast<const float4*>(smem + dif_pos<R0, R1, R2>(km) * C + c);
                if (DH_IN(P.status, (long long)(fb * P.pols + pol) * M * N + (long long)q * N + x0 + c + half + 1, B.r1_len,
                          kSiteYpassR1) &&
                    DH_ALIGNED16(P.status, r1 + (size_t)q * N + x0 + c) && DH_ALIGNED16(P.status, r1 + (size_t)q * N + x0 + c + half)) {
                    *reinterpret_cast<float4*>(r1 + (size_t)q * N + x0 + c) =
                        make_float4(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y), 0.5f * (za.z + zb.z), 0.5f * (za.w - zb.w));
                    *reinterpret_cast<float4*>(r1 + (size_t)q * N + x0 + c + half) =
                        make_float4(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x), 0.5f * (za.w + zb.w), 0.5f * (zb.z - za.z));
                }
            }
        } else {
            for (int idx = tid; idx < M * C; idx += kThreads) {
                const int q = idx >> LOGC, c = idx & (C - 1);
                int k = (pd.kly + q) % N;
                if (k < 0) k += N;
                const int km = (N - k) & (N - 1);
                const float2 za = smem[dif_pos<R0, R1, R2>(k) * C + c];
                const float2 zb = smem[dif_pos<R0, R1, R2>(km) * C + c];
                if (DH_IN(P.status, (long long)(fb * P.pols + pol) * M * N + (long long)q * N + x0 + c + half, B.r1_len, kSiteYpassR1)) {
                    r1[(size_t)q * N + x0 + c] = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
                    r1[(size_t)q * N + x0 + c + half] = make_float2(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x));
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int N, int R0, int R1, int R2, int LOGC>
static void launch_ys(const Plan& P, const Batch& B, int zf, cudaStream_t st) {
    constexpr int C = 1 << LOGC;
    dim3 g((N / 2) / C, P.pols, zf);
    const size_t sm = ((size_t)N * C + N) * sizeof(float2);
    k_ypass_s<T, N, R0, R1, R2, LOGC><<<g, kThreads, sm, st>>>(P, B);
}

template <typename T>
static bool launch_ypass_static(const Plan& P, const Batch& B, int zf, cudaStream_t st) {
    // only for the host's radix plans of these sizes
    auto is = [&](int a, int b, int c) {
        const int n = c > 1 ? 3 : 2;
        return P.nrad_n == n && P.rad_n[0] == a && P.rad_n[1] == b && (n == 2 || P.rad_n[2] == c);
    };
    switch (P.n) {
        case 128: if (!is(16, 8, 1)) return false; launch_ys<T, 128, 16, 8, 1, 5>(P, B, zf, st); return true;
        case 256: if (!is(16, 16, 1)) return false; launch_ys<T, 256, 16, 16, 1, 4>(P, B, zf, st); return true;
        case 512: if (!is(8, 8, 8)) return false; launch_ys<T, 512, 8, 8, 8, 4>(P, B, zf, st); return true;
        case 1024: if (!is(16, 8, 8)) return false; launch_ys<T, 1024, 16, 8, 8, 3>(P, B, zf, st); return true;
        default: return false;
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_xpass(const __grid_constant__ Plan P, const __grid_constant__ Batch B,
                                                    int logr, int logn) {
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int R = 1 << logr, es = R + 1;
    // M_y box rows of N_x values each; M_x box columns kept and inverse transformed along x
    const int N = P.n, M = P.m, MY = P.my;
    float2* bufN = smem;
    float2* bufM = smem + (size_t)N * es;
    const int pol = blockIdx.y;
    const PolDev& pd = P.pol[pol];
    const int q0 = blockIdx.x * R;
    for (int fb = blockIdx.z; fb < B.count; fb += gridDim.z) {
        const int f = B.frame0 + fb;
        const float2* r1 = B.r1 + (size_t)(fb * P.pols + pol) * MY * N;
        // eight independent loads in flight per thread before their shared-memory stores
        for (int i0 = tid; i0 < R * N; i0 += 8 * nthr) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                const int row = idx >> logn, x = idx & (N - 1);
                const int q = q0 + row;
                v[u] = (idx < R * N && q < MY &&
                        DH_IN(P.status, (long long)(fb * P.pols + pol) * MY * N + (long long)q * N + x, B.r1_len, kSiteXpassR1))
                           ? r1[(size_t)q * N + x] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                if (idx < R * N) bufN[(idx & (N - 1)) * es + (idx >> logn)] = v[u];
            }
        }
        __syncthreads();
        fft_run<false>(bufN, N, P.rad_n, P.nrad_n, logr, es, P.tw_fwd_n, tid, nthr);
        for (int idx = tid; idx < R * M; idx += nthr) {
            const int row = idx & (R - 1), pp = idx >> logr;
            const int q = q0 + row;
            float2 v = make_float2(0.f, 0.f);
            if (q < MY) {
                if (pp >= pd.mask_lo[q] && pp <= pd.mask_hi[q]) {
                    int kx = (pd.klx + pp) % N;
                    if (kx < 0) kx += N;
                    v = cmul(cmul(bufN[P.pos_n[kx] * es + row], pd.phase_x[pp]), pd.phase_y[q]);
                }
                if (B.window && DH_IN(P.status, ((long long)pol * MY + q) * M + pp, (long long)P.pols * MY * M, kSiteXpassWindow))
                    B.window[((size_t)(f * P.pols + pol) * MY + q) * M + pp] = v;
            }
            bufM[P.pos_m[pp] * es + row] = v;
        }
        __syncthreads();
        fft_run<true>(bufM, M, P.rad_m, P.nrad_m, logr, es, P.tw_inv_m, tid, nthr);
        float2* g = B.g + (size_t)(fb * P.pols + pol) * MY * M;
        for (int idx = tid; idx < R * M; idx += nthr) {
            const int row = idx / M, i = idx - row * M;
            const int q = q0 + row;
            if (q < MY && DH_IN(P.status, (long long)(fb * P.pols + pol) * MY * M + (long long)q * M + i, B.g_len, kSiteXpassG))
                g[(size_t)q * M + i] = bufM[i * es + row];
        }
        __syncthreads();
    }
}

// k_xpass with the x transform's radix sequence fixed at compile time (the same plans as k_ypass_s) and its
// twiddles in shared memory; the M-point inverse keeps the runtime plan.  Same results as k_xpass.
template <int N, int R0, int R1, int R2, int LOGR, int MR0, int MR1, int MR2>
__global__ void __launch_bounds__(kThreads, (N == 256 && LOGR == 4 && MR0 != 0) ? 4 : 2) k_xpass_s(const __grid_constant__ Plan P, const __grid_constant__ Batch B) {
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int R = 1 << LOGR, es = R + 1, logr = LOGR, logn = (N == 128 ? 7 : N == 256 ? 8 : N == 512 ? 9 : 10);
    static_assert(R0 * R1 * R2 == N && (1 << logn) == N, "the radices multiply to N");
    const int M = P.m;
    float2* bufN = smem;
    float2* bufM = smem + (size_t)N * es;
    float2* twN = bufM + (size_t)M * es;
    float2* phx = twN + N;                       // [M] beam-centre phase along x
    float2* phy = phx + M;                       // [R] along y, this block's box rows
    int* mlo = reinterpret_cast<int*>(phy + R);  // [R] kept column range of this block's box rows
    int* mhi = mlo + R;
    for (int i = tid; i < N; i += kThreads) twN[i] = P.tw_fwd_n[i];
    const int pol = blockIdx.y;
    const PolDev& pd = P.pol[pol];
    const int q0 = blockIdx.x * R;
    for (int i = tid; i < M; i += kThreads) phx[i] = pd.phase_x[i];
    for (int i = tid; i < R; i += kThreads) {
        const bool in = q0 + i < M;
        phy[i] = in ? pd.phase_y[q0 + i] : make_float2(0.f, 0.f);
        mlo[i] = in ? pd.mask_lo[q0 + i] : 1;
        mhi[i] = in ? pd.mask_hi[q0 + i] : 0;
    }
    for (int fb = blockIdx.z; fb < B.count; fb += gridDim.z) {
        const int f = B.frame0 + fb;
        const float2* r1 = B.r1 + (size_t)(fb * P.pols + pol) * M * N;
        // eight independent loads in flight per thread before their shared-memory stores
        for (int i0 = tid; i0 < R * N; i0 += 8 * nthr) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                const int row = idx >> logn, x = idx & (N - 1);
                const int q = q0 + row;
                v[u] = (idx < R * N && q < M &&
                        DH_IN(P.status, (long long)(fb * P.pols + pol) * M * N + (long long)q * N + x, B.r1_len, kSiteXpassR1))
                           ? r1[(size_t)q * N + x] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                if (idx < R * N) bufN[(idx & (N - 1)) * es + (idx >> logn)] = v[u];
            }
        }
        __syncthreads();
        spass<R0, false, false, N, N, R, es, 1, kThreads>(bufN, twN, tid);
        __syncthreads();
        spass<R1, false, false, N, N / R0, R, es, 1, kThreads>(bufN, twN, tid);
        __syncthreads();
        if constexpr (R2 > 1) {
            spass<R2, false, false, N, N / (R0 * R1), R, es, 1, kThreads>(bufN, twN, tid);
            __syncthreads();
        }
        for (int idx = tid; idx < R * M; idx += nthr) {
            const int row = idx & (R - 1), pp = idx >> logr;
            const int q = q0 + row;
            float2 v = make_float2(0.f, 0.f);
            if (q < M) {
                if (pp >= mlo[row] && pp <= mhi[row]) {
                    int kx = (pd.klx + pp) % N;
                    if (kx < 0) kx += N;
                    v = cmul(cmul(bufN[dif_pos<R0, R1, R2>(kx) * es + row], phx[pp]), phy[row]);
                }
                if (B.window && DH_IN(P.status, ((long long)pol * M + q) * M + pp, (long long)P.pols * M * M, kSiteXpassWindow))
                    B.window[((size_t)(f * P.pols + pol) * M + q) * M + pp] = v;
            }
            bufM[plan_pos<MR0, MR1, MR2>(P.pos_m, pp) * es + row] = v;
        }
        __syncthreads();
        if constexpr (MR0 == 0)
            fft_run<true>(bufM, M, P.rad_m, P.nrad_m, logr, es, P.tw_inv_m, tid, nthr);
        else
            ifft_static<MR0, MR1, MR2, R, es, kThreads>(bufM, P.tw_inv_m, tid);
        float2* g = B.g + (size_t)(fb * P.pols + pol) * M * M;
        for (int idx = tid; idx < R * M; idx += nthr) {
            const int row = idx / M, i = idx - row * M;
            const int q = q0 + row;
            if (q < M && DH_IN(P.status, (long long)(fb * P.pols + pol) * M * M + (long long)q * M + i, B.g_len, kSiteXpassG))
                g[(size_t)q * M + i] = bufM[i * es + row];
        }
        __syncthreads();
    }
}

// Whether the host plan of M is the radix sequence (a, b, c) (c = 1: two radices).
static bool m_plan_is(const Plan& P, int a, int b, int c) {
    const int n = c > 1 ? 3 : 2;
    return P.nrad_m == n && P.rad_m[0] == a && P.rad_m[1] == b && (n == 2 || P.rad_m[2] == c);
}

template <int N, int R0, int R1, int R2, int LOGR>
static void launch_xs(const Plan& P, const Batch& B, int zf, cudaStream_t st) {
    constexpr int R = 1 << LOGR;
    dim3 g((P.m + R - 1) / R, P.pols, zf);
    const size_t sm = ((size_t)(N + P.m) * (R + 1) + N + P.m + 2 * R) * sizeof(float2);
    // the precision (256: M = 96) and large (512: M = 176) configurations also fix the inverse plan
    if constexpr (N == 256) {
        if (P.m == 96 && m_plan_is(P, 8, 4, 3)) {
            k_xpass_s<N, R0, R1, R2, LOGR, 8, 4, 3><<<g, kThreads, sm, st>>>(P, B);
            return;
        }
    }
    if constexpr (N == 512) {
        if (P.m == 176 && m_plan_is(P, 16, 11, 1)) {
            k_xpass_s<N, R0, R1, R2, LOGR, 16, 11, 1><<<g, kThreads, sm, st>>>(P, B);
            return;
        }
    }
    k_xpass_s<N, R0, R1, R2, LOGR, 0, 0, 0><<<g, kThreads, sm, st>>>(P, B);
}

static bool launch_xpass_static(const Plan& P, const Batch& B, int zf, cudaStream_t st) {
    auto is = [&](int a, int b, int c) {
        const int n = c > 1 ? 3 : 2;
        return P.nrad_n == n && P.rad_n[0] == a && P.rad_n[1] == b && (n == 2 || P.rad_n[2] == c);
    };
    switch (P.n) {
        case 128: if (!is(16, 8, 1)) return false; launch_xs<128, 16, 8, 1, 5>(P, B, zf, st); return true;
        case 256: if (!is(16, 16, 1)) return false; launch_xs<256, 16, 16, 1, 4>(P, B, zf, st); return true;
        case 512: if (!is(8, 8, 8)) return false; launch_xs<512, 8, 8, 8, 4>(P, B, zf, st); return true;
        case 1024: if (!is(16, 8, 8)) return false; launch_xs<1024, 16, 8, 8, 4>(P, B, zf, st); return true;
        default: return false;
    }
}

// MR0 MR1 MR2: the radix plan of M fixed at compile time, or MR0 = 0 for the runtime plan.  The compile-time
// plans fit 64 registers at M <= 128 (four blocks per SM) and 85 above (three); the runtime plan needs more
// and runs two.
template <int MR0, int MR1, int MR2>
__global__ void __launch_bounds__(kThreads, MR0 == 0 ? 2 : (MR0 * MR1 * MR2 <= 128 ? 4 : 3)) k_yinv(const __grid_constant__ Plan P, const __grid_constant__ Batch B) {
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    // M: field columns (x), MY: field rows (y; equal to M for square fields)
    const int M = P.m, MY = P.my, G = P.groups, modes = P.modes;
    float2* buf = smem;                          // [MY][kChunkI]
    float2* tp = smem + (size_t)MY * kChunkI;    // [G][kChunkI]
    // u_n(y'_j) for the rows j <= M/2, two modes of one parity per entry: block k holds n = 4 (k/2) + k%2 and
    // n + 2 (zero beyond G); [M/2 + 1][nbk]
    const int nbk = 2 * ((G + 3) / 4), hm = MY / 2;
    float2* u2 = tp + (size_t)std::max(G, 1) * kChunkI;
    float2* cxy = u2 + (size_t)(hm + 1) * nbk;   // [M + MY] correction phases along x, then y
    // compile-time plans: u_m(x'_i) dx' as [G][M + 1] (the odd pitch puts the modes of a warp on distinct banks)
    float* hgxs = reinterpret_cast<float*>(cxy + M + MY);
    const int pol = blockIdx.x;
    const PolDev& pd = P.pol[pol];
    for (int i = tid; i < M; i += nthr) cxy[i] = pd.corr_x[i];
    for (int i = tid; i < MY; i += nthr) cxy[M + i] = pd.corr_y[i];
    if constexpr (MR0 != 0) {
        for (int t = tid; t < G * M; t += nthr) {
            const int n = t / M, i = t - n * M;
            hgxs[n * (M + 1) + i] = pd.hg_x[t];
        }
    }
    for (int t = tid; t < (hm + 1) * nbk; t += nthr) {
        const int j = t / nbk, k = t - j * nbk;
        const int na = 4 * (k >> 1) + (k & 1), nb = na + 2;
        u2[t] = make_float2(na < G ? pd.hg_y[(size_t)na * MY + j] : 0.f, nb < G ? pd.hg_y[(size_t)nb * MY + j] : 0.f);
    }
    const bool g16 = ((uintptr_t)B.g & 15) == 0;   // 16-byte loads of the rows (M is even)
    for (int fb = blockIdx.y; fb < B.count; fb += gridDim.y) {
        const int f = B.frame0 + fb;
        const float2* g = B.g + (size_t)(fb * P.pols + pol) * MY * M;
        float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int i0 = 0; i0 < M; i0 += kChunkI) {
            if (g16) {
                // two columns per 16-byte load and store (M and the chunk start are even), eight loads in flight
                // per thread before their shared-memory stores
                for (int j0 = tid; j0 < MY * kChunkI / 2; j0 += 8 * nthr) {
                    float4 v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int idx = j0 + u * nthr;
                        const int q = idx / (kChunkI / 2), i = 2 * (idx % (kChunkI / 2));
                        v[u] = (idx < MY * kChunkI / 2 && i0 + i < M &&
                                DH_IN(P.status, (long long)(fb * P.pols + pol) * MY * M + (long long)q * M + i0 + i + 1, B.g_len,
                                      kSiteYinvG) &&
                                DH_ALIGNED16(P.status, g + (size_t)q * M + i0 + i))
                                   ? *reinterpret_cast<const float4*>(g + (size_t)q * M + i0 + i)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int idx = j0 + u * nthr;
                        if (idx < MY * kChunkI / 2)
                            *reinterpret_cast<float4*>(buf + plan_pos<MR0, MR1, MR2>(P.pos_my, idx / (kChunkI / 2)) * kChunkI +
                                                       2 * (idx % (kChunkI / 2))) = v[u];
                    }
                }
            } else {
                // eight independent loads in flight per thread before their shared-memory stores
                for (int j0 = tid; j0 < MY * kChunkI; j0 += 8 * nthr) {
                    float2 v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int idx = j0 + u * nthr;
                        const int q = idx >> 5, i = idx & (kChunkI - 1);
                        v[u] = (idx < MY * kChunkI && i0 + i < M &&
                                DH_IN(P.status, (long long)(fb * P.pols + pol) * MY * M + (long long)q * M + i0 + i, B.g_len, kSiteYinvG))
                                   ? g[(size_t)q * M + i0 + i] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int idx = j0 + u * nthr;
                        if (idx < MY * kChunkI) buf[plan_pos<MR0, MR1, MR2>(P.pos_my, idx >> 5) * kChunkI + (idx & (kChunkI - 1))] = v[u];
                    }
                }
            }
            __syncthreads();
            if constexpr (MR0 == 0)
                fft_run<true>(buf, MY, P.rad_my, P.nrad_my, 5, kChunkI, P.tw_inv_my, tid, nthr);
            else
                ifft_static<MR0, MR1, MR2, kChunkI, kChunkI, kThreads>(buf, P.tw_inv_my, tid);
            for (int idx = tid; idx < MY * kChunkI; idx += nthr) {
                const int j = idx >> 5, i = idx & (kChunkI - 1);
                if (i0 + i < M) {
                    const float2 e = cmul(cmul(buf[idx], cxy[M + j]), cxy[i0 + i]);
                    buf[idx] = e;
                    if (B.fields && DH_IN(P.status, ((long long)pol * MY + j) * M + i0 + i, (long long)P.pols * MY * M, kSiteYinvField))
                        B.fields[((size_t)(f * P.pols + pol) * MY + j) * M + i0 + i] = e;
                } else {
                    buf[idx] = make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
            if (G > 0) {
                // T[n][i] = sum_j u_n(y'_j) E[j][i].  Rows j and M - j carry u_n(y'_{M-j}) = (-1)^n u_n(y'_j), so
                // rows j = 1 .. M/2 - 1 become E_j + E_{M-j} (kept at j, for the even modes) and E_j - E_{M-j}
                // (at M - j, for the odd ones); rows 0 and M/2 have no partner and serve both parities.
                for (int idx = tid; idx < (hm - 1) * kChunkI; idx += nthr) {
                    const int j = 1 + (idx >> 5), i = idx & (kChunkI - 1);
                    const float2 a = buf[j * kChunkI + i], b = buf[(MY - j) * kChunkI + i];
                    buf[j * kChunkI + i] = cadd(a, b);
                    buf[(MY - j) * kChunkI + i] = csub(a, b);
                }
                __syncthreads();
                for (int idx = tid; idx < nbk * kChunkI; idx += nthr) {
                    const int k = idx >> 5, i = idx & (kChunkI - 1);   // k is the same across a warp
                    const bool odd = k & 1;
                    float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
                    {
                        const float2 w = u2[k], e = buf[i];
                        sa.x = fmaf(w.x, e.x, sa.x); sa.y = fmaf(w.x, e.y, sa.y);
                        sb.x = fmaf(w.y, e.x, sb.x); sb.y = fmaf(w.y, e.y, sb.y);
                    }
                    for (int j = 1; j < hm; ++j) {
                        const float2 w = u2[j * nbk + k];
                        const float2 e = buf[(odd ? MY - j : j) * kChunkI + i];
                        sa.x = fmaf(w.x, e.x, sa.x); sa.y = fmaf(w.x, e.y, sa.y);
                        sb.x = fmaf(w.y, e.x, sb.x); sb.y = fmaf(w.y, e.y, sb.y);
                    }
                    {
                        const float2 w = u2[hm * nbk + k], e = buf[hm * kChunkI + i];
                        sa.x = fmaf(w.x, e.x, sa.x); sa.y = fmaf(w.x, e.y, sa.y);
                        sb.x = fmaf(w.y, e.x, sb.x); sb.y = fmaf(w.y, e.y, sb.y);
                    }
                    const int na = 4 * (k >> 1) + (k & 1);
                    if (na < G) tp[na * kChunkI + i] = sa;
                    if (na + 2 < G) tp[(na + 2) * kChunkI + i] = sb;
                }
                __syncthreads();
                // c_mn += sum_i u_m(x'_i) T[n][i]
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    const int k = tid + kk * nthr;
                    if (k < modes) {
                        const float2* t = tp + P.mode_n[k] * kChunkI;
                        const int lim = min(kChunkI, M - i0);
                        if constexpr (MR0 != 0) {
                            const float* u = hgxs + (size_t)P.mode_m[k] * (M + 1) + i0;
                            for (int i = 0; i < lim; ++i) {
                                acc[kk].x = fmaf(u[i], t[i].x, acc[kk].x);
                                acc[kk].y = fmaf(u[i], t[i].y, acc[kk].y);
                            }
                        } else {
                            const float* u = pd.hg_x + (size_t)P.mode_m[k] * M + i0;
                            for (int i = 0; i < lim; ++i) {
                                const float w = __ldg(&u[i]);
                                acc[kk].x = fmaf(w, t[i].x, acc[kk].x);
                                acc[kk].y = fmaf(w, t[i].y, acc[kk].y);
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (B.coefs) {
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const int k = tid + kk * nthr;
                if (k < modes && DH_IN(P.status, (long long)pol * modes + k, (long long)P.pols * modes, kSiteYinvCoef))
                    B.coefs[(size_t)(f * P.pols + pol) * modes + k] = acc[kk];
            }
        }
    }
}

static int ilog2(int v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

cudaError_t split_init() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_ypass<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_ypass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_xpass, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) return e;
#define DH_YS_ATTR(T, N, A, B2, C2, L)                                                                            \
    if ((e = cudaFuncSetAttribute(k_ypass_s<T, N, A, B2, C2, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) \
        return e;
    DH_YS_ATTR(uint16_t, 128, 16, 8, 1, 5) DH_YS_ATTR(float, 128, 16, 8, 1, 5)
    DH_YS_ATTR(uint16_t, 256, 16, 16, 1, 4) DH_YS_ATTR(float, 256, 16, 16, 1, 4)
    DH_YS_ATTR(uint16_t, 512, 8, 8, 8, 4) DH_YS_ATTR(float, 512, 8, 8, 8, 4)
    DH_YS_ATTR(uint16_t, 1024, 16, 8, 8, 3) DH_YS_ATTR(float, 1024, 16, 8, 8, 3)
#undef DH_YS_ATTR
#define DH_XS_ATTR(...)                                                                                         \
    if ((e = cudaFuncSetAttribute(k_xpass_s<__VA_ARGS__>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) \
        return e;
    DH_XS_ATTR(128, 16, 8, 1, 5, 0, 0, 0) DH_XS_ATTR(256, 16, 16, 1, 4, 0, 0, 0)
    DH_XS_ATTR(512, 8, 8, 8, 4, 0, 0, 0) DH_XS_ATTR(1024, 16, 8, 8, 4, 0, 0, 0)
    DH_XS_ATTR(256, 16, 16, 1, 4, 8, 4, 3) DH_XS_ATTR(512, 8, 8, 8, 4, 16, 11, 1)
#undef DH_XS_ATTR
    if ((e = cudaFuncSetAttribute(k_yinv<8, 4, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_yinv<16, 11, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_yinv<0, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem))) return e;
    return cudaSuccess;
}

cudaError_t launch_split(const Plan& P, const Batch& B, cudaStream_t st, StageTimer* tm) {
    cudaError_t e = launch_forward(P, B, st, tm);
    if (e != cudaSuccess) return e;
    return launch_last(P, B, st, tm);
}

// The compile-time specialisations serve square windows and fields only.
static bool square(const Plan& P) { return P.ny == P.n && P.my == P.m; }

cudaError_t launch_forward(const Plan& P, const Batch& B, cudaStream_t st, StageTimer* tm) {
    const int N = P.n, M = P.m;
    const int zf = std::min(B.count, 65535);
    // k_ypass: C packed column pairs per block, N_y x C complex in shared memory
    int logc = (std::max(N, P.ny) >= 1024) ? 4 : 5;
    logc = std::min(logc, ilog2(N / 2));
    const int C = 1 << logc;
    dim3 g1((N / 2) / C, P.pols, zf);
    const size_t sm1 = (size_t)P.ny * C * sizeof(float2);
    if (tm) tm->start(st);
    const bool done = square(P) && (B.dtype == DH_DTYPE_U16 ? launch_ypass_static<uint16_t>(P, B, zf, st)
                                                            : launch_ypass_static<float>(P, B, zf, st));
    if (!done) {
        if (B.dtype == DH_DTYPE_U16)
            k_ypass<uint16_t><<<g1, kThreads, sm1, st>>>(P, B, logc);
        else
            k_ypass<float><<<g1, kThreads, sm1, st>>>(P, B, logc);
    }
    if (tm) tm->stop(st, "k_ypass");
    // k_xpass: R box rows per block
    const int logr = (N >= 512) ? 4 : 5;
    const int R = 1 << logr;
    dim3 g2((P.my + R - 1) / R, P.pols, zf);
    const size_t sm2 = (size_t)(N + M) * (R + 1) * sizeof(float2);
    if (tm) tm->start(st);
    if (!(square(P) && launch_xpass_static(P, B, zf, st))) k_xpass<<<g2, kThreads, sm2, st>>>(P, B, logr, ilog2(N));
    if (tm) tm->stop(st, "k_xpass");
    return cudaGetLastError();
}

cudaError_t launch_last(const Plan& P, const Batch& B, cudaStream_t st, StageTimer* tm) {
    // k_yinv (or its tensor-core variant): one block per window
    const int zf = std::min(B.count, 65535);
    dim3 g3(P.pols, zf);
    const size_t sm3 = ((size_t)(P.my + std::max(P.groups, 1)) * kChunkI +
                        (size_t)(P.my / 2 + 1) * 2 * ((P.groups + 3) / 4) + (size_t)P.m + (size_t)P.my) * sizeof(float2);
    if (coef_tc_supported(P, B)) {
        // no field requested: the y transform and the y overlap as one tensor-core contraction
        if (tm) tm->start(st);
        cudaError_t e = launch_coef_tc(P, B, st);
        if (tm) tm->stop(st, "k_coef_tc");
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (tc_supported(P)) {
        if (tm) tm->start(st);
        cudaError_t e = launch_yinv_tc(P, B, st);
        if (tm) tm->stop(st, "k_yinv_tc");
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const size_t sm3s = sm3 + (size_t)P.groups * (P.m + 1) * sizeof(float);   // with the staged x table
    if (tm) tm->start(st);
    if (square(P) && P.m == 96 && m_plan_is(P, 8, 4, 3))
        k_yinv<8, 4, 3><<<g3, kThreads, sm3s, st>>>(P, B);
    else if (square(P) && P.m == 176 && m_plan_is(P, 16, 11, 1))
        k_yinv<16, 11, 1><<<g3, kThreads, sm3s, st>>>(P, B);
    else
        k_yinv<0, 0, 0><<<g3, kThreads, sm3, st>>>(P, B);
    if (tm) tm->stop(st, "k_yinv");
    return cudaGetLastError();
}

cudaError_t launch_ypass(const Plan& P, const Batch& B, cudaStream_t st, StageTimer* tm) {
    const int N = P.n;
    const int zf = std::min(B.count, 65535);
    int logc = (std::max(N, P.ny) >= 1024) ? 4 : 5;
    logc = std::min(logc, ilog2(N / 2));
    const int C = 1 << logc;
    dim3 g1((N / 2) / C, P.pols, zf);
    const size_t sm1 = (size_t)P.ny * C * sizeof(float2);
    if (tm) tm->start(st);
    const bool done = square(P) && (B.dtype == DH_DTYPE_U16 ? launch_ypass_static<uint16_t>(P, B, zf, st)
                                                            : launch_ypass_static<float>(P, B, zf, st));
    if (!done) {
        if (B.dtype == DH_DTYPE_U16)
            k_ypass<uint16_t><<<g1, kThreads, sm1, st>>>(P, B, logc);
        else
            k_ypass<float><<<g1, kThreads, sm1, st>>>(P, B, logc);
    }
    if (tm) tm->stop(st, "k_ypass");
    return cudaGetLastError();
}

}  // namespace dhk
