// Split-BF16 tensor-core variant of the generic path's last kernel (pipeline step 2 along y, tilt and defocus
// removal, and the HG modal decomposition of step 3).
//
// One block per (frame, polarisation) window, 64 field columns per chunk (48 at M = 96).  After the y inverse
// transform and the correction, the chunk's field E[j][i] (FP32) is split into bfloat16 hi + lo parts and
// written as the A operand of a 128 x NP x M contraction (rows: real parts of the chunk's columns at i,
// imaginary parts at 64 + i; K: the field row j), whose B operand holds u_n(y'_j) dy' as bfloat16 hi + lo
// (host-built, FP64 -> bf16).  One elected thread
// issues the three products hi*hi + hi*lo + lo*hi per 16-wide K step with tcgen05.mma (kind::f16, FP32
// accumulation in tensor memory) and commits them to an mbarrier; the four warps of the first warpgroup read
// the 128 x NP accumulator back with tcgen05.ld into shared memory, and one thread per mode finishes the
// second (x) contraction on CUDA cores in a fixed order.  The lo*lo product is below FP32 rounding of the result and is dropped.
//
// Operands use the no-swizzle K-major canonical layout of umma.cuh.
// Every wait on the mbarrier is bounded; on expiry the window's coefficients are written as NaN, the plan's
// status word records it, and the block releases its tensor memory before it returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"
#include "kernels.cuh"
#include "sync.cuh"
#include "umma.cuh"

namespace dhk {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcCols = 64;          // field columns per chunk (A rows = 2 * 64 = 128)
constexpr int kTcMaxM = 192;         // shared-memory bound of this kernel
constexpr int kTmemCols = 32;
constexpr long kWaitLimit = 1L << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return smem_u32(p); }

__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity) { return bounded_mbar_wait(mbar, parity, kWaitLimit); }

constexpr int kTsPitch = 129;        // accumulator rows per mode row in shared memory (padded)

struct TcLayout {
    size_t buf, a, b, c, h, bytes;
};

// buf holds the field chunk, then (after the A operand is built from it) the accumulator T[n][r]
// hg_rows: modes of the staged x table u_m(x'_i) dx' ([hg_rows][M + 1] floats; 0 = read from global memory)
__host__ __device__ inline TcLayout tc_layout(int M, int NP, int cols, int hg_rows) {
    TcLayout L;
    L.buf = 0;                                             // float2 [M][cols]  /  float [NP][129]
    size_t bufb = (size_t)M * cols * 8;
    const size_t tsb = (size_t)NP * kTsPitch * 4;
    if (tsb > bufb) bufb = tsb;
    L.a = L.buf + ((bufb + 1023) & ~(size_t)1023);         // bf16 [2][128][M]
    L.b = L.a + (size_t)2 * 128 * M * 2;                    // bf16 [2][NP][M]
    L.c = L.b + (size_t)2 * NP * M * 2;                     // float2 [2][M]: correction along x, then y
    L.h = L.c + (size_t)2 * M * 8;
    L.bytes = L.h + (size_t)hg_rows * (M + 1) * 4;
    L.bytes = (L.bytes + 1023) & ~(size_t)1023;
    return L;
}

}  // namespace

// R0 R1 R2: the host plan's radices of M fixed at compile time (inverse passes run last radix first), or
// R0 = 0 for the runtime plan.  COLS: field columns per chunk (A rows: real parts at i, imaginary parts at
// 64 + i; with fewer than 64 columns the other rows stay zero), 48 at M = 96 so that no chunk is padded.  NT:
// threads per block; 512 at M = 176, whose shared memory allows one block per SM.
template <int R0, int R1, int R2, int COLS = kTcCols, int NT = kTcThreads>
__global__ void __launch_bounds__(NT, NT == kTcThreads ? 2 : 1) k_yinv_tc(const __grid_constant__ Plan P, const __grid_constant__ Batch B) {
    static_assert(COLS % 16 == 0 && COLS <= kTcCols && (R0 != 0 || COLS == kTcCols), "chunk width");
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = P.m, modes = P.modes, NP = P.tc_np;
    // compile-time plans stage u_m(x'_i) dx' as [G][M + 1] (odd pitch: the modes of a warp on distinct banks)
    const TcLayout L = tc_layout(M, NP, COLS, R0 != 0 ? P.groups : 0);
    float2* buf = reinterpret_cast<float2*>(sm + L.buf);
    float* Ts = reinterpret_cast<float*>(sm + L.buf);
    __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(sm + L.a);
    __nv_bfloat16* Bm = reinterpret_cast<__nv_bfloat16*>(sm + L.b);
    float2* cxy = reinterpret_cast<float2*>(sm + L.c);
    float* hgxs = reinterpret_cast<float*>(sm + L.h);
    const int pol = blockIdx.x;
    const PolDev& pd = P.pol[pol];
    for (int i = tid; i < M; i += NT) {
        cxy[i] = pd.corr_x[i];
        cxy[M + i] = pd.corr_y[i];
    }
    if constexpr (R0 != 0) {
        for (int t = tid; t < P.groups * M; t += NT) {
            const int n = t / M, i = t - n * M;
            hgxs[n * (M + 1) + i] = pd.hg_x[t];
        }
    }

    // B operand (static per polarisation): 16-byte copies
    {
        const uint4* src = reinterpret_cast<const uint4*>(pd.hgy_tc);
        uint4* dst = reinterpret_cast<uint4*>(Bm);
        const int n16 = (2 * NP * M * 2) / 16;
        for (int i = tid; i < n16; i += NT) dst[i] = __ldg(&src[i]);
    }
    if constexpr (COLS < kTcCols) {
        // the A rows no column maps to (COLS .. 63 and 64 + COLS .. 127) stay zero in both planes
        constexpr int ZR = kTcCols - COLS;
        for (int t = tid; t < 2 * 2 * ZR * M; t += NT) {
            const int plane = t / (2 * ZR * M), rem = t - plane * 2 * ZR * M;
            const int rr = rem / M, k = rem - rr * M;
            const int row = rr < ZR ? COLS + rr : kTcCols + COLS + (rr - ZR);
            A[(size_t)plane * 128 * M + umma_off(row, k, M)] = __float2bfloat16_rn(0.f);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (warp == 0) {
        tmem_alloc(smem_addr(&tmem_slot), kTmemCols);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mbar_a = smem_addr(&mbar);
    const uint32_t a_hi = smem_addr(A), a_lo = a_hi + 128 * M * 2;
    const uint32_t b_hi = smem_addr(Bm), b_lo = b_hi + NP * M * 2;
    const uint32_t lbo = 128, sbo = 16 * M;
    const uint32_t idesc = umma_idesc_bf16(128, NP);
    uint32_t phase = 0;
    bool ok = true;

    const bool g16 = ((uintptr_t)B.g & 15) == 0;   // 16-byte loads of the rows (M is even)
    for (int fb = blockIdx.y; fb < B.count; fb += gridDim.y) {
        const int f = B.frame0 + fb;
        const float2* g = B.g + (size_t)(fb * P.pols + pol) * M * M;
        float2 acc = make_float2(0.f, 0.f);   // mode tid (modes <= 256)
        for (int i0 = 0; i0 < M; i0 += COLS) {
            // loads in flight per thread: eight for a small fixed plan, four for a larger one (one block per SM),
            // one for the runtime plan
            constexpr int LB = R0 == 0 ? 1 : (R0 * R1 * R2 <= 128 ? 8 : 4);
            if (g16) {
                // two columns per 16-byte load and store (M, COLS and the chunk start are even)
                for (int j0 = tid; j0 < M * COLS / 2; j0 += LB * NT) {
                    float4 v[LB];
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                        const int idx = j0 + u * NT;
                        const int q = idx / (COLS / 2), i = 2 * (idx % (COLS / 2));
                        v[u] = (idx < M * COLS / 2 && i0 + i < M &&
                                DH_IN(P.status, (long long)(fb * P.pols + pol) * M * M + (long long)q * M + i0 + i + 1, B.g_len,
                                      kSiteYinvG) &&
                                DH_ALIGNED16(P.status, g + (size_t)q * M + i0 + i))
                                   ? *reinterpret_cast<const float4*>(g + (size_t)q * M + i0 + i)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                        const int idx = j0 + u * NT;
                        if (idx < M * COLS / 2)
                            *reinterpret_cast<float4*>(buf + plan_pos<R0, R1, R2>(P.pos_m, idx / (COLS / 2)) * COLS +
                                                       2 * (idx % (COLS / 2))) = v[u];
                    }
                }
            } else {
                for (int j0 = tid; j0 < M * COLS; j0 += LB * NT) {
                    float2 v[LB];
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                        const int idx = j0 + u * NT;
                        const int q = idx / COLS, i = idx % COLS;
                        v[u] = (idx < M * COLS && i0 + i < M &&
                                DH_IN(P.status, (long long)(fb * P.pols + pol) * M * M + (long long)q * M + i0 + i, B.g_len, kSiteYinvG))
                                   ? g[(size_t)q * M + i0 + i] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                        const int idx = j0 + u * NT;
                        if (idx < M * COLS) buf[plan_pos<R0, R1, R2>(P.pos_m, idx / COLS) * COLS + idx % COLS] = v[u];
                    }
                }
            }
            __syncthreads();
            if constexpr (R0 == 0) {
                fft_run<true>(buf, M, P.rad_m, P.nrad_m, 6, kTcCols, P.tw_inv_m, tid, NT);
            } else {
                ifft_static<R0, R1, R2, COLS, COLS, NT>(buf, P.tw_inv_m, tid);
            }
            for (int idx = tid; idx < M * COLS; idx += NT) {
                const int j = idx / COLS, i = idx % COLS;
                if (i0 + i < M) {
                    const float2 e = cmul(cmul(buf[idx], cxy[M + j]), cxy[i0 + i]);
                    buf[idx] = e;
                    if (B.fields && DH_IN(P.status, ((long long)pol * M + j) * M + i0 + i, (long long)P.pols * M * M, kSiteYinvField))
                        B.fields[((size_t)(f * P.pols + pol) * M + j) * M + i0 + i] = e;
                } else {
                    buf[idx] = make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
            // A operand: rows r = i (real part) and 64 + i (imaginary part), K = j; 8 consecutive j per task
            for (int t = tid; t < COLS * (M / 8); t += NT) {
                const int i = t % COLS, jb = t / COLS;
                __align__(16) __nv_bfloat16 hr[8], hi_[8], lr[8], li[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float2 e = buf[(8 * jb + c) * COLS + i];
                    const __nv_bfloat16 xr = __float2bfloat16_rn(e.x), xi = __float2bfloat16_rn(e.y);
                    hr[c] = xr;
                    hi_[c] = xi;
                    lr[c] = __float2bfloat16_rn(e.x - __bfloat162float(xr));
                    li[c] = __float2bfloat16_rn(e.y - __bfloat162float(xi));
                }
                const int rr = i, ri = 64 + i;
                const size_t o_r = ((size_t)(rr >> 3) * (M >> 3) + jb) * 64 + (rr & 7) * 8;
                const size_t o_i = ((size_t)(ri >> 3) * (M >> 3) + jb) * 64 + (ri & 7) * 8;
                *reinterpret_cast<uint4*>(A + o_r) = *reinterpret_cast<const uint4*>(hr);
                *reinterpret_cast<uint4*>(A + o_i) = *reinterpret_cast<const uint4*>(hi_);
                *reinterpret_cast<uint4*>(A + 128 * M + o_r) = *reinterpret_cast<const uint4*>(lr);
                *reinterpret_cast<uint4*>(A + 128 * M + o_i) = *reinterpret_cast<const uint4*>(li);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (tid == 0 && ok) {
                for (int ks = 0; ks < M / 16; ++ks) {
                    const uint32_t ko = ks * 256;
                    umma_bf16(tmem, umma_desc(a_hi + ko, lbo, sbo), umma_desc(b_hi + ko, lbo, sbo), idesc, ks > 0);
                    umma_bf16(tmem, umma_desc(a_hi + ko, lbo, sbo), umma_desc(b_lo + ko, lbo, sbo), idesc, 1);
                    umma_bf16(tmem, umma_desc(a_lo + ko, lbo, sbo), umma_desc(b_hi + ko, lbo, sbo), idesc, 1);
                }
                umma_commit(mbar_a);
            }
            const bool done = ok && wait_parity(mbar_a, phase);
            phase ^= 1u;
            if (ok && !done && tid == 0 && P.status) atomicOr(P.status, 2);
            ok = ok && done;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (warp < 4) {
                // accumulator row r = 32 warp + lane (column i = r mod 64; real part for r < 64, imaginary
                // part above) to shared memory, T[n][r] with a padded pitch
                float T[16];
                const int r = 32 * warp + lane;
                for (int c0 = 0; c0 < NP; c0 += 16) {
                    if (ok) tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, T);
#pragma unroll
                    for (int n = 0; n < 16; ++n) Ts[(c0 + n) * kTsPitch + r] = ok ? T[n] : 0.f;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            // c_mn += sum_i u_m(x'_i) T[n][i] over this chunk's columns, one mode per thread, fixed order
            if (tid < modes) {
                const int m = P.mode_m[tid], n = P.mode_n[tid];
                const float* tr = Ts + n * kTsPitch;
                const int lim = min(COLS, M - i0);
                float sr = 0.f, si = 0.f;
                if constexpr (R0 != 0) {
                    const float* u = hgxs + (size_t)m * (M + 1) + i0;
                    for (int i = 0; i < lim; ++i) {
                        sr = fmaf(u[i], tr[i], sr);
                        si = fmaf(u[i], tr[64 + i], si);
                    }
                } else {
                    const float* u = pd.hg_x + (size_t)m * M + i0;
                    for (int i = 0; i < lim; ++i) {
                        const float w = __ldg(&u[i]);
                        sr = fmaf(w, tr[i], sr);
                        si = fmaf(w, tr[64 + i], si);
                    }
                }
                acc.x += sr;
                acc.y += si;
            }
            __syncthreads();
        }
        if (B.coefs && tid < modes && DH_IN(P.status, (long long)pol * modes + tid, (long long)P.pols * modes, kSiteYinvCoef))
            B.coefs[(size_t)(f * P.pols + pol) * modes + tid] = ok ? acc : make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) tmem_free(tmem, kTmemCols);
}

// A plan reaches the tensor-core kernel only with a B operand built for it: tc_np > 0 rows and a bf16
// hi/lo table for every polarisation (an N = 0 instruction descriptor or a missing table is never launched).
bool tc_supported(const Plan& P) {
    if (!(P.precision == DH_PRECISION_SPLIT_BF16 && P.ny == P.n && P.my == P.m && P.groups > 0 && P.modes <= kTcThreads && P.m <= kTcMaxM &&
          P.m % 16 == 0 && P.tc_np > 0 && P.tc_np % 16 == 0 && P.tc_np <= kTmemCols))
        return false;
    for (int p = 0; p < P.pols; ++p)
        if (!P.pol[p].hgy_tc) return false;
    return true;
}

cudaError_t tc_init() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_yinv_tc<0, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 1024)))
        return e;
    if ((e = cudaFuncSetAttribute(k_yinv_tc<8, 4, 3, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 1024)))
        return e;
    return cudaFuncSetAttribute(k_yinv_tc<16, 11, 1, kTcCols, 2 * kTcThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024 - 1024);
}

cudaError_t launch_yinv_tc(const Plan& P, const Batch& B, cudaStream_t st) {
    const TcLayout L = tc_layout(P.m, P.tc_np, kTcCols, 0);
    dim3 grid(P.pols, B.count < 65535 ? B.count : 65535);
    // the field sizes of the precision (96 = 8 4 3) and large (176 = 16 11) configurations run with their
    // radix plan fixed at compile time
    auto plan_is = [&](int a, int b, int c) {
        const int n = c > 1 ? 3 : 2;
        return P.nrad_m == n && P.rad_m[0] == a && P.rad_m[1] == b && (n == 2 || P.rad_m[2] == c);
    };
    if (P.m == 96 && plan_is(8, 4, 3))   // two chunks of 48 columns
        k_yinv_tc<8, 4, 3, 48><<<grid, kTcThreads, tc_layout(P.m, P.tc_np, 48, P.groups).bytes, st>>>(P, B);
    else if (P.m == 176 && plan_is(16, 11, 1))
        k_yinv_tc<16, 11, 1, kTcCols, 2 * kTcThreads><<<grid, 2 * kTcThreads, tc_layout(P.m, P.tc_np, kTcCols, P.groups).bytes, st>>>(P, B);
    else
        k_yinv_tc<0, 0, 0><<<grid, kTcThreads, L.bytes, st>>>(P, B);
    return cudaGetLastError();
}

}  // namespace dhk
