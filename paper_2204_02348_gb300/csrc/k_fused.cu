// Fused single-kernel path for 128 x 128 windows (field sizes 32, 48 and 64): one thread block reconstructs
// one (frame, polarisation) window entirely in shared memory, persistent over windows, two blocks per SM.
//
// Per window (the guide's pipeline steps 1-3 and digHoloProcessRemoveTilt):
//   y pass   real columns x and x + 64 packed as one complex column; radix-16 DIF pass from the window staged
//            in shared memory by a tensor copy, radix-8 pass fused with the separation of the two real spectra
//            (Z(k), conj Z(-k)) and the selection of the M box rows;
//   x pass   radix-16 then radix-8 DIF along x on the M box rows, the second pass fused with the box-column
//            selection, the circular mask and the beam-centre phase;
//   inverse  M-point inverse transform along x (DIT, digit-reversed in / natural out) and along y (DIF,
//            natural in / digit-reversed out), in place;
//   epilogue residual tilt and defocus removal in registers inside the last y pass, field write (coalesced
//            along x), and the separable HG contraction: partial sums over y per thread group, then the modes
//            spread over the warps with fixed shuffle trees (deterministic, no atomics).
// Shared memory: r1[N][M+1] box rows (x-major, padded pitch) and one union region used in turn as the y-pass
// tile, the M x (M+1) window / field, and the overlap partials; twiddles and the digit-reversal table.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "fft.cuh"
#include "runtime.hpp"
#include "sync.cuh"

namespace dhk {

constexpr int kFN = 128;          // window size of this path
constexpr int kFThreads = 512;
constexpr int kFGMax = 16;        // largest group count of this path
constexpr int kFRows = 128;       // staged window rows
constexpr long kFWaitLimit = 1L << 24;

struct FusedArgs {
    const void* src;              // frames [B][H][W]
    int frame0, count;
    int xo[DH_MAX_POLS];          // window origin minus the 16-byte-aligned staging origin, per polarisation
    int x0[DH_MAX_POLS];          // staging origin (16-byte aligned element index), per polarisation
    float2* fields;               // nullable [B][pol][M][M]
    float2* coefs;                // nullable [B][pol][modes]
};

template <typename T>
struct Staging {
    static constexpr int ALIGN = 16 / (int)sizeof(T);     // elements per 16 bytes
    static constexpr int W = kFN + ALIGN;                  // staged row width (window plus alignment slack)
    static constexpr int BYTES = kFRows * W * (int)sizeof(T);
};

template <int M, typename T>
struct FusedLayout {
    static constexpr int PITCH = M + 1;
    static constexpr int R1 = kFN * PITCH;
    static constexpr int YT = kFN * (kFN / 2);                 // y tile: 128 rows x 64 column pairs
    static constexpr int WB = M * PITCH;
    static constexpr int UN = YT > WB ? YT : WB;
    static_assert(UN >= kFGMax * M, "the union region holds T");
    static constexpr int F2 = R1 + UN + kFN + M + 4 * M;
    static constexpr int FL = 2 * kFGMax * M;
    static constexpr int IN = 3 * M + 2 * (kFGMax * (kFGMax + 1) / 2);
    static constexpr size_t STG = (size_t)Staging<T>::BYTES;   // first, 1024-byte aligned
    static constexpr size_t bytes = STG + (size_t)F2 * sizeof(float2) + (size_t)FL * sizeof(float) + (size_t)IN * sizeof(int);
};

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) { return bounded_mbar_wait(mbar, parity, kFWaitLimit); }

// One thread: expect the window's bytes on the mbarrier and start the tensor copy of frame f.
__device__ __forceinline__ void stage_window(const CUtensorMap* tmap, uint32_t dst, uint32_t mbar, int x0, int y0, int f,
                                             int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0), "r"(f), "r"(mbar)
        : "memory");
}

// Columns x and x + N/2 of a staged row, packed as one complex value.
template <typename T>
__device__ __forceinline__ float2 staged_pair(const T* row, int x) {
    return make_float2((float)row[x], (float)row[x + kFN / 2]);
}

// Write the separated spectra of columns x and x + N/2 at frequency k (if k is a box row).
__device__ __forceinline__ void emit_pair(float2* r1, int pitch, int M, int kly, int x, int k, float2 zk, float2 zm) {
    const int q = (k - kly) & (kFN - 1);
    if (q < M) {
        r1[x * pitch + q] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        r1[(x + kFN / 2) * pitch + q] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
}

template <int M, int MR0, int MR1, typename T>
__global__ void __launch_bounds__(kFThreads, 1) k_fused128(const __grid_constant__ Plan P, const __grid_constant__ FusedArgs A,
                                                           const __grid_constant__ CUtensorMap tmap) {
    using L = FusedLayout<M, T>;
    using S = Staging<T>;
    constexpr int N = kFN, PITCH = L::PITCH, NT = kFThreads;
    static_assert(M == MR0 * MR1, "field size = product of the two radices");
    static_assert(L::R1 >= (M / MR1) * kFGMax * M, "r1 holds the overlap partial sums");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int abort_flag;
    T* stg = reinterpret_cast<T*>(smem_raw);
    float2* r1 = reinterpret_cast<float2*>(smem_raw + L::STG);
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
        posM[i] = (i % MR0) * MR1 + i / MR0;   // position of index i after DIF passes of radix MR0 then MR1
        phx[i] = pd.phase_x[i];
        phy[i] = pd.phase_y[i];
        cx[i] = pd.corr_x[i];
        cy[i] = pd.corr_y[i];
        mlo[i] = pd.mask_lo[i];
        mhi[i] = pd.mask_hi[i];
    }
    for (int i = tid; i < G * M; i += NT) hgx[i] = pd.hg_x[i];
    // u_n(y'_j) stored [j][n] (n fastest, kFGMax wide) so the y contraction reads four groups per load
    for (int i = tid; i < kFGMax * M; i += NT) {
        const int j = i / kFGMax, n = i - j * kFGMax;
        hgy[i] = n < G ? pd.hg_y[n * M + j] : 0.f;
    }
    for (int i = tid; i < modes; i += NT) {
        mdm[i] = P.mode_m[i];
        mdn[i] = P.mode_n[i];
    }
    const uint32_t mb = smem_u32(&mbar), dst = smem_u32(stg);
    const int fstride = gridDim.x / P.pols;
    int b = blockIdx.x / P.pols;
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (b < A.count) stage_window(&tmap, dst, mb, A.x0[pol], pd.oy, A.frame0 + b, S::BYTES);
    }
    __syncthreads();
    const int xo = A.xo[pol];
    uint32_t parity = 0;
    for (; b < A.count; b += fstride) {
        const int f = A.frame0 + b;
        const bool ok = mbar_wait(mb, parity);
        parity ^= 1u;
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) {
            if (tid == 0 && P.status) atomicOr(P.status, 1);
            break;
        }

        // ---------------------------------------------------------------- y pass on 64 column pairs
        {
            const int c = tid & 63, j = tid >> 6;
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = staged_pair<T>(stg + (j + 8 * r) * S::W, xo + c);
            dft16<false>(v);
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twN[j * r]);
#pragma unroll
            for (int r = 0; r < 16; ++r) un[(j + 8 * r) * 64 + c] = v[r];
        }
        // the staged window has been read: order those reads before the next tensor copy into the buffer
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0 && b + fstride < A.count) stage_window(&tmap, dst, mb, A.x0[pol], pd.oy, f + fstride, S::BYTES);
        {
            const int c = tid & 63, u = tid >> 6;
            const int d1 = u, d2 = (u == 0) ? 8 : 16 - u;
            float2 z1[8], z2[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                z1[r] = un[(8 * d1 + r) * 64 + c];
                z2[r] = un[(8 * d2 + r) * 64 + c];
            }
            dft8<false>(z1);
            dft8<false>(z2);
            const int x = c;
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

        // ---------------------------------------------------------------- last y pass, correction, field, y overlap
        // The last DIF pass (span MR1, no twiddles) leaves output j = blk + MR0 r at position blk MR1 + r of
        // column i; it is corrected in registers, written to the field (coalesced along i) and contracted with
        // u_n(y'_j) into the partial sums part[blk][n][i] over the thread's MR1 rows.
        constexpr int NBLK = M / MR1;
        float2* part = r1;                         // [NBLK][G][M]
        float2* tsum = un;                         // [G][M]
        const bool ov = A.coefs && G > 0;
        {
            float2* fld = A.fields ? A.fields + (size_t)(f * P.pols + pol) * M * M : nullptr;
            for (int t = tid; t < M * NBLK; t += NT) {
                const int i = t % M, blk = t / M;
                float2 v[MR1];
#pragma unroll
                for (int r = 0; r < MR1; ++r) v[r] = un[i * PITCH + blk * MR1 + r];
                dft<MR1, true>(v, twM, M / MR1);
                const float2 ci = cx[i];
#pragma unroll
                for (int r = 0; r < MR1; ++r) {
                    const int j = blk + MR0 * r;
                    v[r] = cmul(cmul(v[r], ci), cy[j]);
                    if (fld) fld[j * M + i] = v[r];
                }
                if (ov) {
#pragma unroll
                    for (int n4 = 0; n4 < kFGMax; n4 += 4) {
                        if (n4 < G) {
                            float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                           make_float2(0.f, 0.f)};
#pragma unroll
                            for (int r = 0; r < MR1; ++r) {
                                const float4 u = *reinterpret_cast<const float4*>(hgy + (blk + MR0 * r) * kFGMax + n4);
                                a[0].x = fmaf(u.x, v[r].x, a[0].x);
                                a[0].y = fmaf(u.x, v[r].y, a[0].y);
                                a[1].x = fmaf(u.y, v[r].x, a[1].x);
                                a[1].y = fmaf(u.y, v[r].y, a[1].y);
                                a[2].x = fmaf(u.z, v[r].x, a[2].x);
                                a[2].y = fmaf(u.z, v[r].y, a[2].y);
                                a[3].x = fmaf(u.w, v[r].x, a[3].x);
                                a[3].y = fmaf(u.w, v[r].y, a[3].y);
                            }
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if (n4 + c < G) part[(blk * G + n4 + c) * M + i] = a[c];
                        }
                    }
                }
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- HG overlap, x contraction
        if (ov) {
            // T[n][i]: the partial sums of the NBLK row groups added in a fixed order
            for (int t = tid; t < G * M; t += NT) {
                float2 v = part[t];
#pragma unroll
                for (int q = 1; q < NBLK; ++q) {
                    const float2 w = part[q * G * M + t];
                    v.x += w.x;
                    v.y += w.y;
                }
                tsum[t] = v;
            }
            __syncthreads();
            // c_mn = sum_i u_m(x'_i) T[n][i]: modes spread over the warps in groups of KW; independent
            // products first, then interleaved shuffle trees (fixed order)
            const int warp = tid >> 5, lane = tid & 31;
            constexpr int NW = NT / 32, KW = 4;
            float2* cf = A.coefs + (size_t)(f * P.pols + pol) * modes;
            for (int k0 = 0; warp + k0 * NW < modes; k0 += KW) {
                float2 sacc[KW];
#pragma unroll
                for (int kk = 0; kk < KW; ++kk) {
                    sacc[kk] = make_float2(0.f, 0.f);
                    const int k = warp + (k0 + kk) * NW;
                    if (k < modes) {
                        const float* um = hgx + mdm[k] * M;
                        const float2* tn = tsum + mdn[k] * M;
#pragma unroll
                        for (int i = lane; i < M; i += 32) {
                            const float u = um[i];
                            const float2 t = tn[i];
                            sacc[kk].x = fmaf(u, t.x, sacc[kk].x);
                            sacc[kk].y = fmaf(u, t.y, sacc[kk].y);
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int kk = 0; kk < KW; ++kk) {
                        sacc[kk].x += __shfl_xor_sync(0xffffffffu, sacc[kk].x, o);
                        sacc[kk].y += __shfl_xor_sync(0xffffffffu, sacc[kk].y, o);
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int kk = 0; kk < KW; ++kk) {
                        const int k = warp + (k0 + kk) * NW;
                        if (k < modes) cf[k] = sacc[kk];
                    }
                }
            }
        }
        __syncthreads();
    }
    // a tensor copy still in flight (only after an expired wait) must land before the block exits
    if (abort_flag && tid == 0) mbar_wait(mb, parity);
}

template <int M, int MR0, int MR1>
static cudaError_t set_attr() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)FusedLayout<M, uint16_t>::bytes)))
        return e;
    return cudaFuncSetAttribute(k_fused128<M, MR0, MR1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FusedLayout<M, float>::bytes);
}

template <int M, int MR0, int MR1>
static void launch(const Plan& P, const FusedArgs& A, const CUtensorMap& tm, int dtype, int grid, cudaStream_t st) {
    if (dtype == DH_DTYPE_U16)
        k_fused128<M, MR0, MR1, uint16_t><<<grid, kFThreads, FusedLayout<M, uint16_t>::bytes, st>>>(P, A, tm);
    else
        k_fused128<M, MR0, MR1, float><<<grid, kFThreads, FusedLayout<M, float>::bytes, st>>>(P, A, tm);
}

}  // namespace dhk

namespace dh {

static int g_sm_count[64] = {0};
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool use_fused(const dhk::Plan& P) {
    if (P.n != dhk::kFN || P.groups > dhk::kFGMax || P.precision != DH_PRECISION_FP32) return false;
    if (P.pol[0].cal) return false;   // the reference calibration runs on the generic path
    return P.m == 32 || P.m == 48 || P.m == 64;
}

bool fused_frames_ok(const dhk::Plan& P, const void* frames, int dtype) {
    const int esz = dtype == DH_DTYPE_U16 ? 2 : 4;
    // tensor-copy rules: 16-byte aligned base and row pitch
    return ((uintptr_t)frames % 16 == 0) && ((size_t)P.width * esz) % 16 == 0;
}

cudaError_t fused_init() {
    cudaError_t e;
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if ((e = dhk::set_attr<32, 8, 4>())) return e;
    if ((e = dhk::set_attr<48, 3, 16>())) return e;
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
    if (!g_encode) return fail(DH_ERROR_ERROR, "tensor-map encoder unavailable");
    const int esz = dtype == DH_DTYPE_U16 ? 2 : 4;
    const int align = 16 / esz;
    // frames as a 3-D tensor [batch][height][width]; one box = the window rows plus alignment slack
    CUtensorMap tmap;
    const cuuint64_t gdim[3] = {(cuuint64_t)P.width, (cuuint64_t)P.height, (cuuint64_t)batch};
    const cuuint64_t gstride[2] = {(cuuint64_t)P.width * esz, (cuuint64_t)P.width * P.height * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(dhk::kFN + align), (cuuint32_t)dhk::kFRows, 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    CUresult cr = g_encode(&tmap, dtype == DH_DTYPE_U16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                           const_cast<void*>(frames), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(DH_ERROR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    dhk::FusedArgs A;
    A.src = frames;
    A.frame0 = 0;
    A.count = batch;
    for (int p = 0; p < DH_MAX_POLS; ++p) {
        const int ox = p < P.pols ? P.pol[p].ox : 0;
        A.x0[p] = (ox / align) * align;          // window origins are >= 0
        A.xo[p] = ox - A.x0[p];
    }
    A.fields = (float2*)fields;
    A.coefs = (float2*)coefs;
    // one block per SM; each block serves one polarisation, so the grid is a multiple of the polarisation count
    const long long per_pol = std::min<long long>(batch, std::max(1, g_sm_count[dev] / P.pols));
    const int grid = (int)per_pol * P.pols;
    if (tm) tm->start(st);
    switch (P.m) {
        case 32: dhk::launch<32, 8, 4>(P, A, tmap, dtype, grid, st); break;
        case 48: dhk::launch<48, 3, 16>(P, A, tmap, dtype, grid, st); break;
        default: dhk::launch<64, 8, 8>(P, A, tmap, dtype, grid, st); break;
    }
    if (tm) tm->stop(st, "k_fused128");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DH_SUCCESS;
}

}  // namespace dh
