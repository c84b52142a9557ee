// Fused single-kernel path for 128 x 128 windows (field sizes 32, 48 and 64): one thread block reconstructs
// one (frame, polarisation) window entirely in shared memory, persistent over windows.  uint16 frames run two
// blocks per SM, float32 frames (twice the staging buffer) one 512-thread block.
//
// Per window (the guide's pipeline steps 1-3 and digHoloProcessRemoveTilt):
//   y pass   real columns x and x + 64 packed as one complex column (times the reference-calibration factors
//            when enabled); radix-16 DIF pass from the window staged in shared memory by a tensor copy,
//            radix-8 pass fused with the separation of the two real spectra (Z(k), conj Z(-k)) and the
//            selection of the M box rows;
//   x pass   radix-16 then radix-8 DIF along x on the M box rows, the second pass fused with the box-column
//            selection, the circular mask and the beam-centre phase;
//   inverse  M-point inverse transform along x (DIT, digit-reversed in / natural out) and along y (DIF,
//            natural in / digit-reversed out), in place;
//   epilogue residual tilt and defocus removal in registers inside the last y pass, field write (coalesced
//            along x), and the separable HG contraction: partial sums over y per group of row blocks (mirrored
//            rows j and M - j paired, using the parity of u_n), then eight threads per mode summing the groups
//            and contracting along x with a fixed shuffle tree (deterministic, no atomics).
//            Split-BF16 variant (field size 64): the corrected field is written as the bf16 hi / lo A operand
//            of one 128 x 16 x 64 tcgen05 contraction over y (three products per K step, FP32 accumulation in
//            tensor memory, issued by one thread and awaited on an mbarrier with a bounded wait), read back by
//            four warps and contracted along x as above.
// Shared memory: the staging buffer of the next window (filled by the tensor copy while the current one is
// processed), one complex work buffer used in place by every step (y tile, box rows, window, field partial
// sums), twiddles, phases, the HG tables and the digit-reversal table: ~112 KB for uint16 frames, so two blocks
// share an SM.  Where a step writes over data other threads still read, the reads complete first (held in
// registers across a barrier).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>

#include <cuda_bf16.h>

#include "fft.cuh"
#include "runtime.hpp"
#include "sync.cuh"
#include "umma.cuh"

namespace dhk {

constexpr int kFN = 128;          // window size of this path
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
    float2* win_out;              // forward-only mode: windows [count][pol][M][M] (rows in digit-reversed order)
    const float2* win_in;         // inverse-only mode: windows in the same layout
};


template <typename T>
struct Staging {
    static constexpr int ALIGN = 16 / (int)sizeof(T);     // elements per 16 bytes
    static constexpr int W = kFN + ALIGN;                  // staged row width (window plus alignment slack)
    static constexpr int BYTES = kFRows * W * (int)sizeof(T);
};

// Threads per block and blocks per SM: uint16 frames fit two blocks per SM (two windows in flight, so one
// block's barriers overlap the other's work), of 512 threads at 64 registers for M = 64 (no spills) and of
// 256 threads otherwise; float32 frames need twice the staging buffer and run one 512-thread block per SM.
template <int M, typename T>
struct FusedShape {
    static constexpr int NT = (sizeof(T) == 2 && M != 64) ? 256 : 512;
    static constexpr int MINB = sizeof(T) == 2 ? 2 : 1;
};

template <int M, typename T>
struct FusedLayout {
    static constexpr int PITCH = M + 1;
    static constexpr int R1 = kFN * PITCH;                     // box rows r1[x][q], x-major
    static constexpr int YT = kFN * (kFN / 2);                 // y tile: 128 rows x 64 column pairs
    static constexpr int BUF = R1 > YT ? R1 : YT;              // the one complex work buffer, used in place
    static constexpr int WB = M * PITCH;                       // window / field [.][pitch]
    static constexpr int F2 = BUF + kFN + M + 4 * M;
    static constexpr int FL = 2 * kFGMax * M;                  // HG table as [n][i] and as [j][n]
    static constexpr int IN = 3 * M + 2 * (kFGMax * (kFGMax + 1) / 2);
    static constexpr size_t STG = (size_t)Staging<T>::BYTES;   // first, 128-byte aligned
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

// Write the separated spectra of columns x and x + N/2 at frequency k (if k is a box row), times 2: the
// factor 1/2 of the separation is carried by the y beam-centre phase (a power of two, so the rounding of every
// step in between is unchanged).
__device__ __forceinline__ void emit_pair(float2* r1, int pitch, int M, int kly, int x, int k, float2 zk, float2 zm) {
    const int q = (k - kly) & (kFN - 1);
    if (q < M) {
        r1[x * pitch + q] = make_float2(zk.x + zm.x, zk.y - zm.y);
        r1[(x + kFN / 2) * pitch + q] = make_float2(zk.y + zm.y, zm.x - zk.x);
    }
}

// TC: the y contraction in split-BF16 on the tensor cores (the split-BF16 precision; field size 64 only).
template <int M, int MR0, int MR1, typename T, int MODE, bool TC = false>
__global__ void __launch_bounds__(FusedShape<M, T>::NT, FusedShape<M, T>::MINB)
    k_fused128(const __grid_constant__ Plan P, const __grid_constant__ FusedArgs A, const __grid_constant__ CUtensorMap tmap) {
    using L = FusedLayout<M, T>;
    using S = Staging<T>;
    constexpr int N = kFN, PITCH = L::PITCH, NT = FusedShape<M, T>::NT;
    constexpr int NBLK = M / MR1;                  // row blocks of the last inverse pass
    constexpr int QB = NBLK < 4 ? NBLK : 4;        // partial-sum groups of the y contraction
    constexpr int BPQ = NBLK / QB;                 // row blocks per group
    static_assert(M == MR0 * MR1, "field size = product of the two radices");
    static_assert(NBLK % QB == 0, "row blocks split evenly into the partial-sum groups");
    static_assert(L::WB + QB * kFGMax * M <= L::BUF, "the partial sums fit behind the window");
    // y contraction over mirrored rows: group 0 holds blocks 0 and MR0/2, group qb > 0 blocks qb and MR0 - qb
    constexpr bool PAIRS = !TC && MR0 == 8 && QB == 4 && BPQ == 2 && MR1 % 2 == 0;
    // tensor-core y contraction: A = the corrected field as bf16 hi + lo, 2M rows (real parts of columns i, then
    // imaginary parts) by K = M field rows in the order kappa = MR1 blk + r of the last pass's outputs (row
    // j = blk + MR0 r), 2 x 2M x M bf16 behind the window; B = u_n(y'_j) dy' as bf16 hi + lo with its K rows
    // permuted the same way, in place of the FP32 y table; D = 2M x 16 FP32 in tensor memory
    static_assert(!TC || (M == 64 && MR1 == 8 && MODE != kModeForward), "tensor-core variant: M = 64");
    static_assert(!TC || L::WB * 8 + 8 * M * M <= L::BUF * 8, "A operand fits behind the window");
    constexpr uint32_t kTcTmemCols = 32;
    static_assert(M % 8 == 0, "box rows below M come in whole radix-8 tasks");
    // 128-byte alignment: tensor-copy destination; no larger, so that two blocks fit an SM
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t mbar_mma;   // TC: completion of the window's MMAs
    __shared__ uint32_t tmem_slot;               // TC: tensor-memory address
    __shared__ int abort_flag;
    T* stg = reinterpret_cast<T*>(smem_raw);
    float2* buf = reinterpret_cast<float2*>(smem_raw + L::STG);
    float2* twN = buf + L::BUF;
    float2* twM = twN + N;
    float2* phx = twM + M;
    float2* phy = phx + M;
    float2* cx = phy + M;
    float2* cy = cx + M;
    float* hgx = reinterpret_cast<float*>(cy + M);   // u_m(x'_i) dx' at [m][i]
    float* hgy = hgx + kFGMax * M;                   // u_n(y'_j) dy' at [j][n] (n fastest, kFGMax wide)
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
        phy[i] = cscale(pd.phase_y[i], 0.5f);   // with the 1/2 of the real-spectra separation
        cx[i] = pd.corr_x[i];
        cy[i] = pd.corr_y[i];
        mlo[i] = pd.mask_lo[i];
        mhi[i] = pd.mask_hi[i];
    }
    for (int i = tid; i < G * M; i += NT) hgx[i] = pd.hg_x[i];
    if constexpr (TC) {
        // B operand: the host's bf16 hi / lo planes of u_n(y'_j) dy' (rows n < 16, K = j), K permuted to kappa
        __nv_bfloat16* bop = reinterpret_cast<__nv_bfloat16*>(hgy);
        const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(pd.hgy_tc);
        for (int t = tid; t < 2 * kFGMax * M; t += NT) {
            const int hl = t / (kFGMax * M), rem = t - hl * kFGMax * M, n = rem / M, kap = rem - n * M;
            const int j = kap / MR1 + MR0 * (kap % MR1);
            bop[hl * kFGMax * M + umma_off(n, kap, M)] =
                G > 0 ? src[(size_t)hl * P.tc_np * M + umma_off(n, j, M)] : __float2bfloat16_rn(0.f);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (tid < 32) tmem_alloc(smem_u32(&tmem_slot), kTcTmemCols);
    } else {
        // u_n(y'_j) stored [j][n] (n fastest, kFGMax wide) so the y contraction reads four groups per load
        for (int i = tid; i < kFGMax * M; i += NT) {
            const int j = i / kFGMax, n = i - j * kFGMax;
            hgy[i] = n < G ? pd.hg_y[n * M + j] : 0.f;
        }
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
        if constexpr (TC) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_mma)));
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        if (MODE != kModeInverse) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            if (b < A.count) stage_window(&tmap, dst, mb, A.x0[pol], pd.oy, A.frame0 + b, S::BYTES);
        }
    }
    __syncthreads();
    const int xo = A.xo[pol];
    uint32_t parity = 0;
    uint32_t tmem = 0, mma_parity = 0;
    bool tc_ok = true;                           // TC: every MMA wait so far completed
    if constexpr (TC) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        tmem = tmem_slot;
    }
    for (; b < A.count; b += fstride) {
        const int f = A.frame0 + b;
        if constexpr (MODE == kModeInverse) {
            // the window comes from memory, rows already in the inverse transform's input order
            const float2* w = A.win_in + (size_t)(b * P.pols + pol) * M * M;
            for (int t = tid; t < M * M; t += NT)
                if (DH_IN(P.status, ((long long)b * P.pols + pol) * M * M + t, (long long)A.count * P.pols * M * M, kSiteFusedWindow))
                    buf[(t / M) * PITCH + t % M] = w[t];
            __syncthreads();
        } else {
        const bool ok = mbar_wait(mb, parity);
        parity ^= 1u;
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) {
            if (tid == 0 && P.status) atomicOr(P.status, 1);
            break;
        }

        // ---------------------------------------------------------------- y pass on 64 column pairs
        for (int t = tid; t < 512; t += NT) {
            const int c = t & 63, j = t >> 6;
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = staged_pair<T>(stg + (j + 8 * r) * S::W, xo + c);
            if (pd.cal) {
                // reference calibration: window pixel (x, y) times sqrt(max cal / cal), from the L2-resident table
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const float* k = pd.cal + (j + 8 * r) * N + c;
                    v[r].x *= __ldg(k);
                    v[r].y *= __ldg(k + N / 2);
                }
            }
            dft16<false>(v);
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twN[j * r]);
#pragma unroll
            for (int r = 0; r < 16; ++r) buf[(j + 8 * r) * 64 + c] = v[r];
        }
        // the staged window has been read (into registers) by every thread once the barrier completes; the next
        // tensor copy into the buffer is issued after it (a read-before-write across the proxies, ordered by the
        // barrier alone, as tensor-copy pipelines release a consumed stage)
        __syncthreads();
        if (tid == 0 && b + fstride < A.count) stage_window(&tmap, dst, mb, A.x0[pol], pd.oy, f + fstride, S::BYTES);
        {
            // radix-8 pass and separation of the two real spectra, in place: every task's inputs are read
            // before the box rows r1[x][q] overwrite the tile
            constexpr int TPT = 512 / NT;
            float2 z1[TPT][8], z2[TPT][8];
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                const int t = tid + k * NT, c = t & 63, u = t >> 6;
                const int d1 = u, d2 = (u == 0) ? 8 : 16 - u;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    z1[k][r] = buf[(8 * d1 + r) * 64 + c];
                    z2[k][r] = buf[(8 * d2 + r) * 64 + c];
                }
                dft8<false>(z1[k]);
                dft8<false>(z2[k]);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                const int t = tid + k * NT, x = t & 63, u = t >> 6;
                const int d1 = u, d2 = (u == 0) ? 8 : 16 - u;
                if (u != 0) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        emit_pair(buf, PITCH, M, pd.kly, x, d1 + 16 * r, z1[k][r], z2[k][7 - r]);
                        emit_pair(buf, PITCH, M, pd.kly, x, d2 + 16 * r, z2[k][r], z1[k][7 - r]);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        emit_pair(buf, PITCH, M, pd.kly, x, 16 * r, z1[k][r], z1[k][(8 - r) & 7]);
                        emit_pair(buf, PITCH, M, pd.kly, x, 8 + 16 * r, z2[k][r], z2[k][7 - r]);
                    }
                }
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- x pass on the M box rows
        spass<16, false, false, N, N, M, PITCH, 1, NT>(buf, twN, tid);
        __syncthreads();
        {
            // radix-8 pass fused with the box-column selection, mask and beam-centre phase, writing the window
            // w[posM[p]][q] over box rows x < M: the tasks that read those rows (d < M/8) keep their outputs in
            // registers across a barrier; the others read rows >= M, which nothing overwrites
            constexpr int LOW = (M / 8) * M;
            constexpr int LT = (LOW + NT - 1) / NT;
            float2 keep[LT][8];
#pragma unroll
            for (int k = 0; k < LT; ++k) {
                const int t = tid + k * NT;
                if (t < LOW) {
                    const int q = t % M, d = t / M;
#pragma unroll
                    for (int r = 0; r < 8; ++r) keep[k][r] = buf[(8 * d + r) * PITCH + q];
                    dft8<false>(keep[k]);
                    const int lo = mlo[q], hi = mhi[q];
                    const float2 py = phy[q];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int p = (d + 16 * r - pd.klx) & (N - 1);
                        if (p < M)   // the same for the whole warp (d is)
                            keep[k][r] = (p >= lo && p <= hi) ? cmul(cmul(keep[k][r], phx[p]), py) : make_float2(0.f, 0.f);
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < LT; ++k) {
                const int t = tid + k * NT;
                if (t < LOW) {
                    const int q = t % M, d = t / M;
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int p = (d + 16 * r - pd.klx) & (N - 1);
                        if (p < M) buf[posM[p] * PITCH + q] = keep[k][r];
                    }
                }
            }
            for (int t = LOW + tid; t < M * 16; t += NT) {
                const int q = t % M, d = t / M;
                float2 v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = buf[(8 * d + r) * PITCH + q];
                dft8<false>(v);
                const int lo = mlo[q], hi = mhi[q];
                const float2 py = phy[q];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int p = (d + 16 * r - pd.klx) & (N - 1);
                    if (p < M) {
                        float2 val = make_float2(0.f, 0.f);
                        if (p >= lo && p <= hi) val = cmul(cmul(v[r], phx[p]), py);
                        buf[posM[p] * PITCH + q] = val;
                    }
                }
            }
        }
        __syncthreads();
        }   // forward part
        if constexpr (MODE == kModeForward) {
            float2* w = A.win_out + (size_t)(b * P.pols + pol) * M * M;
            for (int t = tid; t < M * M; t += NT)
                if (DH_IN(P.status, ((long long)b * P.pols + pol) * M * M + t, (long long)A.count * P.pols * M * M, kSiteFusedWindow))
                    w[t] = buf[(t / M) * PITCH + t % M];
            __syncthreads();
            continue;
        }

        // ---------------------------------------------------------------- inverse transforms
        spass<MR1, true, true, M, MR1, M, PITCH, 1, NT>(buf, twM, tid);
        __syncthreads();
        spass<MR0, true, true, M, M, M, PITCH, 1, NT>(buf, twM, tid);
        __syncthreads();
        spass<MR0, true, false, M, M, M, 1, PITCH, NT>(buf, twM, tid);
        __syncthreads();

        // ---------------------------------------------------------------- last y pass, correction, field, y overlap
        // The last DIF pass (span MR1, no twiddles) leaves output j = blk + MR0 r at position blk MR1 + r of
        // column i; it is corrected in registers, written to the field (coalesced along i) and contracted with
        // u_n(y'_j) into the partial sums part[qb][n][i] over the BPQ row blocks of group qb (with PAIRS, the
        // blocks of a group hold each other's mirror rows M - j).
        float2* part = buf + L::WB;                // [QB][G][M], behind the window
        const bool ov = A.coefs && G > 0;
        {
            float2* fld = A.fields ? A.fields + (size_t)(f * P.pols + pol) * M * M : nullptr;
            for (int t = tid; t < M * QB; t += NT) {
                const int i = t % M, qb = t / M;
                const float2 ci = cx[i];
                float2 v[BPQ][MR1];
#pragma unroll
                for (int bb = 0; bb < BPQ; ++bb) {
                    const int blk = PAIRS ? (qb == 0 ? bb * (MR0 / 2) : (bb == 0 ? qb : MR0 - qb)) : qb * BPQ + bb;
#pragma unroll
                    for (int r = 0; r < MR1; ++r) v[bb][r] = buf[i * PITCH + blk * MR1 + r];
                    dft<MR1, true>(v[bb], twM, M / MR1);
#pragma unroll
                    for (int r = 0; r < MR1; ++r) {
                        const int j = blk + MR0 * r;
                        v[bb][r] = cmul(cmul(v[bb][r], ci), cy[j]);
                        if (fld && DH_IN(P.status, (long long)j * M + i, (long long)M * M, kSiteFusedField)) fld[j * M + i] = v[bb][r];
                    }
                }
                if (ov) {
                    if constexpr (TC) {
                        // this thread's rows j = blk + MR0 r are the 8 consecutive K positions kappa = MR1 blk + r:
                        // one 16-byte row of a core matrix per plane (hi / lo) and part (real / imaginary)
                        __nv_bfloat16* aop = reinterpret_cast<__nv_bfloat16*>(buf + L::WB);
#pragma unroll
                        for (int bb = 0; bb < BPQ; ++bb) {
                            const int blk = qb * BPQ + bb;
                            __align__(16) __nv_bfloat16 hr[8], hm[8], lr[8], lm[8];
#pragma unroll
                            for (int r = 0; r < MR1; ++r) {
                                const float2 e = v[bb][r];
                                hr[r] = __float2bfloat16_rn(e.x);
                                hm[r] = __float2bfloat16_rn(e.y);
                                lr[r] = __float2bfloat16_rn(e.x - __bfloat162float(hr[r]));
                                lm[r] = __float2bfloat16_rn(e.y - __bfloat162float(hm[r]));
                            }
                            const int o_r = umma_off(i, MR1 * blk, M), o_m = umma_off(M + i, MR1 * blk, M);
                            *reinterpret_cast<uint4*>(aop + o_r) = *reinterpret_cast<const uint4*>(hr);
                            *reinterpret_cast<uint4*>(aop + o_m) = *reinterpret_cast<const uint4*>(hm);
                            *reinterpret_cast<uint4*>(aop + 2 * M * M + o_r) = *reinterpret_cast<const uint4*>(lr);
                            *reinterpret_cast<uint4*>(aop + 2 * M * M + o_m) = *reinterpret_cast<const uint4*>(lm);
                        }
                    } else if constexpr (PAIRS) {
                        // rows j and M - j carry u_n(y'_{M-j}) = (-1)^n u_n(y'_j): the even modes contract the
                        // sums E_j + E_{M-j}, the odd ones the differences, each with u_n(y'_j) (half the products)
                        float2 sp[MR1 + 1], sm[MR1 + 1];
                        int jr[MR1 + 1];
                        if (qb == 0) {
                            // block 0 (rows MR0 r) pairs r with MR1 - r; row 0 has no mirror and row M/2 is its own
                            // (odd modes vanish there); block MR0/2 pairs r with MR1 - 1 - r
                            int u = 0;
#pragma unroll
                            for (int r = 1; r < MR1 / 2; ++r, ++u) {
                                sp[u] = cadd(v[0][r], v[0][MR1 - r]);
                                sm[u] = csub(v[0][r], v[0][MR1 - r]);
                                jr[u] = MR0 * r;
                            }
                            sp[u] = sm[u] = v[0][0];
                            jr[u++] = 0;
                            sp[u] = sm[u] = v[0][MR1 / 2];
                            jr[u++] = M / 2;
#pragma unroll
                            for (int r = 0; r < MR1 / 2; ++r, ++u) {
                                sp[u] = cadd(v[1][r], v[1][MR1 - 1 - r]);
                                sm[u] = csub(v[1][r], v[1][MR1 - 1 - r]);
                                jr[u] = MR0 / 2 + MR0 * r;
                            }
                        } else {
                            // blocks qb and MR0 - qb: row qb + MR0 r mirrors row (MR0 - qb) + MR0 (MR1 - 1 - r)
#pragma unroll
                            for (int r = 0; r < MR1; ++r) {
                                sp[r] = cadd(v[0][r], v[1][MR1 - 1 - r]);
                                sm[r] = csub(v[0][r], v[1][MR1 - 1 - r]);
                                jr[r] = qb + MR0 * r;
                            }
                            sp[MR1] = sm[MR1] = make_float2(0.f, 0.f);
                            jr[MR1] = 0;
                        }
                        const int nu = qb == 0 ? MR1 + 1 : MR1;
#pragma unroll
                        for (int n4 = 0; n4 < kFGMax; n4 += 4) {
                            if (n4 < G) {
                                float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                               make_float2(0.f, 0.f)};
#pragma unroll
                                for (int u = 0; u < MR1 + 1; ++u) {
                                    if (u < nu) {
                                        const float4 w = *reinterpret_cast<const float4*>(hgy + jr[u] * kFGMax + n4);
                                        a[0].x = fmaf(w.x, sp[u].x, a[0].x);
                                        a[0].y = fmaf(w.x, sp[u].y, a[0].y);
                                        a[1].x = fmaf(w.y, sm[u].x, a[1].x);
                                        a[1].y = fmaf(w.y, sm[u].y, a[1].y);
                                        a[2].x = fmaf(w.z, sp[u].x, a[2].x);
                                        a[2].y = fmaf(w.z, sp[u].y, a[2].y);
                                        a[3].x = fmaf(w.w, sm[u].x, a[3].x);
                                        a[3].y = fmaf(w.w, sm[u].y, a[3].y);
                                    }
                                }
#pragma unroll
                                for (int c = 0; c < 4; ++c)
                                    if (n4 + c < G) part[(qb * G + n4 + c) * M + i] = a[c];
                            }
                        }
                    } else {
#pragma unroll
                        for (int n4 = 0; n4 < kFGMax; n4 += 4) {
                            if (n4 < G) {
                                float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                               make_float2(0.f, 0.f)};
#pragma unroll
                                for (int bb = 0; bb < BPQ; ++bb) {
#pragma unroll
                                    for (int r = 0; r < MR1; ++r) {
                                        const int j = qb * BPQ + bb + MR0 * r;
                                        const float4 u = *reinterpret_cast<const float4*>(hgy + j * kFGMax + n4);
                                        const float2 e = v[bb][r];
                                        a[0].x = fmaf(u.x, e.x, a[0].x);
                                        a[0].y = fmaf(u.x, e.y, a[0].y);
                                        a[1].x = fmaf(u.y, e.x, a[1].x);
                                        a[1].y = fmaf(u.y, e.y, a[1].y);
                                        a[2].x = fmaf(u.z, e.x, a[2].x);
                                        a[2].y = fmaf(u.z, e.y, a[2].y);
                                        a[3].x = fmaf(u.w, e.x, a[3].x);
                                        a[3].y = fmaf(u.w, e.y, a[3].y);
                                    }
                                }
#pragma unroll
                                for (int c = 0; c < 4; ++c)
                                    if (n4 + c < G) part[(qb * G + n4 + c) * M + i] = a[c];
                            }
                        }
                    }
                }
            }
        }
        if constexpr (TC) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        // TC: T[n][r] (r < M: real part of column r, r >= M: imaginary part of column r - M) over the consumed
        // window, [16][kTsPitch]
        constexpr int kTsPitch = 2 * M + 1;
        float* Ts = reinterpret_cast<float*>(buf);
        if constexpr (TC) {
            if (ov) {
                // y contraction: hi hi + hi lo + lo hi per 16-wide K step, FP32 accumulation in tensor memory
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t mbm = smem_u32(&mbar_mma);
                if (tid == 0 && tc_ok) {
                    const uint32_t a_hi = smem_u32(buf + L::WB), a_lo = a_hi + 4 * M * M;
                    const uint32_t b_hi = smem_u32(hgy), b_lo = b_hi + 2 * kFGMax * M;
                    constexpr uint32_t idesc = umma_idesc_bf16(2 * M, kFGMax);
                    const uint32_t lbo = 128, sbo = 16 * M;
#pragma unroll
                    for (int ks = 0; ks < M / 16; ++ks) {
                        const uint32_t ko = ks * 256;
                        umma_bf16(tmem, umma_desc(a_hi + ko, lbo, sbo), umma_desc(b_hi + ko, lbo, sbo), idesc, ks > 0);
                        umma_bf16(tmem, umma_desc(a_hi + ko, lbo, sbo), umma_desc(b_lo + ko, lbo, sbo), idesc, 1);
                        umma_bf16(tmem, umma_desc(a_lo + ko, lbo, sbo), umma_desc(b_hi + ko, lbo, sbo), idesc, 1);
                    }
                    umma_commit(mbm);
                }
                bool done = false;
                if (tc_ok) {   // the same for every thread
                    done = bounded_mbar_wait(mbm, mma_parity, kFWaitLimit);
                    mma_parity ^= 1u;
                }
                // one decision for the whole block (the tensor-memory loads below are warp-collective)
                const bool all = __syncthreads_and(done ? 1 : 0) != 0;
                if (tc_ok && !all && tid == 0 && P.status) atomicOr(P.status, 2);
                tc_ok = tc_ok && all;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int warp = tid >> 5, lane = tid & 31;
                if (warp < 4) {
                    float tv[16];
                    if (tc_ok) tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), tv);
#pragma unroll
                    for (int n = 0; n < kFGMax; ++n) Ts[n * kTsPitch + 32 * warp + lane] = tc_ok ? tv[n] : __int_as_float(0x7fc00000);
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncthreads();
            }
        }

        // ---------------------------------------------------------------- HG overlap, x contraction
        if (ov) {
            // c_mn = sum_i u_m(x'_i) T[n][i] with T[n][i] = sum_qb part[qb][n][i] (groups added in a fixed order):
            // eight threads per mode, thread s taking the column pairs i = 2s + 16h, h < M/16, then a fixed
            // three-level shuffle tree over the eight
            float2* cf = A.coefs + (size_t)(f * P.pols + pol) * modes;
            const int s8 = tid & 7;
            for (int t0 = tid & ~31; t0 < modes * 8; t0 += NT) {
                const int k = (t0 + (tid & 31)) >> 3;
                float2 acc = make_float2(0.f, 0.f);
                if (TC && k < modes) {
                    const float* um = hgx + mdm[k] * M;
                    const float* tr = Ts + mdn[k] * kTsPitch;
#pragma unroll
                    for (int h = 0; h < M / 16; ++h) {
                        const int i = 2 * s8 + 16 * h;
                        const float2 u = *reinterpret_cast<const float2*>(um + i);
                        acc.x = fmaf(u.x, tr[i], acc.x);
                        acc.y = fmaf(u.x, tr[M + i], acc.y);
                        acc.x = fmaf(u.y, tr[i + 1], acc.x);
                        acc.y = fmaf(u.y, tr[M + i + 1], acc.y);
                    }
                } else if (k < modes) {
                    const float* um = hgx + mdm[k] * M;
                    const float2* tn = part + mdn[k] * M;
#pragma unroll
                    for (int h = 0; h < M / 16; ++h) {
                        const int i = 2 * s8 + 16 * h;
                        const float2 u = *reinterpret_cast<const float2*>(um + i);
                        float4 v = *reinterpret_cast<const float4*>(tn + i);
#pragma unroll
                        for (int q = 1; q < QB; ++q) {
                            const float4 w = *reinterpret_cast<const float4*>(tn + q * G * M + i);
                            v.x += w.x;
                            v.y += w.y;
                            v.z += w.z;
                            v.w += w.w;
                        }
                        acc.x = fmaf(u.x, v.x, acc.x);
                        acc.y = fmaf(u.x, v.y, acc.y);
                        acc.x = fmaf(u.y, v.z, acc.x);
                        acc.y = fmaf(u.y, v.w, acc.y);
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
                if (s8 == 0 && k < modes && DH_IN(P.status, k, modes, kSiteFusedCoef)) cf[k] = acc;
            }
        }
        __syncthreads();
    }
    // a tensor copy still in flight (only after an expired wait) must land before the block exits
    if (MODE != kModeInverse && abort_flag && tid == 0) mbar_wait(mb, parity);
    if constexpr (TC) {
        // MMAs still in flight (only after an expired wait: the last ones issued) must complete before their tensor
        // memory is freed
        if (!tc_ok && tid == 0) bounded_mbar_wait(smem_u32(&mbar_mma), mma_parity ^ 1u, kFWaitLimit);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (tid < 32) tmem_free(tmem, kTcTmemCols);
    }
}

template <int M, int MR0, int MR1, int MODE>
static cudaError_t set_attr_mode() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, uint16_t, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)FusedLayout<M, uint16_t>::bytes)))
        return e;
    return cudaFuncSetAttribute(k_fused128<M, MR0, MR1, float, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FusedLayout<M, float>::bytes);
}

template <int M, int MR0, int MR1>
static cudaError_t set_attr() {
    cudaError_t e;
    if ((e = set_attr_mode<M, MR0, MR1, kModeFull>())) return e;
    if ((e = set_attr_mode<M, MR0, MR1, kModeForward>())) return e;
    if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, uint16_t, kModeInverse>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)FusedLayout<M, uint16_t>::bytes)))
        return e;
    if constexpr (M == 64) {
        // the split-BF16 (tensor-core) variants of the modes that contract
        if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, uint16_t, kModeFull, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedLayout<M, uint16_t>::bytes)))
            return e;
        if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, float, kModeFull, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedLayout<M, float>::bytes)))
            return e;
        if ((e = cudaFuncSetAttribute(k_fused128<M, MR0, MR1, uint16_t, kModeInverse, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedLayout<M, uint16_t>::bytes)))
            return e;
    }
    return cudaSuccess;
}

// Resident blocks per SM of one instantiation (the persistent grid is SMs x this).  The inverse-only mode
// does not read frames and always runs the uint16 shape.
template <int M, int MR0, int MR1>
static int blocks_per_sm(int dtype, int mode) {
    int n = 0;
    cudaError_t e;
    if (mode == kModeInverse)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused128<M, MR0, MR1, uint16_t, kModeInverse>,
                                                          FusedShape<M, uint16_t>::NT, FusedLayout<M, uint16_t>::bytes);
    else if (dtype == DH_DTYPE_U16)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused128<M, MR0, MR1, uint16_t, kModeFull>,
                                                          FusedShape<M, uint16_t>::NT, FusedLayout<M, uint16_t>::bytes);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused128<M, MR0, MR1, float, kModeFull>,
                                                          FusedShape<M, float>::NT, FusedLayout<M, float>::bytes);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

template <int M, int MR0, int MR1, typename T, int MODE, bool TC = false>
static void launch_one(const Plan& P, const FusedArgs& A, const CUtensorMap& tm, int grid, cudaStream_t st) {
    k_fused128<M, MR0, MR1, T, MODE, TC><<<grid, FusedShape<M, T>::NT, FusedLayout<M, T>::bytes, st>>>(P, A, tm);
}

// TC: the split-BF16 variant (field size 64; the forward-only mode does not contract and has none)
template <int M, int MR0, int MR1, bool TC>
static void launch(const Plan& P, const FusedArgs& A, const CUtensorMap& tm, int dtype, int mode, int grid,
                   cudaStream_t st) {
    if (mode == kModeInverse)
        launch_one<M, MR0, MR1, uint16_t, kModeInverse, TC>(P, A, tm, grid, st);
    else if (dtype == DH_DTYPE_U16)
        mode == kModeForward ? launch_one<M, MR0, MR1, uint16_t, kModeForward>(P, A, tm, grid, st)
                             : launch_one<M, MR0, MR1, uint16_t, kModeFull, TC>(P, A, tm, grid, st);
    else
        mode == kModeForward ? launch_one<M, MR0, MR1, float, kModeForward>(P, A, tm, grid, st)
                             : launch_one<M, MR0, MR1, float, kModeFull, TC>(P, A, tm, grid, st);
}

}  // namespace dhk

namespace dh {

static int g_sm_count[64] = {0};
static int g_bps[64][9] = {};   // resident blocks per SM per (field size, pixel type or inverse mode)
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool use_fused(const dhk::Plan& P) {
    if (P.n != dhk::kFN || P.ny != P.n || P.my != P.m || P.groups > dhk::kFGMax) return false;
    if (P.precision == DH_PRECISION_SPLIT_BF16)   // the tensor-core variant: field size 64, B operand of 16 rows
        return P.m == 64 && (P.groups == 0 || P.tc_np == dhk::kFGMax);
    return P.precision == DH_PRECISION_FP32 && (P.m == 32 || P.m == 48 || P.m == 64);
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

int launch_fused(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int total, int frame0, int count,
                 int mode, const float2* win_in, float2* win_out, void* fields, void* coefs, cudaStream_t st,
                 dhk::StageTimer* tm) {
    int dev = H->device;
    if (dev < 0 || dev >= 64) return fail(DH_ERROR_ERROR, "device index out of range");
    if (count < 1) return DH_SUCCESS;
    if (!g_sm_count[dev]) {
        int n = 0;
        cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device attribute");
        g_sm_count[dev] = n;
    }
    const int esz = dtype == DH_DTYPE_U16 ? 2 : 4;
    const int align = 16 / esz;
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof tmap);   // unused by the inverse-only mode, which reads no frames
    if (mode != dhk::kModeInverse) {
        if (!g_encode) return fail(DH_ERROR_ERROR, "tensor-map encoder unavailable");
        // frames as a 3-D tensor [total][height][width]; one box = the window rows plus alignment slack
        const cuuint64_t gdim[3] = {(cuuint64_t)P.width, (cuuint64_t)P.height, (cuuint64_t)total};
        const cuuint64_t gstride[2] = {(cuuint64_t)P.width * esz, (cuuint64_t)P.width * P.height * esz};
        const cuuint32_t box[3] = {(cuuint32_t)(dhk::kFN + align), (cuuint32_t)dhk::kFRows, 1};
        const cuuint32_t estride[3] = {1, 1, 1};
        CUresult cr = g_encode(&tmap, dtype == DH_DTYPE_U16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               3, const_cast<void*>(frames), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return fail(DH_ERROR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    }
    dhk::FusedArgs A;
    A.src = frames;
    A.frame0 = frame0;
    A.count = count;
    for (int p = 0; p < DH_MAX_POLS; ++p) {
        const int ox = p < P.pols ? P.pol[p].ox : 0;
        A.x0[p] = (ox / align) * align;          // window origins are >= 0
        A.xo[p] = ox - A.x0[p];
    }
    A.fields = (float2*)fields;
    A.coefs = (float2*)coefs;
    A.win_out = win_out;
    A.win_in = win_in;
    // a persistent grid of every resident block; each block serves one polarisation, so the grid is a multiple
    // of the polarisation count
    const int slot = (P.m == 32 ? 0 : P.m == 48 ? 1 : 2) * 3 + (mode == dhk::kModeInverse ? 2 : dtype == DH_DTYPE_U16 ? 0 : 1);
    if (!g_bps[dev][slot]) {
        g_bps[dev][slot] = P.m == 32   ? dhk::blocks_per_sm<32, 8, 4>(dtype, mode)
                           : P.m == 48 ? dhk::blocks_per_sm<48, 3, 16>(dtype, mode)
                                       : dhk::blocks_per_sm<64, 8, 8>(dtype, mode);
    }
    const int resident = g_sm_count[dev] * g_bps[dev][slot];
    const long long per_pol = std::min<long long>(count, std::max(1, resident / P.pols));
    const int grid = (int)per_pol * P.pols;
    if (tm) tm->start(st);
    switch (P.m) {
        case 32: dhk::launch<32, 8, 4, false>(P, A, tmap, dtype, mode, grid, st); break;
        case 48: dhk::launch<48, 3, 16, false>(P, A, tmap, dtype, mode, grid, st); break;
        default:
            if (P.precision == DH_PRECISION_SPLIT_BF16)
                dhk::launch<64, 8, 8, true>(P, A, tmap, dtype, mode, grid, st);
            else
                dhk::launch<64, 8, 8, false>(P, A, tmap, dtype, mode, grid, st);
            break;
    }
    const bool tc = P.precision == DH_PRECISION_SPLIT_BF16 && mode != dhk::kModeForward;
    if (tm)
        tm->stop(st, mode == dhk::kModeForward ? "k_fused128_fwd"
                     : mode == dhk::kModeInverse ? (tc ? "k_fused128_inv_tc" : "k_fused128_inv")
                                                 : (tc ? "k_fused128_tc" : "k_fused128"));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DH_SUCCESS;
}

}  // namespace dh
