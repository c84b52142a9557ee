// Fused single-kernel path for 256 x 256 windows with 96 x 96 fields (uint16 frames, FP32 overlap, G <= 16): one
// 512-thread block per SM reconstructs one (frame, polarisation) window at a time entirely in shared memory,
// persistent over windows.
//
// The y-transformed box rows of a 256 x 256 window (96 rows of 256 complex values, 192 KB) do not fit beside a
// staging buffer, so the window is transformed along x first and along y by decimation in time over four row
// groups: window row n = 4 n1 + n2 belongs to group n2, and the spectrum at row frequency k is
//     X[k] = sum_{n2 < 4} W_256^{n2 k} A_{n2}[k mod 64],   A_{n2} = the 64-point DFT over n1 of group n2's rows,
// so each group's contribution is added to the 96 x 96 box sums (in registers) as soon as it is transformed (the guide's
// pipeline steps 1-2: FFT of the window, selection of the off-axis window; the same sums in another order).
// Per group (64 rows, staged by two tensor copies of 136-column boxes through a 4-D view of the window rows):
//   x pass      rows n1 and n1 + 32 packed as one complex row (times the reference-calibration factors when
//               enabled), radix-16 DIF pass from the staged rows, radix-16 pass written out in natural frequency
//               order;
//   y pass      on the 96 box columns: the separation of the two real spectra (Z(k), conj Z(-k)) as the first
//               pass reads them, radix-16 then radix-4 DIF over n1; each output is multiplied by W_256^{n2 k}
//               and added to the sum of its box row (one or two rows per output).  The circular mask and the
//               beam-centre phase are applied after the last group.
// Then (pipeline step 3 and digHoloProcessRemoveTilt):
//   inverse     96-point inverse transforms with radices 12 (prime-factor 3 x 4, no twiddles) and 8, along x
//               (DIT: the first pass reads the summed spectrum and writes the window in digit-reversed order) and
//               along y (DIF);
//   epilogue    the last y pass in registers with the residual tilt and defocus removal, the field write and the
//               separable HG contraction (mirrored row pairs, then eight threads per mode along x), as the
//               128 x 128 kernel does.  Split-BF16 variant (TC): the corrected field is written as the bf16 hi / lo
//               A operand (192 rows: real, then imaginary parts of the 96 columns; K = the 96 field rows in the
//               order the last pass leaves them) of two 128 x 16 x 96 tcgen05 contractions over y (three products
//               per K step, FP32 accumulation in 32 tensor-memory columns, issued by one thread and awaited on an
//               mbarrier with a bounded wait), read back by four warps and contracted along x.
// Shared memory: staging of one row group (34.8 KB, refilled by the next group's tensor copies while the current
// group is transformed), two work buffers (the packed x rows, then the box columns, then the window during the
// inverse; and the x spectra, then the summed window spectrum, then the partial sums of the y contraction or the
// tensor-core A operand) and the tables: 209 KB, one block per SM.
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

constexpr int k2N = 256;             // window size
constexpr int k2M = 96;              // field size
constexpr int k2G = 16;              // largest group count
constexpr int k2NT = 512;            // threads per block
constexpr int k2Rows = 64;           // window rows per group (n1)
constexpr int k2BoxW = 136;          // staged columns per tensor copy (128 plus the 16-byte alignment slack)
constexpr int k2BoxBytes = k2BoxW * k2Rows * 2;
constexpr int k2PW = k2N + 1;        // pitch of the packed x rows (odd: conflict-free column access)
constexpr int k2PB = k2Rows + 1;     // pitch of the box columns [c][n1]
constexpr int k2PA = k2M + 1;        // pitch of the summed spectrum [c][q] and of the window [x][q]
constexpr int k2MR0 = 8, k2MR1 = 12; // inverse radix plan (DIF order)
constexpr long k2WaitLimit = 1L << 24;

struct F256Args {
    int count;                       // frames [0, count)
    int xo[DH_MAX_POLS];             // window origin minus the 16-byte-aligned staging origin, per polarisation
    int x0[DH_MAX_POLS];             // staging origin (16-byte aligned element index), per polarisation
    float2* fields;                  // nullable [B][pol][M][M]
    float2* coefs;                   // nullable [B][pol][modes]
};

struct F256Smem {
    static constexpr size_t STG = 2 * (size_t)k2BoxBytes;                                    // two boxes
    static constexpr size_t WORKN = (32 * k2PW > k2M * k2PA) ? 32 * k2PW : k2M * k2PA;       // float2
    static constexpr size_t ACCN = (size_t)k2M * k2PA;                                       // float2
    static constexpr size_t TABN = 2 * k2N + 5 * k2M + 4 * k2M + 64;                         // float2
    static constexpr size_t HGN = 2 * (size_t)k2G * k2M;                                     // float
    static constexpr size_t INTN = 2 * k2M + 2 * (k2G * (k2G + 1) / 2);                      // int
    static constexpr size_t bytes = STG + (WORKN + ACCN + TABN) * 8 + HGN * 4 + INTN * 4;
};
static_assert(F256Smem::STG % 16 == 0 && (F256Smem::WORKN * 8) % 16 == 0 && (F256Smem::ACCN * 8) % 16 == 0,
              "16-byte aligned regions");
static_assert(4 * k2G * k2M <= (int)F256Smem::ACCN, "the partial sums fit in the second buffer");
static_assert(32 * k2PW <= (int)F256Smem::ACCN, "the x spectra fit in the second buffer");
static_assert(k2M * k2PB <= (int)F256Smem::WORKN, "the box columns fit in the work buffer");

// 12-point DFT in registers by the prime-factor map (3 x 4, coprime, so no twiddles): input n = (4 n1 + 3 n2)
// mod 12 enters the 3-point transform n2 at position n1, and output k = (4 k1 + 9 k2) mod 12 leaves the
// 4-point transform k1 at position k2.
template <bool INV>
__device__ __forceinline__ void dft12(float2* a) {
    float2 t[4][3];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1) t[n2][n1] = a[(4 * n1 + 3 * n2) % 12];
        dft3<INV>(t[n2]);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        float2 h0 = t[0][k1], h1 = t[1][k1], h2 = t[2][k1], h3 = t[3][k1];
        dft4<INV>(h0, h1, h2, h3);
        a[(4 * k1) % 12] = h0;
        a[(4 * k1 + 9) % 12] = h1;
        a[(4 * k1 + 18) % 12] = h2;
        a[(4 * k1 + 27) % 12] = h3;
    }
}

// One thread: expect one row group's bytes on the mbarrier and start its two tensor copies (columns x0 .. x0 + 135
// and x0 + 128 .. x0 + 263 of window rows n2, n2 + 4, ..., n2 + 252 of frame f).
__device__ __forceinline__ void stage_group(const CUtensorMap* tmap, uint32_t dst, uint32_t mbar, int x0, int n2, int f) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(2 * k2BoxBytes) : "memory");
#pragma unroll
    for (int h = 0; h < 2; ++h)
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(
                dst + h * k2BoxBytes),
            "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0 + 128 * h), "r"(n2), "r"(0), "r"(f), "r"(mbar)
            : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    return bounded_mbar_wait(mbar, parity, k2WaitLimit);
}

// bf16 bits (round to nearest even) of a and b packed low / high, and of their remainders a - hi(a), b - hi(b).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// Twelve bf16 values (six packed pairs) at K positions kb .. kb + 11 of one row of a canonical K-major operand with
// K = 96 (kb a multiple of 4): one 16-byte and one 8-byte store.
__device__ __forceinline__ void store_run12(__nv_bfloat16* op, int row, int kb, const uint32_t* w) {
    if ((kb & 7) == 0) {
        *reinterpret_cast<uint4*>(op + umma_off(row, kb, k2M)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint2*>(op + umma_off(row, kb + 8, k2M)) = make_uint2(w[4], w[5]);
    } else {
        *reinterpret_cast<uint2*>(op + umma_off(row, kb, k2M)) = make_uint2(w[0], w[1]);
        *reinterpret_cast<uint4*>(op + umma_off(row, kb + 4, k2M)) = make_uint4(w[2], w[3], w[4], w[5]);
    }
}

// TC: the y contraction in split-BF16 on the tensor cores (the split-BF16 precision).
template <bool TC>
__global__ void __launch_bounds__(k2NT, 1)
    k_fused256(const __grid_constant__ Plan P, const __grid_constant__ F256Args A,
               const __grid_constant__ CUtensorMap tmap0, const __grid_constant__ CUtensorMap tmap1) {
    using L = F256Smem;
    constexpr int N = k2N, M = k2M, NT = k2NT, MR0 = k2MR0, MR1 = k2MR1;
    constexpr int QB = 4, BPQ = 2;   // partial-sum groups of the y contraction, row blocks per group
    static_assert(M == MR0 * MR1 && MR0 == 8 && MR1 % 2 == 0, "mirrored-row y contraction: eight row blocks");
    // TC: A = [2M rows][K = M] bf16 hi, then lo, over the second buffer; K position kappa = MR1 blk + r holds field
    // row j = blk + MR0 r.  The second 128-row tile (rows 128 .. 255) reads 64 rows past the 2M written ones: they
    // only feed tensor-memory rows 192 .. 255, which nothing reads, and stay inside the block's shared memory.
    static_assert(4 * M * M * 2 <= (int)L::ACCN * 8, "the A operand's two planes fit in the second buffer");
    static_assert(L::STG + L::WORKN * 8 + 4 * M * M + 256 * M * 2 <= L::bytes, "the second tile's reads stay in shared memory");
    constexpr uint32_t kTcCols = 32;
    constexpr int kTsPitch = 2 * M + 1;   // TC: T[n][r] read back from tensor memory, r < M real, r >= M imaginary
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t mbar_mma;   // TC: completion of the window's MMAs
    __shared__ uint32_t tmem_slot;               // TC: tensor-memory address
    __shared__ int abort_flag;
    const uint16_t* stg = reinterpret_cast<const uint16_t*>(smem_raw);
    float2* work = reinterpret_cast<float2*>(smem_raw + L::STG);
    float2* buf2 = work + L::WORKN;
    float2* twN = buf2 + L::ACCN;
    float2* tw16 = twN + N;                          // W_256^{j r} at [r][j]: the first x pass's twiddles
    float2* twM = tw16 + N;
    float2* phx = twM + M;
    float2* phy = phx + M;
    float2* cx = phy + M;
    float2* cy = cx + M;
    float2* twq = cy + M;                            // W_256^{n2 (kly + q)} at [n2][q]: the group sums' twiddles
    float2* ty1 = twq + 4 * M;                       // the first y pass's twiddles at [j][r] (see there)
    float* hgx = reinterpret_cast<float*>(ty1 + 64); // u_m(x'_i) dx' at [m][i]
    float* hgy = hgx + k2G * M;                      // u_n(y'_j) dy' at [j][n] (n fastest, k2G wide); TC: B operand
    int* mlo = reinterpret_cast<int*>(hgy + k2G * M);
    int* mhi = mlo + M;
    int* mdm = mhi + M;
    int* mdn = mdm + k2G * (k2G + 1) / 2;
    float2* Z = buf2;                                // x spectra [u][k] of the packed rows, natural order
    float2* B = work;                                // box columns [c][n1] of the current group
    float2* acc = buf2;                              // the window spectrum [c][q] after the last group
    float2* win = work;                              // window [x position][q] during the inverse
    float2* part = buf2;                             // y-contraction partial sums [QB][G][M] during the epilogue
    const int tid = threadIdx.x;
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    const CUtensorMap* tmap = pol == 0 ? &tmap0 : &tmap1;
    const int G = P.groups, modes = P.modes;
    const int klx = pd.klx, kly = pd.kly;
    for (int i = tid; i < N; i += NT) {
        twN[i] = P.tw_fwd_n[i];
        tw16[i] = P.tw_fwd_n[((i >> 4) * (i & 15)) & (N - 1)];
    }
    for (int i = tid; i < M; i += NT) {
        twM[i] = P.tw_inv_m[i];
        phx[i] = pd.phase_x[i];
        phy[i] = cscale(pd.phase_y[i], 0.5f);   // with the 1/2 of the real-spectra separation
        cx[i] = pd.corr_x[i];
        cy[i] = pd.corr_y[i];
        mlo[i] = pd.mask_lo[i];
        mhi[i] = pd.mask_hi[i];
    }
    for (int i = tid; i < 4 * M; i += NT) twq[i] = P.tw_fwd_n[((i / M) * (kly + i % M)) & (N - 1)];
    for (int i = tid; i < 64; i += NT) {
        // output r of first-pass task j is input j of second-pass block r; its twiddle W_64^{j r} carries the factor
        // W_4^{-j tr(r)} that rotates that block's four outputs by tr(r) = ((r - kly) mod 64) / 16 (see the second
        // pass)
        const int j = i >> 4, r = i & 15, tr = ((r - kly) & 63) >> 4;
        ty1[i] = P.tw_fwd_n[(4 * j * r - 64 * j * tr) & (N - 1)];
    }
    for (int i = tid; i < G * M; i += NT) hgx[i] = pd.hg_x[i];
    if constexpr (TC) {
        // B operand: the host's bf16 hi / lo planes of u_n(y'_j) dy' (rows n < 16, K = j), K permuted to kappa
        __nv_bfloat16* bop = reinterpret_cast<__nv_bfloat16*>(hgy);
        const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(pd.hgy_tc);
        for (int t = tid; t < 2 * k2G * M; t += NT) {
            const int hl = t / (k2G * M), rem = t - hl * k2G * M, n = rem / M, kap = rem - n * M;
            const int j = kap / MR1 + MR0 * (kap % MR1);
            bop[hl * k2G * M + umma_off(n, kap, M)] =
                G > 0 ? src[(size_t)hl * P.tc_np * M + umma_off(n, j, M)] : __float2bfloat16_rn(0.f);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (tid < 32) tmem_alloc(smem_u32(&tmem_slot), kTcCols);
    } else {
        for (int i = tid; i < k2G * M; i += NT) {
            const int j = i / k2G, n = i - j * k2G;
            hgy[i] = n < G ? pd.hg_y[n * M + j] : 0.f;
        }
    }
    for (int i = tid; i < modes; i += NT) {
        mdm[i] = P.mode_m[i];
        mdn[i] = P.mode_n[i];
    }
    const uint32_t mb = smem_u32(&mbar), dst = smem_u32(smem_raw);
    const int fstride = gridDim.x / P.pols;
    const int x0 = A.x0[pol], xo = A.xo[pol];
    int b = blockIdx.x / P.pols;
    if (tid == 0) {
        abort_flag = 0;
        if constexpr (TC) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_mma)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (b < A.count) stage_group(tmap, dst, mb, x0, 0, b);
    }
    __syncthreads();
    uint32_t parity = 0;
    bool aborted = false;
    uint32_t tmem = 0, mma_parity = 0;
    bool tc_ok = true;                           // TC: every MMA wait so far completed
    if constexpr (TC) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        tmem = tmem_slot;
    }
    // the second y pass: task k of this thread is box column c = t mod M, block blk = t / M of t = tid + k NT; its
    // outputs k1 = blk + 16 r2 (r2 < 4) feed the box rows q with kly + q = k1 mod 64.  With (blk - kly) mod 64 =
    // s + 16 tr (s < 16), those are the six rows q = s + 16 m (m < 6), row m fed by output r2 = (m - tr) mod 4;
    // the first pass's twiddles rotate each block's outputs by tr, so output m mod 4 feeds row m.  The rows' sums
    // over the four groups stay in registers
    constexpr int YT = 16 * M / NT;
    static_assert(16 * M % NT == 0 && M == 96, "whole second-pass tasks per thread; six rows per task");
    for (; b < A.count && !aborted; b += fstride) {
        const int f = b;
        float2 ya[YT][6];
        for (int n2 = 0; n2 < 4; ++n2) {
            if (!mbar_wait_bounded(mb, parity)) abort_flag = 1;
            __syncthreads();
            if (abort_flag) {
                if (tid == 0 && P.status) atomicOr(P.status, 1);
                aborted = true;
                break;
            }
            parity ^= 1u;

            // ------------------------------------------------------------ x pass 1: radix 16 from the staged rows
            {
                // the two half-warps take rows u and u + 2 (their staged rows 8 banks apart)
                const int w = tid >> 5, j = tid & 15;
                const int u = 4 * (w >> 1) + (w & 1) + 2 * ((tid >> 4) & 1);
                const uint16_t* ra = stg + u * k2BoxW + xo + j;                        // row n1 = u, box 0
                const uint16_t* rb = ra + 32 * k2BoxW;                                 // row n1 = u + 32
                const uint16_t* sa = ra + k2Rows * k2BoxW - 128;                       // box 1 (columns from 128)
                const uint16_t* sb = rb + k2Rows * k2BoxW - 128;
                float2 v[16];
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = make_float2((float)ra[16 * r], (float)rb[16 * r]);
#pragma unroll
                for (int r = 8; r < 16; ++r) v[r] = make_float2((float)sa[16 * r], (float)sb[16 * r]);
                if (pd.cal) {
                    // reference calibration: window pixel (x, y) times sqrt(max cal / cal), from the L2-resident table
                    const float* ka = pd.cal + (4 * u + n2) * N + j;
                    const float* kb = pd.cal + (4 * (u + 32) + n2) * N + j;
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        v[r].x *= __ldg(ka + 16 * r);
                        v[r].y *= __ldg(kb + 16 * r);
                    }
                }
                dft16<false>(v);
#pragma unroll
                for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw16[r * 16 + j]);
#pragma unroll
                for (int r = 0; r < 16; ++r) work[u * k2PW + j + 16 * r] = v[r];
            }
            // the staged rows have been read (into registers) by every thread once the barrier completes; the next
            // tensor copies into the buffer are issued after it (a read-before-write across the proxies, ordered by
            // the barrier alone, as tensor-copy pipelines release a consumed stage)
            __syncthreads();
            if (tid == 0) {
                if (n2 < 3)
                    stage_group(tmap, dst, mb, x0, n2 + 1, f);
                else if (b + fstride < A.count)
                    stage_group(tmap, dst, mb, x0, 0, f + fstride);
            }

            // ------------------------------------------------------------ x pass 2: radix 16, natural order out
            {
                // block blk's outputs are frequencies blk + 16 r of packed row u
                const int u = tid & 31, blk = tid >> 5;
                float2 v[16];
                const float2* row = work + u * k2PW + 16 * blk;
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = row[r];
                dft16<false>(v);
#pragma unroll
                for (int r = 0; r < 16; ++r) Z[u * k2PW + blk + 16 * r] = v[r];
            }
            __syncthreads();

            // ------------------------------------------------------------ y pass 1: radix 16 over n1 (span 64)
            if (tid < 4 * M) {
                // box column c, frequency k = klx + c: packed row u gives rows n1 = u (Z(k) + conj Z(-k)) and
                // n1 = u + 32 (-i (Z(k) - conj Z(-k))), inputs r and r + 8 of this task (u = j + 4 r, r < 8)
                const int c = tid % M, j = tid / M;
                const int kx = (klx + c) & (N - 1), km = (N - kx) & (N - 1);
                float2 v[16];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float2 zk = Z[(j + 4 * r) * k2PW + kx];
                    const float2 zm = Z[(j + 4 * r) * k2PW + km];
                    v[r] = make_float2(zk.x + zm.x, zk.y - zm.y);
                    v[r + 8] = make_float2(zk.y + zm.y, zm.x - zk.x);
                }
                float2* col = B + c * k2PB + j;
                dft16<false>(v);
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], ty1[j * 16 + r]);   // W_64^{j r} W_4^{-j tr(r)}
#pragma unroll
                for (int r = 0; r < 16; ++r) col[4 * r] = v[r];
            }
            __syncthreads();

            // ------------------------------------------------------------ y pass 2: radix 4, accumulate
#pragma unroll
            for (int k = 0; k < YT; ++k) {
                const int blk = (tid + k * NT) / M, c = (tid + k * NT) % M;
                const int qs = (blk - kly) & 15;
                const float2* col = B + c * k2PB + 4 * blk;
                // the inputs carry W_4^{-n tr}, so output m is the one of frequency k1 = blk + 16 ((m - tr) mod 4)
                float2 o[4] = {col[0], col[1], col[2], col[3]};
                dft4<false>(o[0], o[1], o[2], o[3]);
                const float2* tq = twq + n2 * M + qs;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    if (n2 == 0)
                        ya[k][m] = o[m & 3];
                    else
                        ya[k][m] = cadd(ya[k][m], cmul(o[m & 3], tq[16 * m]));
                }
            }
            // (the next group's wait ends in a barrier before anything here is overwritten)
        }
        if (aborted) break;
        // the window: the circular mask and the beam-centre phase on the summed spectrum, written [c][q]
#pragma unroll
        for (int k = 0; k < YT; ++k) {
            const int blk = (tid + k * NT) / M, c = (tid + k * NT) % M;
            const int qs = (blk - kly) & 15;
            const float2 px = phx[c];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int q = qs + 16 * m;
                acc[c * k2PA + q] = (c >= mlo[q] && c <= mhi[q]) ? cmul(cmul(ya[k][m], px), phy[q]) : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();

        // ---------------------------------------------------------------- inverse transforms
        // x, first DIT pass (radix 12, span 12): window position blk MR1 + r holds box column blk + MR0 r
        for (int t = tid; t < MR0 * M; t += NT) {
            const int q = t % M, blk = t / M;
            float2 v[MR1];
#pragma unroll
            for (int r = 0; r < MR1; ++r) v[r] = acc[(blk + MR0 * r) * k2PA + q];
            dft12<true>(v);
#pragma unroll
            for (int r = 0; r < MR1; ++r) win[(blk * MR1 + r) * k2PA + q] = v[r];
        }
        __syncthreads();
        spass<MR0, true, true, M, M, M, k2PA, 1, NT>(win, twM, tid);
        __syncthreads();
        spass<MR0, true, false, M, M, M, 1, k2PA, NT>(win, twM, tid);
        __syncthreads();

        // ---------------------------------------------------------------- last y pass, correction, field, y overlap
        // The last DIF pass (span MR1, no twiddles) leaves output j = blk + MR0 r at position blk MR1 + r of column
        // i; it is corrected in registers, written to the field (coalesced along i) and contracted with u_n(y'_j)
        // into part[qb][n][i] over row blocks qb and MR0 - qb (block 0 with MR0 / 2), whose rows mirror each other
        // (M - j): the even modes contract sums of mirrored rows, the odd ones differences.
        const bool ov = A.coefs && G > 0;
        {
            float2* fld = A.fields ? A.fields + (size_t)(f * P.pols + pol) * M * M : nullptr;
            for (int t = tid; t < M * QB; t += NT) {
                const int i = t % M, qb = t / M;
                const float2 ci = cx[i];
                if constexpr (TC) {
                    // one row block at a time (no mirrored pairs): field, then the A operand: rows j = blk + MR0 r
                    // sit at K positions MR1 blk + r of rows i (real parts) and M + i (imaginary parts), hi plane
                    // then lo plane
                    __nv_bfloat16* aop = reinterpret_cast<__nv_bfloat16*>(buf2);
#pragma unroll 1
                    for (int bb = 0; bb < BPQ; ++bb) {
                        const int blk = qb == 0 ? bb * (MR0 / 2) : (bb == 0 ? qb : MR0 - qb);
                        float2 w[MR1];
#pragma unroll
                        for (int r = 0; r < MR1; ++r) w[r] = win[i * k2PA + blk * MR1 + r];
                        dft12<true>(w);
#pragma unroll
                        for (int r = 0; r < MR1; ++r) {
                            const int j = blk + MR0 * r;
                            w[r] = cmul(cmul(w[r], ci), cy[j]);
                            if (fld && DH_IN(P.status, (long long)j * M + i, (long long)M * M, kSiteFusedField)) fld[j * M + i] = w[r];
                        }
                        if (ov) {
                            uint32_t hr[MR1 / 2], lr[MR1 / 2], hm[MR1 / 2], lm[MR1 / 2];
#pragma unroll
                            for (int t2 = 0; t2 < MR1 / 2; ++t2) {
                                split_pair(w[2 * t2].x, w[2 * t2 + 1].x, hr[t2], lr[t2]);
                                split_pair(w[2 * t2].y, w[2 * t2 + 1].y, hm[t2], lm[t2]);
                            }
                            store_run12(aop, i, MR1 * blk, hr);
                            store_run12(aop, M + i, MR1 * blk, hm);
                            store_run12(aop + 2 * M * M, i, MR1 * blk, lr);
                            store_run12(aop + 2 * M * M, M + i, MR1 * blk, lm);
                        }
                    }
                    continue;
                }
                float2 v[BPQ][MR1];
#pragma unroll
                for (int bb = 0; bb < BPQ; ++bb) {
                    const int blk = qb == 0 ? bb * (MR0 / 2) : (bb == 0 ? qb : MR0 - qb);
#pragma unroll
                    for (int r = 0; r < MR1; ++r) v[bb][r] = win[i * k2PA + blk * MR1 + r];
                    dft12<true>(v[bb]);
#pragma unroll
                    for (int r = 0; r < MR1; ++r) {
                        const int j = blk + MR0 * r;
                        v[bb][r] = cmul(cmul(v[bb][r], ci), cy[j]);
                        if (fld && DH_IN(P.status, (long long)j * M + i, (long long)M * M, kSiteFusedField)) fld[j * M + i] = v[bb][r];
                    }
                }
                if (ov) {
                    float2 sp[MR1 + 1], sm[MR1 + 1];
                    int jr[MR1 + 1];
                    if (qb == 0) {
                        // block 0 (rows MR0 r) pairs r with MR1 - r; row 0 has no mirror and row M/2 is its own (odd
                        // modes vanish there); block MR0/2 pairs r with MR1 - 1 - r
                        int w = 0;
#pragma unroll
                        for (int r = 1; r < MR1 / 2; ++r, ++w) {
                            sp[w] = cadd(v[0][r], v[0][MR1 - r]);
                            sm[w] = csub(v[0][r], v[0][MR1 - r]);
                            jr[w] = MR0 * r;
                        }
                        sp[w] = sm[w] = v[0][0];
                        jr[w++] = 0;
                        sp[w] = sm[w] = v[0][MR1 / 2];
                        jr[w++] = M / 2;
#pragma unroll
                        for (int r = 0; r < MR1 / 2; ++r, ++w) {
                            sp[w] = cadd(v[1][r], v[1][MR1 - 1 - r]);
                            sm[w] = csub(v[1][r], v[1][MR1 - 1 - r]);
                            jr[w] = MR0 / 2 + MR0 * r;
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
                    for (int n4 = 0; n4 < k2G; n4 += 4) {
                        if (n4 < G) {
                            float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                           make_float2(0.f, 0.f)};
#pragma unroll
                            for (int w = 0; w < MR1 + 1; ++w) {
                                if (w < nu) {
                                    const float4 u = *reinterpret_cast<const float4*>(hgy + jr[w] * k2G + n4);
                                    a[0].x = fmaf(u.x, sp[w].x, a[0].x);
                                    a[0].y = fmaf(u.x, sp[w].y, a[0].y);
                                    a[1].x = fmaf(u.y, sm[w].x, a[1].x);
                                    a[1].y = fmaf(u.y, sm[w].y, a[1].y);
                                    a[2].x = fmaf(u.z, sp[w].x, a[2].x);
                                    a[2].y = fmaf(u.z, sp[w].y, a[2].y);
                                    a[3].x = fmaf(u.w, sm[w].x, a[3].x);
                                    a[3].y = fmaf(u.w, sm[w].y, a[3].y);
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
        if constexpr (TC) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        float* Ts = reinterpret_cast<float*>(work);   // TC: T[n][r] over the consumed window, [16][kTsPitch]
        if constexpr (TC) {
            if (ov) {
                // y contraction: hi hi + hi lo + lo hi per 16-wide K step, two 128-row tiles, FP32 accumulation in
                // tensor memory (tile t in columns 16 t .. 16 t + 15)
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t mbm = smem_u32(&mbar_mma);
                if (tid == 0 && tc_ok) {
                    const uint32_t a_hi = smem_u32(buf2), a_lo = a_hi + 4 * M * M;
                    const uint32_t b_hi = smem_u32(hgy), b_lo = b_hi + 2 * k2G * M;
                    constexpr uint32_t idesc = umma_idesc_bf16(128, k2G);
                    const uint32_t lbo = 128, sbo = 16 * M;
#pragma unroll
                    for (int tile = 0; tile < 2; ++tile) {
                        const uint32_t ao = tile * 16 * sbo;
#pragma unroll
                        for (int ks = 0; ks < M / 16; ++ks) {
                            const uint32_t ko = ks * 256, d = tmem + tile * k2G;
                            umma_bf16(d, umma_desc(a_hi + ao + ko, lbo, sbo), umma_desc(b_hi + ko, lbo, sbo), idesc, ks > 0);
                            umma_bf16(d, umma_desc(a_hi + ao + ko, lbo, sbo), umma_desc(b_lo + ko, lbo, sbo), idesc, 1);
                            umma_bf16(d, umma_desc(a_lo + ao + ko, lbo, sbo), umma_desc(b_hi + ko, lbo, sbo), idesc, 1);
                        }
                    }
                    umma_commit(mbm);
                }
                bool done = false;
                if (tc_ok) {   // the same for every thread
                    done = bounded_mbar_wait(mbm, mma_parity, k2WaitLimit);
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
                    for (int n = 0; n < k2G; ++n) Ts[n * kTsPitch + 32 * warp + lane] = tc_ok ? tv[n] : __int_as_float(0x7fc00000);
                    if (warp < 2) {
                        // the second tile's rows 128 .. 191 (imaginary parts of columns 32 .. 95)
                        if (tc_ok) tmem_ld16(tmem + k2G + ((uint32_t)(32 * warp) << 16), tv);
#pragma unroll
                        for (int n = 0; n < k2G; ++n)
                            Ts[n * kTsPitch + 128 + 32 * warp + lane] = tc_ok ? tv[n] : __int_as_float(0x7fc00000);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncthreads();
            }
        } else {
            if (ov) {
                // T[n][i] = sum_qb part[qb][n][i] (groups added in a fixed order), in place of group 0
                for (int t = tid; t < G * M; t += NT) {
                    float2 s = part[t];
#pragma unroll
                    for (int q = 1; q < QB; ++q) s = cadd(s, part[q * G * M + t]);
                    part[t] = s;
                }
            }
            __syncthreads();
        }

        // ---------------------------------------------------------------- HG overlap, x contraction
        if (ov) {
            // c_mn = sum_i u_m(x'_i) T[n][i]: eight threads per mode, thread s taking the column pairs i = 2s + 16h,
            // then a fixed shuffle tree
            float2* cf = A.coefs + (size_t)(f * P.pols + pol) * modes;
            const int s8 = tid & 7;
            for (int t0 = tid & ~31; t0 < modes * 8; t0 += NT) {
                const int k = (t0 + (tid & 31)) >> 3;
                float2 sum = make_float2(0.f, 0.f);
                if (TC && k < modes) {
                    const float* um = hgx + mdm[k] * M;
                    const float* tr = Ts + mdn[k] * kTsPitch;
#pragma unroll
                    for (int h = 0; h < M / 16; ++h) {
                        const int i = 2 * s8 + 16 * h;
                        const float2 u = *reinterpret_cast<const float2*>(um + i);
                        sum.x = fmaf(u.x, tr[i], sum.x);
                        sum.y = fmaf(u.x, tr[M + i], sum.y);
                        sum.x = fmaf(u.y, tr[i + 1], sum.x);
                        sum.y = fmaf(u.y, tr[M + i + 1], sum.y);
                    }
                } else if (k < modes) {
                    const float* um = hgx + mdm[k] * M;
                    const float2* tn = part + mdn[k] * M;
#pragma unroll
                    for (int h = 0; h < M / 16; ++h) {
                        const int i = 2 * s8 + 16 * h;
                        const float2 u = *reinterpret_cast<const float2*>(um + i);
                        const float4 v = *reinterpret_cast<const float4*>(tn + i);
                        sum.x = fmaf(u.x, v.x, sum.x);
                        sum.y = fmaf(u.x, v.y, sum.y);
                        sum.x = fmaf(u.y, v.z, sum.x);
                        sum.y = fmaf(u.y, v.w, sum.y);
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
                    sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
                }
                if (s8 == 0 && k < modes && DH_IN(P.status, k, modes, kSiteFusedCoef)) cf[k] = sum;
            }
        }
        __syncthreads();
    }
    // a tensor copy still in flight (only after an expired wait) must land before the block exits
    if (aborted && tid == 0) mbar_wait_bounded(mb, parity);
    if constexpr (TC) {
        // MMAs still in flight (only after an expired wait: the last ones issued) must complete before their tensor
        // memory is freed
        if (!tc_ok && tid == 0) bounded_mbar_wait(smem_u32(&mbar_mma), mma_parity ^ 1u, k2WaitLimit);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (tid < 32) tmem_free(tmem, kTcCols);
    }
}

}  // namespace dhk

namespace dh {

static int g_256_sms[64] = {0};
static int g_256_bps[64] = {0};
static PFN_cuTensorMapEncodeTiled_v12000 g_256_encode = nullptr;

bool use_fused256(const dhk::Plan& P) {
    if (P.n != dhk::k2N || P.ny != dhk::k2N || P.m != dhk::k2M || P.my != dhk::k2M || P.groups > dhk::k2G || P.pols > 2)
        return false;
    if (P.precision == DH_PRECISION_SPLIT_BF16)   // the tensor-core variant: B operand of 16 rows
        return P.groups == 0 || (P.tc_np == dhk::k2G && P.pol[0].hgy_tc && (P.pols < 2 || P.pol[1].hgy_tc));
    return P.precision == DH_PRECISION_FP32;
}

cudaError_t fused256_init() {
    if (!g_256_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        g_256_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    cudaError_t e = cudaFuncSetAttribute(dhk::k_fused256<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dhk::F256Smem::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(dhk::k_fused256<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dhk::F256Smem::bytes);
}

int launch_fused256(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                    cudaStream_t st, dhk::StageTimer* tm) {
    const int dev = H->device;
    if (dev < 0 || dev >= 64) return fail(DH_ERROR_ERROR, "device index out of range");
    if (batch < 1) return DH_SUCCESS;
    if (dtype != DH_DTYPE_U16) return fail(DH_ERROR_INVALIDARGUMENT, "the 256 x 256 fused kernel reads uint16 frames");
    if (!g_256_encode) return fail(DH_ERROR_ERROR, "tensor-map encoder unavailable");
    if (!g_256_sms[dev]) {
        int n = 0;
        cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device attribute");
        g_256_sms[dev] = n;
    }
    if (!g_256_bps[dev]) {
        int n = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dhk::k_fused256<false>, dhk::k2NT, dhk::F256Smem::bytes);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        g_256_bps[dev] = n > 0 ? n : 1;
    }
    // per polarisation, the window rows as a 4-D tensor [frame][n1 < 64][n2 < 4][x]: window row 4 n1 + n2 of frame
    // f at (frames + f H W + (oy + 4 n1 + n2) W) (every row inside the frame); one box = 64 rows n1 of one group
    // n2 by 136 columns
    const size_t esz = 2;
    CUtensorMap tmap[DH_MAX_POLS];
    std::memset(tmap, 0, sizeof tmap);
    for (int p = 0; p < P.pols; ++p) {
        const cuuint64_t gdim[4] = {(cuuint64_t)P.width, 4, (cuuint64_t)dhk::k2Rows, (cuuint64_t)batch};
        const cuuint64_t gstride[3] = {(cuuint64_t)P.width * esz, (cuuint64_t)P.width * esz * 4,
                                       (cuuint64_t)P.width * P.height * esz};
        const cuuint32_t box[4] = {(cuuint32_t)dhk::k2BoxW, 1, (cuuint32_t)dhk::k2Rows, 1};
        const cuuint32_t estride[4] = {1, 1, 1, 1};
        void* base = (unsigned char*)const_cast<void*>(frames) + (size_t)P.pol[p].oy * P.width * esz;
        CUresult cr = g_256_encode(&tmap[p], CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, base, gdim, gstride, box, estride,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return fail(DH_ERROR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    }
    if (P.pols == 1) tmap[1] = tmap[0];
    dhk::F256Args A;
    std::memset(&A, 0, sizeof A);
    A.count = batch;
    for (int p = 0; p < P.pols; ++p) {
        const int ox = P.pol[p].ox;               // window origins are >= 0
        A.x0[p] = (ox / 8) * 8;                   // 16-byte aligned staging origin
        A.xo[p] = ox - A.x0[p];
    }
    A.fields = (float2*)fields;
    A.coefs = (float2*)coefs;
    // a persistent grid of every resident block; each block serves one polarisation
    const int resident = g_256_sms[dev] * g_256_bps[dev];
    const long long per_pol = std::min<long long>(batch, std::max(1, resident / P.pols));
    const int grid = (int)per_pol * P.pols;
    if (tm) tm->start(st);
    const bool tc = P.precision == DH_PRECISION_SPLIT_BF16;
    if (tc)
        dhk::k_fused256<true><<<grid, dhk::k2NT, dhk::F256Smem::bytes, st>>>(P, A, tmap[0], tmap[1]);
    else
        dhk::k_fused256<false><<<grid, dhk::k2NT, dhk::F256Smem::bytes, st>>>(P, A, tmap[0], tmap[1]);
    if (tm) tm->stop(st, tc ? "k_fused256_tc" : "k_fused256");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DH_SUCCESS;
}

}  // namespace dh
