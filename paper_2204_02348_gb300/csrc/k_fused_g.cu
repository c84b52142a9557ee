// Group-transform fused path for 128 x 128 windows with 64 x 64 fields and the FP32 overlap: one thread block
// reconstructs one (frame, polarisation) window at a time in shared memory, persistent over windows (the guide's
// pipeline steps 1-3 and digHoloProcessRemoveTilt).  Every 1-D transform is owned by one group of eight threads
// (a quarter of a warp): its exchanges go through shared memory with warp barriers only, and the block
// synchronises five times per window.
//
//   Y   y transform of the 64 packed column pairs (window columns 2c and 2c + 1 as one complex column), radix 16
//       over rows n1 + 8 n2 in registers, twiddles, an exchange through the group's own column of the box-row
//       buffer, radix 8 over n1; the lane owning frequencies k2 = t, 16 - t (0 and 8 for lane 0) holds every
//       Z(k) beside its mirror Z(-k) and writes the separated spectra of the two real columns for the box rows
//       the circular window touches.
//   X   per box row that the window touches (rows it misses are zero and skipped), the x transform (radix 8 over
//       x = a + 16 b, twiddles, exchange, radix 16 over a: lane t ends with X(t + 8 d), d < 16), the window
//       selection (of X(t + 8 d) and X(t + 8 (d + 8)) exactly one lies in the box), mask and x beam-centre
//       phase, and the 64-point x inverse in the same lane group: radix 8 over the eight kept bins of the lane,
//       the twiddle exp(2 pi i (t - k_lx) x0 / 64), an exchange, radix 8 over the lanes.  The result is scaled
//       by the y beam-centre phase and by the x correction (residual tilt, defocus, and the factor
//       exp(-2 pi i k_lx x1 / 8) the box offset leaves).
//   YI  per field column, the 64-point y inverse (radix 8 x 8 with an exchange), the y correction and the
//       field write.
//   overlap  y contraction over mirrored row pairs (the parity of u_n on the centred grid) by 256 threads, then
//       x contraction with eight threads per mode and a fixed shuffle tree (deterministic, no atomics).
//
// Shared memory: the staging buffer of the next window (filled by a tensor copy while the current one is
// processed), the 64 x 128 complex box-row buffer (16-byte chunks swizzled by row & 7, so the column-wise and
// row-wise accesses of every stage are free of bank conflicts) and the tables: ~110 KB for uint16 frames, two
// blocks per SM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "fft.cuh"
#include "runtime.hpp"
#include "sync.cuh"

namespace dhk {

constexpr int kGN = 128;           // window size of this path
constexpr int kGM = 64;            // field size
constexpr int kGNT = 512;          // threads per block: 64 groups of eight
constexpr int kGG = 16;            // most HG groups
constexpr int kGModes = kGG * (kGG + 1) / 2;
constexpr long kGWaitLimit = 1L << 24;

template <typename T>
struct GStage {
    static constexpr int ALIGN = 16 / (int)sizeof(T);   // elements per 16 bytes
    static constexpr int W = kGN + ALIGN;                // staged row: the window plus the alignment slack
    static constexpr int BYTES = kGN * W * (int)sizeof(T);
    static_assert(BYTES % 128 == 0, "the box-row buffer starts on a 128-byte boundary");
};

// Shared-memory layout (bytes): staging, box rows [64][128] float2, then the tables.
template <typename T>
struct GSmem {
    static constexpr size_t R1 = GStage<T>::BYTES;
    static constexpr size_t TY = R1 + (size_t)kGM * kGN * 8;   // float2 [16 k2][8 t]: W128^(t k2)
    static constexpr size_t TX = TY + 128 * 8;                  // float2 [8 c][16 a]: W128^(a c)
    static constexpr size_t TD = TX + 128 * 8;                  // float2 [8 x0][8 t]: exp(+2 pi i (t - klx) x0 / 64)
    static constexpr size_t TI = TD + 64 * 8;                   // float2 [8 y0][8 u]: exp(+2 pi i u y0 / 64)
    static constexpr size_t PXL = TI + 64 * 8;                  // float2 [8 m][8 t]: x phase of the lane's bin m
    static constexpr size_t PHY = PXL + 64 * 8;                 // float2 [64]: y phase x 1/2
    static constexpr size_t CXK = PHY + 64 * 8;                 // float2 [64]: x correction x exp(-2 pi i klx x1 / 8)
    static constexpr size_t CY = CXK + 64 * 8;                  // float2 [64]: y correction
    static constexpr size_t HGX = CY + 64 * 8;                  // float [16][64]: u_m(x'_i) dx'
    static constexpr size_t HY = HGX + (size_t)kGG * kGM * 4;   // float [33][16]: u_n(y'_j) dy', j <= 32
    static constexpr size_t MD = HY + 33 * kGG * 4;             // int [2][kGModes]: mode orders m, n
    static constexpr size_t bytes = MD + 2 * (size_t)kGModes * 4;
};

// Element of box row r, column c (complex index): 16-byte chunks XOR-swizzled by r & 7.
__device__ __forceinline__ int r1_at(int r, int c) { return r * kGN + (c ^ ((r & 7) << 1)); }

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 f4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// One thread: expect the window's bytes on the mbarrier and start the tensor copy of frame f.
__device__ __forceinline__ void g_stage(const CUtensorMap* tmap, uint32_t dst, uint32_t mbar, int x0, int y0, int f,
                                        int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0), "r"(f), "r"(mbar)
        : "memory");
}

// Stage X's box-row slot of group gi: slots permuted within each eight groups so that the two groups of a
// half-warp hold rows four apart (their 8-byte stores then fall in distinct banks).
__device__ __forceinline__ int g_row_slot(int gi) { return (gi & ~7) | ((gi & 1) << 2) | ((gi >> 1) & 3); }

// A shared-memory word read where it is used, not hoisted out of the window loop.
__device__ __forceinline__ uint32_t ld_keep(const void* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }

// y contraction of one column over NT mirrored-pair terms: even modes take the sums sp, odd modes the differences
// sm, each times u_n at the term's table row (row(u) points at u_0..u_15 of that row); the partial sums of modes
// n < G go to row 4 n + qb, column 64 + x of the box-row buffer.
template <int NT, typename RowFn>
__device__ __forceinline__ void g_ycontract(const float2 (&sp)[NT], const float2 (&sm)[NT], RowFn row, int G, float2* r1,
                                            int qb, int x) {
#pragma unroll
    for (int n4 = 0; n4 < kGG; n4 += 4) {
        if (n4 < G) {
            float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                const float4 w = *reinterpret_cast<const float4*>(row(u) + n4);
                a[0].x = fmaf(w.x, sp[u].x, a[0].x);
                a[0].y = fmaf(w.x, sp[u].y, a[0].y);
                a[1].x = fmaf(w.y, sm[u].x, a[1].x);
                a[1].y = fmaf(w.y, sm[u].y, a[1].y);
                a[2].x = fmaf(w.z, sp[u].x, a[2].x);
                a[2].y = fmaf(w.z, sp[u].y, a[2].y);
                a[3].x = fmaf(w.w, sm[u].x, a[3].x);
                a[3].y = fmaf(w.w, sm[u].y, a[3].y);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (n4 + c < G) r1[r1_at(4 * (n4 + c) + qb, kGM + x)] = a[c];
        }
    }
}

struct GArgs {
    int count;                    // frames of the launch (the tensor map's outermost extent)
    int xo[DH_MAX_POLS];          // window origin minus the 16-byte-aligned staging origin, per polarisation
    int x0[DH_MAX_POLS];          // staging origin (16-byte aligned element index), per polarisation
    float2* fields;               // nullable [B][pol][64][64]
    float2* coefs;                // nullable [B][pol][modes]
};

template <typename T>
__global__ void __launch_bounds__(kGNT, sizeof(T) == 2 ? 2 : 1)
    k_fused128g(const __grid_constant__ Plan P, const __grid_constant__ GArgs A, const __grid_constant__ CUtensorMap tmap) {
    using L = GSmem<T>;
    using S = GStage<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    // per-block and per-thread constants of the window loop, kept in shared memory and reloaded by the stage that
    // uses them (fewer registers live across the loop)
    __shared__ int s_qlo, s_nrows;
    __shared__ uint32_t s_blk, s_bits[kGNT];
    const T* stg = reinterpret_cast<const T*>(smem);
    float2* r1 = reinterpret_cast<float2*>(smem + L::R1);
    float2* TY = reinterpret_cast<float2*>(smem + L::TY);
    float2* TX = reinterpret_cast<float2*>(smem + L::TX);
    float2* TD = reinterpret_cast<float2*>(smem + L::TD);
    float2* TI = reinterpret_cast<float2*>(smem + L::TI);
    float2* PXL = reinterpret_cast<float2*>(smem + L::PXL);
    float2* PHY = reinterpret_cast<float2*>(smem + L::PHY);
    float2* CXK = reinterpret_cast<float2*>(smem + L::CXK);
    float2* CY = reinterpret_cast<float2*>(smem + L::CY);
    float* HGX = reinterpret_cast<float*>(smem + L::HGX);
    float* HY = reinterpret_cast<float*>(smem + L::HY);
    int* MDM = reinterpret_cast<int*>(smem + L::MD);
    int* MDN = MDM + kGModes;

    const int tid = threadIdx.x, lane = tid & 31, t = tid & 7;
    const int gi = tid >> 3;                       // group: column pair (Y), box row slot (X), field column (YI)
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    const int G = P.groups, modes = P.modes;
    const int klx = pd.klx, kly = pd.kly;

    // ------------------------------------------------------------------------------------------- tables
    for (int i = tid; i < 128; i += kGNT) {
        TY[i] = P.tw_fwd_n[((i & 7) * (i >> 3)) & (kGN - 1)];
        TX[i] = P.tw_fwd_n[((i & 15) * (i >> 4)) & (kGN - 1)];
    }
    for (int i = tid; i < 64; i += kGNT) {
        const int hi = i >> 3, lo = i & 7;
        const int D = (lo - klx) & (kGN - 1);
        TD[i] = P.tw_inv_m[(D * hi) & (kGM - 1)];
        TI[i] = P.tw_inv_m[(lo * hi) & (kGM - 1)];
        PXL[i] = pd.phase_x[(D + 8 * hi) & (kGM - 1)];
        PHY[i] = cscale(pd.phase_y[i], 0.5f);        // with the 1/2 of the real-spectra separation
        // exp(-2 pi i klx x1 / 8) = conj(exp(+2 pi i 8 (klx x1 mod 8) / 64))
        const float2 w = P.tw_inv_m[8 * ((klx * hi) & 7)];
        CXK[i] = cmul(pd.corr_x[i], make_float2(w.x, -w.y));
        CY[i] = pd.corr_y[i];
    }
    for (int i = tid; i < G * kGM; i += kGNT) HGX[i] = pd.hg_x[i];
    for (int i = tid; i < 33 * kGG; i += kGNT) {
        const int j = i / kGG, n = i - j * kGG;
        HY[i] = n < G ? pd.hg_y[n * kGM + j] : 0.f;
    }
    for (int i = tid; i < modes; i += kGNT) {
        MDM[i] = P.mode_m[i];
        MDN[i] = P.mode_n[i];
    }
    const uint32_t mb = smem_u32(&mbar), dst = smem_u32(smem);
    const int fstride = gridDim.x / P.pols;
    int b = blockIdx.x / P.pols;
    if (tid == 0) {
        // box rows that the circular window touches: [qlo, qlo + nrows)
        int lo = kGM, hi = -1;
        for (int q = 0; q < kGM; ++q)
            if (pd.mask_lo[q] <= pd.mask_hi[q]) {
                lo = min(lo, q);
                hi = max(hi, q);
            }
        s_qlo = hi >= lo ? lo : 0;
        s_nrows = hi >= lo ? hi - lo + 1 : 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (b < A.count) g_stage(&tmap, dst, mb, A.x0[pol], pd.oy, b, S::BYTES);
    }
    __syncthreads();
    {
        const int qlo = s_qlo, nrows = s_nrows;
        // stage Y: 8-row blocks of spectrum rows (k in [8 s, 8 s + 8)) that hold a box row the window touches
        if (tid == 0) {
            uint32_t blk = 0;
            for (int s = 0; s < 16; ++s)
                for (int j = 0; j < 8; ++j)
                    if ((unsigned)(((8 * s + j - kly) & (kGN - 1)) - qlo) < (unsigned)nrows) blk |= 1u << s;
            s_blk = blk;
        }
        // stage X: bits 0-7: bin m of the lane comes from X(t + 8 (m + 8)); bits 8-15: bin m is kept
        const int rho = g_row_slot(gi);
        const int qx = qlo + rho;
        uint32_t bits = 0;
        const int D = (t - klx) & (kGN - 1);
        const int mlo = rho < nrows ? pd.mask_lo[qx] : 1, mhi = rho < nrows ? pd.mask_hi[qx] : 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int s = D + 8 * m, pp = s & (kGM - 1);
            if (s & 64) bits |= 1u << m;
            if (pp >= mlo && pp <= mhi) bits |= 256u << m;
        }
        s_bits[tid] = bits;
    }
    __syncthreads();
    const bool ov = A.coefs != nullptr && G > 0;
    uint32_t parity = 0;

    for (; b < A.count; b += fstride) {
        const bool ok = bounded_mbar_wait(mb, parity, kGWaitLimit);
        parity ^= 1u;

        // ------------------------------------------------------------------------------------------- Y
        {
            const int cp = gi;
            const int xo = A.xo[pol];
            float2 z[16];
            const T* col = stg + xo + 2 * cp;
            if (sizeof(T) == 2 && (xo & 1) == 0) {
#pragma unroll
                for (int n2 = 0; n2 < 16; ++n2) {
                    const uint32_t v = *reinterpret_cast<const uint32_t*>(col + (t + 8 * n2) * S::W);
                    z[n2] = make_float2((float)(v & 0xffffu), (float)(v >> 16));
                }
            } else if (sizeof(T) == 4 && (xo & 1) == 0) {
#pragma unroll
                for (int n2 = 0; n2 < 16; ++n2) z[n2] = *reinterpret_cast<const float2*>(col + (t + 8 * n2) * S::W);
            } else {
#pragma unroll
                for (int n2 = 0; n2 < 16; ++n2) {
                    const T* p = col + (t + 8 * n2) * S::W;
                    z[n2] = make_float2((float)p[0], (float)p[1]);
                }
            }
            if (pd.cal) {
                // reference calibration: window pixel (x, y) times sqrt(max cal / cal), from the L2-resident table
#pragma unroll
                for (int n2 = 0; n2 < 16; ++n2) {
                    const float* k = pd.cal + (t + 8 * n2) * kGN + 2 * cp;
                    z[n2].x *= __ldg(k);
                    z[n2].y *= __ldg(k + 1);
                }
            }
            dft16<false>(z);
#pragma unroll
            for (int k2 = 1; k2 < 16; ++k2) z[k2] = cmul(z[k2], TY[k2 * 8 + t]);
            // exchange through the group's column pair of the box-row buffer: (n1, k2) at row 8 j + (n1 ^ j ^ sw),
            // j = k2 / 2, the pair k2 = 2 j, 2 j + 1 in one 16-byte chunk
            const int sw = (gi & 1) << 2;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = 8 * j + ((t ^ j ^ sw) & 7);
                *reinterpret_cast<float4*>(r1 + r1_at(r, 2 * cp)) = f4(z[2 * j], z[2 * j + 1]);
            }
            __syncwarp();
            const int ka = t, kb = t ? 16 - t : 8;
            const int qlo = (int)ld_keep(&s_qlo), nrows = (int)ld_keep(&s_nrows);
            const uint32_t blk = ld_keep(&s_blk);
            float2 y1[8], y2[8];
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const int ja = ka >> 1, jb = kb >> 1;
                const int ra = 8 * ja + ((n1 ^ ja ^ sw) & 7), rb = 8 * jb + ((n1 ^ jb ^ sw) & 7);
                y1[n1] = r1[r1_at(ra, 2 * cp + (ka & 1))];
                y2[n1] = r1[r1_at(rb, 2 * cp + (kb & 1))];
            }
            __syncwarp();
            dft8<false>(y1);   // Z(ka + 16 k1)
            dft8<false>(y2);   // Z(kb + 16 k1)
            // separation: A(k) = Z(k) + conj Z(-k) (column 2 cp), B(k) = -i (Z(k) - conj Z(-k)) (column 2 cp + 1),
            // both times 2; the mirror of ka + 16 k1 is kb + 16 (7 - k1) (lane 0: 16 ((8 - k1) mod 8))
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) {
#pragma unroll
                for (int set = 0; set < 2; ++set) {
                    if (blk & (1u << (2 * k1 + set))) {
                        const float2 zk = set ? y2[k1] : y1[k1];
                        float2 zm;
                        if (set == 0) zm = t ? y2[7 - k1] : y1[(8 - k1) & 7];
                        else zm = t ? y1[7 - k1] : y2[7 - k1];
                        const int k = (set ? kb : ka) + 16 * k1;
                        const int q = (k - kly) & (kGN - 1);
                        if ((unsigned)(q - qlo) < (unsigned)nrows)
                            *reinterpret_cast<float4*>(r1 + r1_at(q, 2 * cp)) =
                                make_float4(zk.x + zm.x, zk.y - zm.y, zk.y + zm.y, zm.x - zk.x);
                    }
                }
            }
        }
        // the staged window has been read: order those reads before the next tensor copy into the buffer
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0 && P.status) atomicOr(P.status, 1);
            break;
        }
        if (tid == 0 && b + fstride < A.count) g_stage(&tmap, dst, mb, A.x0[pol], pd.oy, b + fstride, S::BYTES);

        // ------------------------------------------------------------------------------------------- X
        const int rho = g_row_slot(gi);
        const bool xact = rho < (int)ld_keep(&s_nrows);
        // the warp barriers of this stage cover the groups of the warp that hold a box row
        const unsigned wm = __ballot_sync(0xffffffffu, xact);
        if (xact) {
            const int q = (int)ld_keep(&s_qlo) + rho, s7 = q & 7;
            const uint32_t bits = ld_keep(&s_bits[tid]);
            float2* row = r1 + q * kGN;
            float2 u[8], v[8];
#pragma unroll
            for (int bb = 0; bb < 8; ++bb) {
                const float4 w = *reinterpret_cast<const float4*>(row + ((2 * t + 16 * bb) ^ (s7 << 1)));
                u[bb] = lo2(w);   // x = 2 t + 16 b
                v[bb] = hi2(w);   // x = 2 t + 1 + 16 b
            }
            dft8<false>(u);
            dft8<false>(v);
#pragma unroll
            for (int c = 1; c < 8; ++c) {
                const float4 w = *reinterpret_cast<const float4*>(TX + c * 16 + 2 * t);
                u[c] = cmul(u[c], lo2(w));
                v[c] = cmul(v[c], hi2(w));
            }
            __syncwarp(wm);
            // exchange 1 (private to the group): (a, c) with a = 2 t, 2 t + 1 in the chunk 8 c + (t ^ c)
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<float4*>(row + 2 * (8 * c + (t ^ c))) = f4(u[c], v[c]);
            __syncwarp(wm);
            float2 X[16];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const float4 w = *reinterpret_cast<const float4*>(row + 2 * (8 * t + (s ^ t)));
                X[2 * s] = lo2(w);
                X[2 * s + 1] = hi2(w);
            }
            dft16<false>(X);   // X[d] = spectrum at t + 8 d
            // window selection, mask and x phase: bin m of the lane is X[m] or X[m + 8]
            float2 F[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float2 val = (bits & (1u << m)) ? X[m + 8] : X[m];
                F[m] = (bits & (256u << m)) ? cmul(val, PXL[m * 8 + t]) : make_float2(0.f, 0.f);
            }
            dft8<true>(F);
#pragma unroll
            for (int x0 = 1; x0 < 8; ++x0) F[x0] = cmul(F[x0], TD[x0 * 8 + t]);
            __syncwarp(wm);
            // exchange 2 (private): (t, x0) in the chunk (4 x0 + ((t / 2) ^ (x0 / 2 mod 4))) ^ h4, half t mod 2
            const int h4 = (gi & 1) << 2;
#pragma unroll
            for (int x0 = 0; x0 < 8; ++x0) {
                const int Lc = 4 * x0 + ((t >> 1) ^ ((x0 >> 1) & 3));
                row[2 * (Lc ^ h4) + (t & 1)] = F[x0];
            }
            __syncwarp(wm);
            float2 H[8];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int Lc = 4 * t + (s ^ ((t >> 1) & 3));
                const float4 w = *reinterpret_cast<const float4*>(row + 2 * (Lc ^ h4));
                H[2 * s] = lo2(w);
                H[2 * s + 1] = hi2(w);
            }
            dft8<true>(H);   // field column x = t + 8 x1, up to exp(-2 pi i klx x1 / 8)
            __syncwarp(wm);
            const float2 py = PHY[q];
#pragma unroll
            for (int x1 = 0; x1 < 8; ++x1) {
                const int x = t + 8 * x1;
                row[x ^ (s7 << 1)] = cmul(cmul(H[x1], CXK[x]), py);
            }
        }
        __syncthreads();

        // ------------------------------------------------------------------------------------------- YI
        {
            const int x = gi;
            const int qlo = (int)ld_keep(&s_qlo), nrows = (int)ld_keep(&s_nrows);
            float2 e[8];
#pragma unroll
            for (int q1 = 0; q1 < 8; ++q1) {
                const int q = t + 8 * q1;
                e[q1] = ((unsigned)(q - qlo) < (unsigned)nrows) ? r1[q * kGN + (x ^ (t << 1))] : make_float2(0.f, 0.f);
            }
            dft8<true>(e);
#pragma unroll
            for (int y0 = 1; y0 < 8; ++y0) e[y0] = cmul(e[y0], TI[y0 * 8 + t]);
            __syncwarp();
            // exchange through the column: (u, y0) at row 8 y0 + (u ^ y0)
#pragma unroll
            for (int y0 = 0; y0 < 8; ++y0) r1[r1_at(8 * y0 + (t ^ y0), x)] = e[y0];
            __syncwarp();
#pragma unroll
            for (int uu = 0; uu < 8; ++uu) e[uu] = r1[r1_at(8 * t + (uu ^ t), x)];
            dft8<true>(e);   // rows y = t + 8 y1
            float2* fld = A.fields ? A.fields + ((size_t)b * P.pols + pol) * kGM * kGM : nullptr;
#pragma unroll
            for (int y1 = 0; y1 < 8; ++y1) {
                const int y = t + 8 * y1;
                e[y1] = cmul(e[y1], CY[y]);
                if (fld && DH_IN(P.status, (long long)y * kGM + x, (long long)kGM * kGM, kSiteFusedField)) fld[y * kGM + x] = e[y1];
            }
            if (ov) {
                __syncwarp();
#pragma unroll
                for (int y1 = 0; y1 < 8; ++y1) r1[(t + 8 * y1) * kGN + (x ^ (t << 1))] = e[y1];
            }
        }

        if (ov) {
            __syncthreads();
            // ----------------------------------------------------------------------------- y contraction
            // thread (x, qb) contracts rows j = b0 + 8 r and b1 + 8 r (blocks qb and 8 - qb; 0 and 4 for qb = 0),
            // pairing each row j with its mirror 64 - j: even modes take E_j + E_{64-j}, odd modes the difference,
            // with u_n at the row of the pair nearer the centre; partial sums at row 4 n + qb, column 64 + x
            if (tid < 256) {
                const int x = tid & 63, qb = tid >> 6;
                const int b0 = qb, b1 = qb ? 8 - qb : 4;
                float2 v0[8], v1[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    v0[r] = r1[r1_at(b0 + 8 * r, x)];
                    v1[r] = r1[r1_at(b1 + 8 * r, x)];
                }
                if (qb == 0) {
                    // block 0 (rows 8 r) pairs r with 8 - r; row 0 has no mirror on the grid and row 32 is its own
                    // (odd modes vanish there); block 4 (rows 4 + 8 r) pairs r with 7 - r
                    float2 sp[9], sm[9];
#pragma unroll
                    for (int r = 1; r < 4; ++r) {
                        sp[r - 1] = cadd(v0[r], v0[8 - r]);
                        sm[r - 1] = csub(v0[r], v0[8 - r]);
                    }
                    sp[3] = sm[3] = v0[0];
                    sp[4] = sm[4] = v0[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        sp[5 + r] = cadd(v1[r], v1[7 - r]);
                        sm[5 + r] = csub(v1[r], v1[7 - r]);
                    }
                    g_ycontract<9>(sp, sm, [&](int u) { return HY + kGG * (u < 3 ? 8 * (u + 1) : u == 3 ? 0 : u == 4 ? 32 : 4 + 8 * (u - 5)); },
                                   G, r1, qb, x);
                } else {
                    // row qb + 8 r mirrors (8 - qb) + 8 (7 - r); the table row is the one nearer the centre
                    float2 sp[8], sm[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        sp[r] = cadd(v0[r], v1[7 - r]);
                        sm[r] = r < 4 ? csub(v0[r], v1[7 - r]) : csub(v1[7 - r], v0[r]);
                    }
                    const float* h0 = HY + kGG * qb;          // rows qb + 8 r, r < 4
                    const float* h1 = HY + kGG * (8 - qb);    // rows (8 - qb) + 8 (7 - r), r >= 4
                    g_ycontract<8>(sp, sm, [&](int u) { return u < 4 ? h0 + 8 * kGG * u : h1 + 8 * kGG * (7 - u); }, G, r1,
                                   qb, x);
                }
            }
            __syncthreads();
            // ----------------------------------------------------------------------------- x contraction
            // c_mn = sum_i u_m(x'_i) dx' T_n[i], T_n[i] = the four partial sums added in a fixed order: eight
            // threads per mode, thread s taking the column pairs i = 2 s + 16 h, then a fixed shuffle tree
            float2* cf = A.coefs + ((size_t)b * P.pols + pol) * modes;
            const int s8 = tid & 7;
            for (int t0 = tid & ~31; t0 < modes * 8; t0 += kGNT) {
                const int k = (t0 + lane) >> 3;
                float2 acc = make_float2(0.f, 0.f);
                if (k < modes) {
                    const float* um = HGX + MDM[k] * kGM;
                    const int rn = 4 * MDN[k];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int i = 2 * s8 + 16 * h;
                        const float2 uv = *reinterpret_cast<const float2*>(um + i);
                        float4 v = *reinterpret_cast<const float4*>(r1 + r1_at(rn, kGM + i));
#pragma unroll
                        for (int qb = 1; qb < 4; ++qb) {
                            const float4 w = *reinterpret_cast<const float4*>(r1 + r1_at(rn + qb, kGM + i));
                            v.x += w.x;
                            v.y += w.y;
                            v.z += w.z;
                            v.w += w.w;
                        }
                        acc.x = fmaf(uv.x, v.x, acc.x);
                        acc.y = fmaf(uv.x, v.y, acc.y);
                        acc.x = fmaf(uv.y, v.z, acc.x);
                        acc.y = fmaf(uv.y, v.w, acc.y);
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
    // the tensor copy of the window whose wait expired may still be in flight: it must land before the block exits
    if (tid == 0 && b < A.count) bounded_mbar_wait(mb, parity ^ 1u, kGWaitLimit);
}

}  // namespace dhk

namespace dh {

static int g_g_sms[64] = {0};
static int g_g_bps[64][2] = {};
static PFN_cuTensorMapEncodeTiled_v12000 g_g_encode = nullptr;

bool use_fused_g(const dhk::Plan& P) {
    return P.n == dhk::kGN && P.m == dhk::kGM && P.ny == P.n && P.my == P.m && P.groups <= dhk::kGG &&
           P.precision == DH_PRECISION_FP32;
}

cudaError_t fused_g_init() {
    cudaError_t e;
    if (!g_g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        g_g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if ((e = cudaFuncSetAttribute(dhk::k_fused128g<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)dhk::GSmem<uint16_t>::bytes)))
        return e;
    return cudaFuncSetAttribute(dhk::k_fused128g<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dhk::GSmem<float>::bytes);
}

int launch_fused_g(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                   cudaStream_t st, dhk::StageTimer* tm) {
    const int dev = H->device;
    if (dev < 0 || dev >= 64) return fail(DH_ERROR_ERROR, "device index out of range");
    if (batch < 1) return DH_SUCCESS;
    if (!g_g_encode) return fail(DH_ERROR_ERROR, "tensor-map encoder unavailable");
    const bool u16 = dtype == DH_DTYPE_U16;
    const int esz = u16 ? 2 : 4, align = 16 / esz;
    if (!g_g_sms[dev]) {
        int n = 0;
        cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device attribute");
        g_g_sms[dev] = n;
    }
    if (!g_g_bps[dev][u16 ? 0 : 1]) {
        int n = 0;
        cudaError_t e = u16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dhk::k_fused128g<uint16_t>, dhk::kGNT,
                                                                           dhk::GSmem<uint16_t>::bytes)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dhk::k_fused128g<float>, dhk::kGNT,
                                                                           dhk::GSmem<float>::bytes);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        g_g_bps[dev][u16 ? 0 : 1] = n > 0 ? n : 1;
    }
    // frames as a 3-D tensor [batch][height][width]; one box = the window rows plus the alignment slack
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof tmap);
    const cuuint64_t gdim[3] = {(cuuint64_t)P.width, (cuuint64_t)P.height, (cuuint64_t)batch};
    const cuuint64_t gstride[2] = {(cuuint64_t)P.width * esz, (cuuint64_t)P.width * P.height * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(dhk::kGN + align), (cuuint32_t)dhk::kGN, 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    CUresult cr = g_g_encode(&tmap, u16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                             const_cast<void*>(frames), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(DH_ERROR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    dhk::GArgs A;
    std::memset(&A, 0, sizeof A);
    A.count = batch;
    for (int p = 0; p < P.pols; ++p) {
        const int ox = P.pol[p].ox;               // window origins are >= 0
        A.x0[p] = (ox / align) * align;           // 16-byte aligned staging origin
        A.xo[p] = ox - A.x0[p];
    }
    A.fields = (float2*)fields;
    A.coefs = (float2*)coefs;
    // a persistent grid of every resident block; each block serves one polarisation
    const int resident = g_g_sms[dev] * g_g_bps[dev][u16 ? 0 : 1];
    const long long per_pol = std::min<long long>(batch, std::max(1, resident / P.pols));
    const int grid = (int)per_pol * P.pols;
    if (tm) tm->start(st);
    if (u16)
        dhk::k_fused128g<uint16_t><<<grid, dhk::kGNT, dhk::GSmem<uint16_t>::bytes, st>>>(P, A, tmap);
    else
        dhk::k_fused128g<float><<<grid, dhk::kGNT, dhk::GSmem<float>::bytes, st>>>(P, A, tmap);
    if (tm) tm->stop(st, "k_fused128g");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DH_SUCCESS;
}

}  // namespace dh
