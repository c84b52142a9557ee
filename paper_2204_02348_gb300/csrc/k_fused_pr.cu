// Column-pruned fused path for 128 x 128 windows with 64 x 64 fields (the guide's pipeline steps 1-3 and
// digHoloProcessRemoveTilt for one (frame, polarisation) window per thread block, persistent over windows).
//
// The window's spectrum is needed only inside the circular Fourier window.  Transforming along x first lets the
// kernel drop every column k_x that the window does not touch before the y transform: only the kept columns
// K = [kxlo, kxlo + nk) (at most 42 of 128 at the guide's radius rule) are transformed along y, selected,
// phase-corrected and inverse transformed along y; the x inverse then runs on the M field rows.
//
//   P1  x transform of the 64 row pairs (rows y and y + 64 packed as one complex row), 8 threads per row pair:
//       radix-8 over n1 (x = n2 + 16 n1, two n2 per thread) from the staged window, twiddles, an exchange
//       through shared memory, radix-16 over n2; writes Z_k[y] for the kept columns k and their mirrors N - k
//       (the conjugate partners that separate the two real rows) into slots of the work buffer F1.
//   P2  per kept column, 8 threads: separation of the two real row spectra, radix-16 / radix-8 y transform,
//       selection of the kept box rows with the beam-centre phase, the 64-point y inverse (radix 8 x 8), the
//       y residual-tilt and defocus removal; writes the column's y-inverse-transformed values (times the x
//       phase) for the field, and its y contraction H_n = sum_j u_n(y'_j) dy' G_j for the coefficients.
//   P3  per field row, 8 threads: 64-point x inverse over the kept columns, x correction, field write.
//   P4  coefficients c_mn = sum_c V_m[c] H_n[c], V the x inverse, x correction and x contraction of column c
//       in one FP64-built complex weight (the two sums regrouped, no other change).
//
// Every exchange inside one transform stays within the 8 threads that own it (one quarter of a warp), so it
// needs a warp barrier, not a block barrier; the block synchronises four times per window (window staged,
// pixels read, P1 written, P2 written).  Shared memory: the tensor-copy staging buffer of the next window
// (also P1's exchange space), F1 (96 slots of 66 complex values: kept columns, mirrors, and P2 / P3 exchange
// space), the table block and the y contractions: ~107 KB for uint16 frames, two blocks per SM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>

#include "fft.cuh"
#include "fused_pr.hpp"
#include "runtime.hpp"
#include "sync.cuh"

namespace dhk {

constexpr int kPrSlots = 2 * kPrMaxK;   // F1 slots: kept columns then their mirrors / exchange space
constexpr int kPrPitch = 66;            // complex values per slot (64 used; 528 bytes, 16-byte aligned)
constexpr int kPrNT = 512;
constexpr int kPrMaxModes = kPrG * (kPrG + 1) / 2;
constexpr long kPrWaitLimit = 1L << 24;

template <typename T>
struct PrStage {
    static constexpr int ALIGN = 16 / (int)sizeof(T);            // elements per 16 bytes
    // staged row: the window plus 32 bytes of slack (the 16-byte alignment of the copy, and a row pitch of
    // 8 banks modulo 32, so that the four row pairs of a warp read pixel pairs from distinct banks)
    static constexpr int W = kPrN + 2 * ALIGN;
    static constexpr int BYTES = kPrN * W * (int)sizeof(T);
    static_assert(BYTES >= 64 * 512, "P1's exchange (512 bytes per row pair) fits in the staging buffer");
    static_assert(BYTES % 128 == 0, "F1 starts on a 128-byte boundary");
};

// F1 slot of x frequency k: kept column k - kxlo, the mirror of kept column c at nk + c, else -1.
__device__ __forceinline__ int pr_slot(int k, int kxlo, int nk) {
    const int c = k - kxlo, mc = ((kPrN - k) & (kPrN - 1)) - kxlo;
    return (unsigned)c < (unsigned)nk ? c : (unsigned)mc < (unsigned)nk ? nk + mc : -1;
}

template <typename T>
struct PrSmem {
    static constexpr size_t F1 = (size_t)PrStage<T>::BYTES;                   // staging first (128-byte aligned)
    static constexpr size_t TB = F1 + (size_t)kPrSlots * kPrPitch * 8;
    static constexpr size_t H = TB + (size_t)PrLayout::BYTES;                 // float2 [kPrG][kPrMaxK]
    static constexpr size_t MD = H + (size_t)kPrG * kPrMaxK * 8;              // int mode_m, mode_n
    static constexpr size_t bytes = MD + 2 * (size_t)kPrMaxModes * 4;
};

// One thread: expect the window's bytes on the mbarrier and start the tensor copy of frame f (rows oy..oy+127,
// columns x0..x0+W-1 of the [frames][height][width] tensor).
__device__ __forceinline__ void pr_stage(const CUtensorMap* tmap, uint32_t dst, uint32_t mbar, int x0, int y0, int f,
                                         int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0), "r"(f), "r"(mbar)
        : "memory");
}

// Pixels x and x + 1 of a staged row (x even) as floats.
template <typename T, bool ODD>
__device__ __forceinline__ void pr_pixels(const T* row, int x, float& a, float& b) {
    if constexpr (sizeof(T) == 2) {
        if constexpr (ODD) {
            a = (float)row[x];
            b = (float)row[x + 1];
        } else {
            const uint32_t v = *reinterpret_cast<const uint32_t*>(row + x);
            a = (float)(v & 0xffffu);
            b = (float)(v >> 16);
        }
    } else {
        if constexpr (ODD) {
            a = row[x];
            b = row[x + 1];
        } else {
            const float2 v = *reinterpret_cast<const float2*>(row + x);
            a = v.x;
            b = v.y;
        }
    }
}

// a[k] *= w^k for k = 1 .. R-1, the powers by binary powering (w^k = w^(k/2) w^((k+1)/2), at most four
// products deep for R = 16): here shared-memory table reads would cost more than these multiplications.
template <int R>
__device__ __forceinline__ void pr_twiddle(float2* a, float2 w) {
    float2 p[R];
    p[1] = w;
#pragma unroll
    for (int k = 2; k < R; ++k) p[k] = cmul(p[k >> 1], p[(k + 1) >> 1]);
#pragma unroll
    for (int k = 1; k < R; ++k) a[k] = cmul(a[k], p[k]);
}

__device__ __forceinline__ float2 f4lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f4hi(float4 v) { return make_float2(v.z, v.w); }

// Position (in complex values) of element [row][col] of an 8 x 8 exchange tile whose reader of row r takes the
// row as four 16-byte chunks: chunks are XOR-swizzled by r / 2 so that the eight readers hit distinct banks.
__device__ __forceinline__ int x8(int row, int col) { return row * 8 + ((((col >> 1) ^ (row >> 1)) & 3) << 1) + (col & 1); }
__device__ __forceinline__ int x8chunk(int row, int k) { return row * 4 + ((k ^ (row >> 1)) & 3); }

struct PrArgs {
    int frame0, count;
    int xo[DH_MAX_POLS];          // window origin minus the 16-byte-aligned staging origin, per polarisation
    int x0[DH_MAX_POLS];          // staging origin (element index), per polarisation
    float2* fields;               // nullable [B][pol][M][M]
    float2* coefs;                // nullable [B][pol][modes]
};

}  // namespace dhk

namespace dhk {

// P2 and P3 are separate functions (not inlined): the window loop's state is saved around the call once per
// window instead of competing for registers with the 16-point transforms.
__device__ __noinline__ void pr_columns(unsigned char* smem_base, size_t f1_off, int nk, int kxlo, int kly, int G,
                                        bool want_f, bool want_c) {
    using L = PrLayout;
    constexpr int N = kPrN, M = kPrM;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, t = tid & 7;
    float2* F1 = reinterpret_cast<float2*>(smem_base + f1_off);
    unsigned char* TB = smem_base + f1_off + (size_t)kPrSlots * kPrPitch * 8;
    float2* Hs = reinterpret_cast<float2*>(TB + L::BYTES);
    // ---------------------------------------------------------------- P2: the kept columns
    {
        // group gq of warp w takes column c; the two groups of a half-warp take columns four apart, so their
        // slots (528 bytes apart per column) start 64 bytes apart in the banks
        const int gq = lane >> 3;
        const int c = 8 * (w >> 1) + 2 * (w & 1) + (gq >> 1) + 4 * (gq & 1);
        const bool act = c < nk;
        if (__any_sync(0xffffffffu, act)) {
            const int cc = act ? c : 0;   // groups without a column compute on column 0 and store nothing
            const int kx = kxlo + cc;
            const int mk = (N - kx) & (N - 1);
            float2* s1 = F1 + cc * kPrPitch;          // the column (Z_k), then its window, then its field values
            float2* s2 = F1 + (nk + cc) * kPrPitch;   // its mirror Z_{N-k} (or spare), then exchange space
            const float2* sm = F1 + pr_slot(mk, kxlo, nk) * kPrPitch;
            // separation: the spectra of rows y (y < 64) and y + 64 at k from Z_k and conj Z_{N-k}
            float2 a16[16];   // y = t + 8 r
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float2 a = s1[t + 8 * r], bm = sm[t + 8 * r];
                a16[r] = make_float2(a.x + bm.x, a.y - bm.y);
                a16[r + 8] = make_float2(a.y + bm.y, bm.x - a.x);
            }
            dft16<false>(a16);   // over r: frequency k1 = ky mod 16
            pr_twiddle<16>(a16, reinterpret_cast<const float2*>(TB + L::TWN)[t]);   // W_N^(t k1)
            __syncwarp();   // the group's slot reads are done
            // exchange: rows k1 in 128-byte blocks of two, block bb read by thread bb (blocks 0..3 in s1, 4..7 in
            // s2); a 16-byte chunk's bank position is XOR-swizzled by the block index, net of the block's own
            // position (slot s starts s * 528 bytes in, i.e. s chunks past a 128-byte boundary)
            const int o1 = cc & 7, o2 = (nk + cc) & 7;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const int bb = k1 >> 1;
                float2* base = (bb < 4 ? s1 : s2) + (bb & 3) * 16;
                const int ch = (((((k1 & 1) << 2) | (t >> 1)) ^ bb) - (bb < 4 ? o1 : o2)) & 7;
                if (act) base[ch * 2 + (t & 1)] = a16[k1];
            }
            __syncwarp();
            float2 b0[8], b1[8];   // k1 = 2t and 2t + 1, over the eight column threads
            {
                const float4* base = reinterpret_cast<const float4*>((t < 4 ? s1 : s2) + (t & 3) * 16);
                const int ob = t < 4 ? o1 : o2;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 v = base[((k ^ t) - ob) & 7];
                    if (k < 4) {
                        b0[2 * k] = f4lo(v);
                        b0[2 * k + 1] = f4hi(v);
                    } else {
                        b1[2 * k - 8] = f4lo(v);
                        b1[2 * k - 7] = f4hi(v);
                    }
                }
            }
            dft8<false>(b0);   // ky = 2t + 16 k2
            dft8<false>(b1);   // ky = 2t + 1 + 16 k2
            __syncwarp();      // the exchange blocks are read
            // the box rows q < M of this column in box-row order in s1 (rotated by one place for every other
            // column pair, so that the two columns of a half-warp write different banks)
            const int rot = (cc >> 2) & 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int k2 = 0; k2 < 8; ++k2) {
                    const int q = (2 * t + h + 16 * k2 - kly) & (N - 1);
                    if (act && q < M) s1[(q + rot) & (M - 1)] = h ? b1[k2] : b0[k2];
                }
            }
            __syncwarp();
            // 64-point y inverse: radix 8 over r (q = t + 8 r) of the window (kept rows [qlo, qhi] times the y
            // beam-centre phase, zero elsewhere), twiddles, exchange, radix 8 over t
            float2 v8[8];
            {
                const int2 ql = reinterpret_cast<const int2*>(TB + L::QLIM)[cc];
                const float2* phy = reinterpret_cast<const float2*>(TB + L::PHY);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int q = t + 8 * r;
                    const float2 v = s1[(q + rot) & (M - 1)];
                    v8[r] = (q >= ql.x && q <= ql.y) ? cmul(v, phy[q]) : make_float2(0.f, 0.f);
                }
            }
            dft8<true>(v8);
            {
                const float2 b = reinterpret_cast<const float2*>(TB + L::TWN)[2 * t];
                pr_twiddle<8>(v8, make_float2(b.x, -b.y));   // exp(+2 pi i t j1 / M)
            }
#pragma unroll
            for (int j1 = 0; j1 < 8; ++j1)
                if (act) s2[x8(j1, t)] = v8[j1];
            __syncwarp();
            float2 cv[8];   // j = t + 8 j2
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = reinterpret_cast<const float4*>(s2)[x8chunk(t, k)];
                cv[2 * k] = f4lo(v);
                cv[2 * k + 1] = f4hi(v);
            }
            dft8<true>(cv);
            {
                const float2* cy = reinterpret_cast<const float2*>(TB + L::CY);
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2) cv[j2] = cmul(cv[j2], cy[t + 8 * j2]);
            }
            if (want_f) {
                // the column's values for the field rows, times its x phase (s1's window was read above)
                const float2 px = reinterpret_cast<const float2*>(TB + L::PHX)[cc];
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2)
                    if (act) s1[t + 8 * j2] = cmul(cv[j2], px);
            }
            if (want_c) {
                // y contraction H_n[c] = sum_j u_n(y'_j) dy' G_j, four modes at a time: per-thread partial sums
                // over its eight rows, then a fixed-order sum over the eight threads through s2
                const float4* hg4 = reinterpret_cast<const float4*>(TB + L::HGY);   // [j][5] float4
                __syncwarp();   // the exchange tile in s2 is read
                for (int n4 = 0; n4 < G; n4 += 4) {
                    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
                    for (int j2 = 0; j2 < 8; ++j2) {
                        const float4 u = hg4[(t + 8 * j2) * 5 + (n4 >> 2)];
                        const float2 e = cv[j2];
                        a0.x = fmaf(u.x, e.x, a0.x);
                        a0.y = fmaf(u.x, e.y, a0.y);
                        a1.x = fmaf(u.y, e.x, a1.x);
                        a1.y = fmaf(u.y, e.y, a1.y);
                        a2.x = fmaf(u.z, e.x, a2.x);
                        a2.y = fmaf(u.z, e.y, a2.y);
                        a3.x = fmaf(u.w, e.x, a3.x);
                        a3.y = fmaf(u.w, e.y, a3.y);
                    }
                    if (act) {
                        s2[t] = a0;
                        s2[8 + t] = a1;
                        s2[16 + t] = a2;
                        s2[24 + t] = a3;
                    }
                    __syncwarp();
                    if (act && t < 4 && n4 + t < G) {
                        const float4* rp = reinterpret_cast<const float4*>(s2 + 8 * t);
                        float2 sum = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float4 v = rp[k];
                            sum.x += v.x;
                            sum.y += v.y;
                            sum.x += v.z;
                            sum.y += v.w;
                        }
                        Hs[(n4 + t) * kPrMaxK + cc] = sum;
                    }
                    __syncwarp();
                }
            }
        }
    }
}

__device__ __noinline__ void pr_rows(unsigned char* smem_base, size_t f1_off, int nk, int kxlo, int klx, float2* fields) {
    using L = PrLayout;
    constexpr int M = kPrM;
    const int tid = threadIdx.x, t = tid & 7;
    const float2* F1c = reinterpret_cast<const float2*>(smem_base + f1_off);
    float2* F1 = const_cast<float2*>(F1c);
    const unsigned char* TB = smem_base + f1_off + (size_t)kPrSlots * kPrPitch * 8;
    // ---------------------------------------------------------------- P3: field rows
    {
        const int jr = tid >> 3;   // field row j
        float2 v8[8];              // box column p = t + 8 r; zero outside the kept columns
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int c = klx + t + 8 * r - kxlo;
            v8[r] = (c >= 0 && c < nk) ? F1[c * kPrPitch + jr] : make_float2(0.f, 0.f);
        }
        dft8<true>(v8);
        {
            const float2 b = reinterpret_cast<const float2*>(TB + L::TWN)[2 * t];
            pr_twiddle<8>(v8, make_float2(b.x, -b.y));   // exp(+2 pi i t j1 / M)
        }
        // exchange in two rounds of a 4 x 8 tile per row, behind the kept columns' slots
        float2* X = F1 + nk * kPrPitch + jr * 32;
        const int rx = jr & 1;
        float2 cv[8];
#pragma unroll
        for (int j1 = 0; j1 < 4; ++j1) X[x8(j1 ^ rx, t)] = v8[j1];
        __syncwarp();
        if (t < 4) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = reinterpret_cast<const float4*>(X)[x8chunk(t ^ rx, k)];
                cv[2 * k] = f4lo(v);
                cv[2 * k + 1] = f4hi(v);
            }
        }
        __syncwarp();
#pragma unroll
        for (int j1 = 0; j1 < 4; ++j1) X[x8(j1 ^ rx, t)] = v8[j1 + 4];
        __syncwarp();
        if (t >= 4) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = reinterpret_cast<const float4*>(X)[x8chunk((t - 4) ^ rx, k)];
                cv[2 * k] = f4lo(v);
                cv[2 * k + 1] = f4hi(v);
            }
        }
        dft8<true>(cv);   // i = t + 8 i2
        const float2* cx = reinterpret_cast<const float2*>(TB + L::CX);
        float2* out = fields + (size_t)jr * M;
#pragma unroll
        for (int i2 = 0; i2 < 8; ++i2) out[t + 8 * i2] = cmul(cv[i2], cx[t + 8 * i2]);
    }

}

// ODD: the window starts on an odd element of the staged row (pixel pairs are then read one by one).
template <typename T, bool ODD>
__global__ void __launch_bounds__(kPrNT, sizeof(T) == 2 ? 2 : 1)
    k_fused128p(const __grid_constant__ Plan P, const __grid_constant__ PrArgs A, const __grid_constant__ CUtensorMap tmap) {
    using SM = PrSmem<T>;
    using S = PrStage<T>;
    using L = PrLayout;
    constexpr int N = kPrN, M = kPrM;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int abort_flag;
    T* stg = reinterpret_cast<T*>(smem);
    float2* F1 = reinterpret_cast<float2*>(smem + SM::F1);
    unsigned char* TB = smem + SM::TB;
    float2* Hs = reinterpret_cast<float2*>(smem + SM::H);
    int* mdm = reinterpret_cast<int*>(smem + SM::MD);
    int* mdn = mdm + kPrMaxModes;
    const int tid = threadIdx.x, t = tid & 7;
    // every block serves one polarisation: its table block is staged once
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    {
        const int4* src = reinterpret_cast<const int4*>(pd.pr);
        int4* dst4 = reinterpret_cast<int4*>(TB);
        for (int i = tid; i < L::BYTES / 16; i += kPrNT) dst4[i] = __ldg(src + i);
        for (int i = tid; i < P.modes; i += kPrNT) {
            mdm[i] = P.mode_m[i];
            mdn[i] = P.mode_n[i];
        }
    }
    const int* hdr = reinterpret_cast<const int*>(pd.pr);
    const int nk = __ldg(hdr), kxlo = __ldg(hdr + 1), klx = __ldg(hdr + 2), kly = __ldg(hdr + 3);
    const int G = P.groups, modes = P.modes;
    const bool want_f = A.fields != nullptr, want_c = A.coefs != nullptr && G > 0;
    const uint32_t mb = smem_u32(&mbar), dst = smem_u32(stg);
    const int fstride = gridDim.x / P.pols;
    int b = blockIdx.x / P.pols;
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (b < A.count) pr_stage(&tmap, dst, mb, A.x0[pol], pd.oy, A.frame0 + b, S::BYTES);
    }
    __syncthreads();
    const int xo = A.xo[pol];
    uint32_t parity = 0;
    for (; b < A.count; b += fstride) {
        const int f = A.frame0 + b;
        const bool ok = bounded_mbar_wait(mb, parity, kPrWaitLimit);
        parity ^= 1u;
        if (!ok) abort_flag = 1;
        __syncthreads();   // window staged; the previous window's P3 / P4 are done with F1 and H
        if (abort_flag) {
            if (tid == 0 && P.status) atomicOr(P.status, 1);
            break;
        }

        // ---------------------------------------------------------------- P1: x transform of the row pairs
        const int g = tid >> 3;   // rows g and g + 64, packed as the real and imaginary parts of one row
        float2 za[8], zb[8];      // x = 2t + 16 n1 (za) and x = 2t + 1 + 16 n1 (zb), n1 = 0..7
        {
            const T* r0 = stg + g * S::W + xo;
            const T* r1 = r0 + 64 * S::W;
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const int x = 2 * t + 16 * n1;
                float a0, a1, b0, b1;
                pr_pixels<T, ODD>(r0, x, a0, a1);
                pr_pixels<T, ODD>(r1, x, b0, b1);
                za[n1] = make_float2(a0, b0);
                zb[n1] = make_float2(a1, b1);
            }
            if (pd.cal) {
                // reference calibration: pixel (x, y) times sqrt(max cal / cal), from the L2-resident table
                const float* c0 = pd.cal + g * N;
                const float* c1 = c0 + 64 * N;
#pragma unroll
                for (int n1 = 0; n1 < 8; ++n1) {
                    const int x = 2 * t + 16 * n1;
                    const float2 u = __ldg(reinterpret_cast<const float2*>(c0 + x));
                    const float2 v = __ldg(reinterpret_cast<const float2*>(c1 + x));
                    za[n1].x *= u.x;
                    zb[n1].x *= u.y;
                    za[n1].y *= v.x;
                    zb[n1].y *= v.y;
                }
            }
        }
        // every pixel is in registers: the staging buffer becomes P1's exchange space
        __syncthreads();
        dft8<false>(za);
        dft8<false>(zb);
        {
            // W_N^(n2 k1) for n2 = 2t, 2t + 1 from the base table (index n2 k1 < N)
            const float2* twn = reinterpret_cast<const float2*>(TB + L::TWN);
#pragma unroll
            for (int k1 = 1; k1 < 8; ++k1) {
                za[k1] = cmul(za[k1], twn[2 * t * k1]);
                zb[k1] = cmul(zb[k1], twn[(2 * t + 1) * k1]);
            }
        }
        float2 y[16];   // after the exchange: n2 = 0..15 at the frequency k1 = t
        {
            // 8 x 8 tile per row pair and round (row k1, column = writing thread); odd row pairs swap row
            // parity so that the two row pairs of a half-warp write different banks
            float2* X = reinterpret_cast<float2*>(stg) + g * 64;
            const int rx = g & 1;
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) X[x8(k1 ^ rx, t)] = za[k1];   // n2 = 2t
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = reinterpret_cast<const float4*>(X)[x8chunk(t ^ rx, k)];
                y[4 * k] = f4lo(v);
                y[4 * k + 2] = f4hi(v);
            }
            __syncwarp();
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) X[x8(k1 ^ rx, t)] = zb[k1];   // n2 = 2t + 1
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = reinterpret_cast<const float4*>(X)[x8chunk(t ^ rx, k)];
                y[4 * k + 1] = f4lo(v);
                y[4 * k + 3] = f4hi(v);
            }
        }
        dft16<false>(y);   // y[k2] = Z(t + 8 k2)
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int sl = pr_slot(t + 8 * k2, kxlo, nk);
            if (sl >= 0) F1[sl * kPrPitch + g] = y[k2];
        }
        // the staging buffer's generic reads and writes are ordered before the next tensor copy into it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0 && b + fstride < A.count) pr_stage(&tmap, dst, mb, A.x0[pol], pd.oy, f + fstride, S::BYTES);

        // ---------------------------------------------------------------- P2: the kept columns
        pr_columns(smem, SM::F1, nk, kxlo, kly, G, want_f, want_c);
        __syncthreads();

        // ---------------------------------------------------------------- P3: field rows
        if (want_f) pr_rows(smem, SM::F1, nk, kxlo, klx, A.fields + ((size_t)f * P.pols + pol) * M * M);

        // ---------------------------------------------------------------- P4: coefficients
        if (want_c) {
            // c_mn = sum_c V_m[c] H_n[c]: eight threads per mode over the kept columns, fixed shuffle tree
            const float2* V = reinterpret_cast<const float2*>(TB + L::V);
            float2* cf = A.coefs + ((size_t)f * P.pols + pol) * modes;
            for (int k0 = 0; k0 < modes; k0 += kPrNT / 8) {
                const int k = k0 + (tid >> 3);
                float2 acc = make_float2(0.f, 0.f);
                if (k < modes) {
                    const float2* vm = V + mdm[k] * kPrMaxK;
                    const float2* hn = Hs + mdn[k] * kPrMaxK;
                    for (int c = t; c < nk; c += 8) {
                        const float2 a = vm[c], h = hn[c];
                        acc.x = fmaf(a.x, h.x, acc.x);
                        acc.x = fmaf(-a.y, h.y, acc.x);
                        acc.y = fmaf(a.x, h.y, acc.y);
                        acc.y = fmaf(a.y, h.x, acc.y);
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
                if (t == 0 && k < modes && DH_IN(P.status, k, modes, kSiteFusedCoef)) cf[k] = acc;
            }
        }
    }
    // a tensor copy still in flight (only after an expired wait) must land before the block exits
    if (abort_flag && tid == 0) bounded_mbar_wait(mb, parity, kPrWaitLimit);
}

}  // namespace dhk

namespace dh {

static PFN_cuTensorMapEncodeTiled_v12000 g_pr_encode = nullptr;
static int g_pr_sms[64] = {0};
static int g_pr_bps[64][2] = {};   // resident blocks per SM, per pixel type

bool use_fused_pr(const dhk::Plan& P) {
    if (P.n != dhk::kPrN || P.m != dhk::kPrM || P.ny != P.n || P.my != P.m || P.groups > dhk::kPrG ||
        P.precision != DH_PRECISION_FP32)
        return false;
    for (int p = 0; p < P.pols; ++p)
        if (!P.pol[p].pr) return false;
    return true;
}

template <typename T>
static cudaError_t pr_attr() {
    cudaError_t e = cudaFuncSetAttribute(dhk::k_fused128p<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dhk::PrSmem<T>::bytes);
    if (e) return e;
    return cudaFuncSetAttribute(dhk::k_fused128p<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dhk::PrSmem<T>::bytes);
}

cudaError_t fused_pr_init() {
    cudaError_t e;
    if (!g_pr_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        g_pr_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if ((e = pr_attr<uint16_t>())) return e;
    return pr_attr<float>();
}

int launch_fused_pr(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                    cudaStream_t st, dhk::StageTimer* tm) {
    const int dev = H->device;
    if (dev < 0 || dev >= 64) return fail(DH_ERROR_ERROR, "device index out of range");
    if (batch < 1) return DH_SUCCESS;
    if (!g_pr_encode) return fail(DH_ERROR_ERROR, "tensor-map encoder unavailable");
    const bool u16 = dtype == DH_DTYPE_U16;
    const int esz = u16 ? 2 : 4, align = 16 / esz;
    if (!g_pr_sms[dev]) {
        int n = 0;
        cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device attribute");
        g_pr_sms[dev] = n;
    }
    if (!g_pr_bps[dev][u16 ? 0 : 1]) {
        int n = 0;
        cudaError_t e = u16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dhk::k_fused128p<uint16_t, false>, dhk::kPrNT,
                                                                           dhk::PrSmem<uint16_t>::bytes)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dhk::k_fused128p<float, false>, dhk::kPrNT,
                                                                           dhk::PrSmem<float>::bytes);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        g_pr_bps[dev][u16 ? 0 : 1] = n > 0 ? n : 1;
    }
    // frames as a 3-D tensor [batch][height][width]; one box = the window rows plus alignment slack
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof tmap);
    const cuuint64_t gdim[3] = {(cuuint64_t)P.width, (cuuint64_t)P.height, (cuuint64_t)batch};
    const cuuint64_t gstride[2] = {(cuuint64_t)P.width * esz, (cuuint64_t)P.width * P.height * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(dhk::kPrN + 2 * align), (cuuint32_t)dhk::kPrN, 1};   // PrStage<T>::W
    const cuuint32_t estride[3] = {1, 1, 1};
    CUresult cr = g_pr_encode(&tmap, u16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              const_cast<void*>(frames), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(DH_ERROR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    dhk::PrArgs A;
    std::memset(&A, 0, sizeof A);
    A.frame0 = 0;
    A.count = batch;
    bool odd = false;
    for (int p = 0; p < P.pols; ++p) {
        const int ox = P.pol[p].ox;               // window origins are >= 0
        A.x0[p] = (ox / align) * align;           // 16-byte aligned staging origin
        A.xo[p] = ox - A.x0[p];
        odd = odd || (A.xo[p] & 1);
    }
    A.fields = (float2*)fields;
    A.coefs = (float2*)coefs;
    // a persistent grid of every resident block; each block serves one polarisation
    const int resident = g_pr_sms[dev] * g_pr_bps[dev][u16 ? 0 : 1];
    const long long per_pol = std::min<long long>(batch, std::max(1, resident / P.pols));
    const int grid = (int)per_pol * P.pols;
    if (tm) tm->start(st);
    if (u16) {
        if (odd)
            dhk::k_fused128p<uint16_t, true><<<grid, dhk::kPrNT, dhk::PrSmem<uint16_t>::bytes, st>>>(P, A, tmap);
        else
            dhk::k_fused128p<uint16_t, false><<<grid, dhk::kPrNT, dhk::PrSmem<uint16_t>::bytes, st>>>(P, A, tmap);
    } else {
        if (odd)
            dhk::k_fused128p<float, true><<<grid, dhk::kPrNT, dhk::PrSmem<float>::bytes, st>>>(P, A, tmap);
        else
            dhk::k_fused128p<float, false><<<grid, dhk::kPrNT, dhk::PrSmem<float>::bytes, st>>>(P, A, tmap);
    }
    if (tm) tm->stop(st, "k_fused128p");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DH_SUCCESS;
}

}  // namespace dh
