// Coefficient-only split-BF16 decomposition on the tensor cores (pipeline step 2 along y, tilt and defocus
// removal, and the HG modal decomposition of step 3, when no field is requested: candidate scoring,
// coefficient-only processing and serving).
//
// With g[q][i] the x-inverse-transformed window rows (box row q, field column i) that the generic path's x
// pass leaves in scratch, the y inverse transform, the y correction and the y overlap weights are one complex
// linear map Y_n[q] (host-built in FP64, plan.cpp), so
//     T_n[i] = sum_q Y_n[q] g[q][i],     c_mn = sum_i X_m[i] T_n[i],     X_m[i] = u_m(x'_i) dx' corr_x[i],
// the same sums as transform-then-overlap, regrouped, with no y transform left to run.  The first contraction
// is a real GEMM on tcgen05: rows = field columns i (tiles of 128), K = 2M (the real parts of the window rows,
// then their imaginary parts), N = 2G rounded up to 16 (real parts of T_n, then imaginary parts), B = the y map
// as bfloat16 hi + lo, A = g split into bfloat16 hi + lo.  Three products per K step (hi hi + hi lo + lo hi),
// FP32 accumulation in tensor memory.  Candidate scoring runs the same kernel on the raw box bins of the
// superset spectra, with the x inverse transform and the beam-centre phases folded into its tables.
//
// Data movement.  K advances in chunks of 16 window rows.  A chunk (its 16 rows of A as FP32 and its slice of
// B, 128 np bytes) is brought into one slot of a ring in shared memory by asynchronous copies (cp.async, every
// thread a share of them) issued slots - 1 chunks ahead, across window boundaries, so the next window's rows
// are in flight while a window's coefficients are formed.  Each chunk is then split into bfloat16 hi / lo in
// the canonical K-major layout of the A stage and multiplied by one elected thread; the next chunk waits for
// those products before it overwrites the stage and refills the slot.  After a window's last chunk four warps
// read the accumulator back with tcgen05.ld and the second contraction (a complex dot product of length M per
// mode) runs on CUDA cores, eight lanes per 2 x 2 block of modes, summed in a fixed order.
//
// Every wait on an mbarrier is bounded; on expiry the window's coefficients are NaN, bit 1 of the plan's status
// word is set, and the block stops issuing products and releases its tensor memory after the ones in flight.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.cuh"
#include "runtime.hpp"
#include "sync.cuh"
#include "umma.cuh"

namespace dhk {

namespace {

constexpr int kCtThreads = 512;
constexpr int kCtQ = 16;                 // window rows per K chunk (K = 32 per chunk: real, then imaginary)
constexpr int kCtK = 2 * kCtQ;
constexpr int kCtSplit = 8;              // lanes per 2 x 2 block of modes in the second contraction
constexpr long kCtWait = 1L << 24;
constexpr int kCtSmemLimit = 227 * 1024 - 1024;

struct CtLayout {
    int stage_bytes;                     // one plane of one tile of the A stage (128 rows x 32 K, bf16)
    int slot_a, slot_b, slot_bytes;      // one ring slot: 16 rows of A as float2 [16][M], then B [2][NP][32] bf16
    size_t a;                            // A stage [2][tiles][128][32] bf16; after the products T [2G][M + 4] FP32
    size_t s;                            // ring [slots]
    size_t x;                            // float2 X [G][M + 4]
    size_t mk;                           // int2 kept column range of each box row [M] (box source)
    size_t bytes;
};

__host__ __device__ inline CtLayout ct_layout(int M, int NP, int G, int tiles, int slots) {
    CtLayout L;
    L.stage_bytes = 128 * kCtK * 2;
    L.slot_a = kCtQ * M * 8;
    L.slot_b = 2 * NP * kCtK * 2;
    L.slot_bytes = (L.slot_a + L.slot_b + 127) & ~127;
    size_t abytes = (size_t)2 * tiles * L.stage_bytes;
    const size_t tbytes = (size_t)2 * G * (M + 4) * 4;
    if (tbytes > abytes) abytes = tbytes;
    L.a = 0;
    L.s = (L.a + abytes + 1023) & ~(size_t)1023;
    L.x = L.s + (size_t)slots * L.slot_bytes;
    L.mk = L.x + (size_t)G * (M + 4) * 8;
    L.bytes = (L.mk + (size_t)M * 8 + 1023) & ~(size_t)1023;
    return L;
}

// Tensor-memory column stride of one tile's accumulator (NP rounded up to 32) and the columns of `tiles` of
// them (a power of two >= 32).
__host__ __device__ inline int ct_tstride(int NP) { return (NP + 31) & ~31; }
__host__ __device__ inline uint32_t ct_tmem_cols(int tiles, int NP) {
    uint32_t c = 32;
    while (c < (uint32_t)(tiles * ct_tstride(NP))) c <<= 1;
    return c;
}

}  // namespace

// Asynchronous global -> shared copies (generic proxy); `bytes` < size fills the rest of the destination with
// zeros (bytes 0: nothing is read).
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most n of this thread's most recent copy groups are pending (n = 0, 1 or 2).
__device__ __forceinline__ void cp_async_wait(int n) {
    if (n <= 0)
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (n == 1)
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

// One item of a chunk: field (or box) column i = item mod M and eight consecutive rows of the chunk (half
// item / M), read from the slot's FP32 rows and stored as bfloat16 hi and lo in the A stage (row i of tile
// i / 128; K: the eight rows' real parts at 8 (half), their imaginary parts 16 further).  Consecutive threads
// take consecutive columns: the slot reads and the 16-byte stores are free of bank conflicts.
template <int TILES>
__device__ __forceinline__ void ct_convert(const float2* slot, unsigned char* sa, int stage_bytes, int M, int item) {
    const int qh = item >= M, i = item - qh * M;
    __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 v = slot[(8 * qh + r) * M + i];
        rh[r] = __float2bfloat16_rn(v.x);
        ih[r] = __float2bfloat16_rn(v.y);
        rl[r] = __float2bfloat16_rn(v.x - __bfloat162float(rh[r]));
        il[r] = __float2bfloat16_rn(v.y - __bfloat162float(ih[r]));
    }
    const int t = i >> 7, row = i & 127;
    __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(sa + (size_t)t * stage_bytes);
    __nv_bfloat16* lo = reinterpret_cast<__nv_bfloat16*>(sa + (size_t)(TILES + t) * stage_bytes);
    *reinterpret_cast<uint4*>(hi + umma_off(row, 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(rh);
    *reinterpret_cast<uint4*>(hi + umma_off(row, kCtQ + 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(ih);
    *reinterpret_cast<uint4*>(lo + umma_off(row, 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(rl);
    *reinterpret_cast<uint4*>(lo + umma_off(row, kCtQ + 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(il);
}

// SCORE: the A rows are a candidate's raw box bins (BoxSrc; bins outside a row's kept range read as zero) and
// the tables its scoring tables; otherwise the x-inverse-transformed rows in B.g with the coefficient-only
// tables.  A persistent grid: every block serves one polarisation and a stride of that polarisation's windows,
// whose chunks pass through the ring as one stream.  slots: ring slots (2 to 4).
template <int TILES, bool SCORE>
__global__ void __launch_bounds__(kCtThreads, 1) k_coef_tc(const __grid_constant__ Plan P, const __grid_constant__ Batch B,
                                                           const __grid_constant__ BoxSrc S, int slots) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = P.m, G = P.groups, NP = P.coef_np, modes = P.modes, chunks = M / kCtQ;
    const int XP = M + 4;                 // pitch of X (float2) and T (float) rows: 2 rows apart = 8 banks apart
    const CtLayout L = ct_layout(M, NP, G, TILES, slots);
    const uint32_t tcols = ct_tmem_cols(TILES, NP);
    const int tstride = ct_tstride(NP);
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    const unsigned char* tab = SCORE ? pd.score_tc : pd.coef_tc;
    unsigned char* As = sm + L.a;
    float* Ts = reinterpret_cast<float*>(sm + L.a);   // T [2G][XP] once a window's products are complete
    float2* X = reinterpret_cast<float2*>(sm + L.x);
    int2* mk = reinterpret_cast<int2*>(sm + L.mk);
    {
        const float2* xs = reinterpret_cast<const float2*>(tab + (size_t)chunks * L.slot_b);
        for (int i = tid; i < G * M; i += kCtThreads) X[(i / M) * XP + i % M] = __ldg(xs + i);
        // the A stage starts zero, so rows past M of the last tile contribute nothing
        uint4* a4 = reinterpret_cast<uint4*>(As);
        for (int i = tid; i < (2 * TILES * L.stage_bytes) / 16; i += kCtThreads) a4[i] = make_uint4(0u, 0u, 0u, 0u);
        if (SCORE)
            for (int i = tid; i < M; i += kCtThreads) mk[i] = make_int2(pd.mask_lo[i], pd.mask_hi[i]);
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), tcols);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t a_base = smem_u32(As), s_base = smem_u32(sm + L.s);
    const uint32_t idesc = umma_idesc_bf16(128, NP);

    // this block's windows fb0, fb0 + fstride, ... and its stream of total chunks
    const int fb0 = blockIdx.x / P.pols, fstride = gridDim.x / P.pols;
    const long nwin = fb0 < B.count ? (long)(B.count - 1 - fb0) / fstride + 1 : 0;
    const long total = nwin * chunks;
    const size_t wstride = SCORE ? (size_t)S.ms * S.msx : (size_t)M * M;
    const int pitch = SCORE ? S.msx : M;
    const float2* src0 = SCORE ? S.xs + (size_t)S.qoff[pol] * S.msx + S.poff[pol] : B.g;
    // this thread's elements of every chunk (the same in each): row << 16 | column, or -1
    constexpr int EMAX = SCORE ? 4 * TILES : 2 * TILES;
    int rp[EMAX];
#pragma unroll
    for (int u = 0; u < EMAX; ++u) {
        const int e = tid + u * kCtThreads;
        if (SCORE)
            rp[u] = e < kCtQ * M ? ((e / M) << 16) | (e % M) : -1;
        else
            rp[u] = e < kCtQ * M / 2 ? e : -1;
    }
    // copies of the next chunk of the stream into the next slot, one commit group per call (empty past the
    // stream's end); the position advances by counters (no division)
    long ij = 0;                          // stream index of the next chunk to copy
    int ic = 0, ifb = fb0, islot = 0;     // its chunk within the window, its window, its slot
    auto issue = [&]() {
        if (ij < total) {
            const uint32_t slot = s_base + (uint32_t)(islot * L.slot_bytes);
            const float2* rows = src0 + (size_t)(ifb * P.pols + pol) * wstride + (size_t)(kCtQ * ic) * pitch;
#pragma unroll
            for (int u = 0; u < EMAX; ++u) {
                if (rp[u] < 0) continue;
                if constexpr (SCORE) {
                    const int r = rp[u] >> 16, p = rp[u] & 0xffff;
                    const int2 k = mk[kCtQ * ic + r];
                    const bool keep = p >= k.x && p <= k.y;
                    cp_async8(slot + 8u * (uint32_t)(r * M + p), rows + (size_t)r * pitch + (keep ? p : 0), keep ? 8u : 0u);
                } else {
                    // 16 contiguous rows of M complex values, 16 bytes a piece (M even)
                    cp_async16(slot + 16u * (uint32_t)rp[u], reinterpret_cast<const float4*>(rows) + rp[u]);
                }
            }
            const uint4* bsrc = reinterpret_cast<const uint4*>(tab + (size_t)ic * L.slot_b);
            for (int e = tid; e < L.slot_b / 16; e += kCtThreads) cp_async16(slot + (uint32_t)L.slot_a + 16u * e, bsrc + e);
            ++ij;
            if (++ic == chunks) {
                ic = 0;
                ifb += fstride;
            }
            if (++islot == slots) islot = 0;
        }
        cp_async_commit();
    };
    for (int k = 0; k < slots - 1; ++k) issue();

    uint32_t phase = 0u, lost = 0u;
    bool pending = false, ok = true;      // ok: every wait so far completed (the same in every thread)
    auto settle = [&]() {
        // the products committed last are complete (tid 0 waits; the barrier passes its finding on)
        bool done = true;
        if (pending) {
            done = ok && (tid != 0 || bounded_mbar_wait(smem_u32(&mbar), phase, kCtWait));
            if (!done) lost = phase;
            phase ^= 1u;
            pending = false;
        }
        return done;
    };
    int c = 0, fb = fb0, cslot = 0;       // the current chunk's position: chunk in window, window, slot
    for (long j = 0; j < total; ++j) {
        const bool done = settle();
        cp_async_wait(slots - 2);          // this thread's copies of chunk j have landed
        const bool all = __syncthreads_and(done ? 1 : 0) != 0;
        if (ok && !all && tid == 0 && P.status) atomicOr(P.status, 2);
        ok = ok && all;
        // the slot chunk j - 1 used is free: refill it; then split chunk j into the A stage
        issue();
        const float2* sl = reinterpret_cast<const float2*>(sm + L.s + (size_t)cslot * L.slot_bytes);
        for (int item = tid; item < 2 * M; item += kCtThreads) ct_convert<TILES>(sl, As, L.stage_bytes, M, item);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t bh = s_base + (uint32_t)(cslot * L.slot_bytes + L.slot_a);
            const uint32_t bl = bh + (uint32_t)(NP * kCtK * 2);
#pragma unroll
            for (int t = 0; t < TILES; ++t) {
                const uint32_t ahi = a_base + (uint32_t)(t * L.stage_bytes), alo = a_base + (uint32_t)((TILES + t) * L.stage_bytes);
                const uint32_t d = tmem + (uint32_t)(t * tstride);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    // K step p: the real parts (p = 0) or the imaginary parts (p = 1) of the chunk's 16 rows
                    const uint32_t o = (uint32_t)(p * 256);
                    const uint64_t dah = umma_desc(ahi + o, 128, 16 * kCtK), dal = umma_desc(alo + o, 128, 16 * kCtK);
                    const uint64_t dbh = umma_desc(bh + o, 128, 16 * kCtK), dbl = umma_desc(bl + o, 128, 16 * kCtK);
                    umma_bf16(d, dah, dbh, idesc, (c > 0 || p > 0) ? 1u : 0u);
                    umma_bf16(d, dah, dbl, idesc, 1u);
                    umma_bf16(d, dal, dbh, idesc, 1u);
                }
            }
            umma_commit(smem_u32(&mbar));
        }
        pending = ok;
        if (++cslot == slots) cslot = 0;
        if (++c != chunks) continue;
        c = 0;

        // ---- the window's last chunk: T from tensor memory, then the second contraction
        {
            const bool d2 = settle();
            const bool all2 = __syncthreads_and(d2 ? 1 : 0) != 0;
            if (ok && !all2 && tid == 0 && P.status) atomicOr(P.status, 2);
            ok = ok && all2;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (warp < 4) {
            // lanes = the tile's columns i; T [n'][i] for n' < 2G, NaN after an expired wait
#pragma unroll
            for (int t = 0; t < TILES; ++t) {
                const int i = t * 128 + 32 * warp + lane;
                for (int cb = 0; cb < 2 * G; cb += 16) {
                    float tv[16];
                    if (ok) tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t * tstride + cb), tv);
                    if (i < M) {
#pragma unroll
                        for (int r = 0; r < 16; ++r)
                            if (cb + r < 2 * G) Ts[(cb + r) * XP + i] = ok ? tv[r] : __int_as_float(0x7fc00000);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (B.coefs) {
            // c_mn = sum_i X_m[i] (T_r[n][i] + i T_i[n][i]) over 2 x 2 blocks of modes (m0, m0 + 1) x (n0, n0 + 1)
            // with m0 + n0 < G, in bm-major order; eight lanes per block take i = s, s + 8, ... and are summed in a
            // fixed butterfly order
            float2* cf = B.coefs + (size_t)((B.frame0 + fb) * P.pols + pol) * modes;
            const int lb = (G - 1) / 2, nblk = (lb + 1) * (lb + 2) / 2;
            for (int b0 = 0; b0 < nblk; b0 += kCtThreads / kCtSplit) {
                const int blk = b0 + tid / kCtSplit, s = tid % kCtSplit;
                float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                int m0 = 0, n0 = 0;
                if (blk < nblk) {
                    int bm = 0, rem = blk;
                    while (rem > lb - bm) {
                        rem -= lb - bm + 1;
                        ++bm;
                    }
                    m0 = 2 * bm;
                    n0 = 2 * rem;
                    const int m1 = m0 + 1 < G ? m0 + 1 : m0, n1 = n0 + 1 < G ? n0 + 1 : n0;
                    const float2 *x0 = X + m0 * XP, *x1 = X + m1 * XP;
                    const float *r0 = Ts + n0 * XP, *i0 = Ts + (G + n0) * XP;
                    const float *r1 = Ts + n1 * XP, *i1 = Ts + (G + n1) * XP;
                    for (int i = s; i < M; i += kCtSplit) {
                        const float2 xa = x0[i], xb = x1[i];
                        const float ta = r0[i], tb = i0[i], tc = r1[i], td = i1[i];
                        a[0] = fmaf(xa.x, ta, fmaf(-xa.y, tb, a[0]));
                        a[1] = fmaf(xa.x, tb, fmaf(xa.y, ta, a[1]));
                        a[2] = fmaf(xa.x, tc, fmaf(-xa.y, td, a[2]));
                        a[3] = fmaf(xa.x, td, fmaf(xa.y, tc, a[3]));
                        a[4] = fmaf(xb.x, ta, fmaf(-xb.y, tb, a[4]));
                        a[5] = fmaf(xb.x, tb, fmaf(xb.y, ta, a[5]));
                        a[6] = fmaf(xb.x, tc, fmaf(-xb.y, td, a[6]));
                        a[7] = fmaf(xb.x, td, fmaf(xb.y, tc, a[7]));
                    }
                }
#pragma unroll
                for (int o = kCtSplit / 2; o > 0; o >>= 1)
#pragma unroll
                    for (int k = 0; k < 8; ++k) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
                if (blk < nblk && s == 0) {
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                        for (int dn = 0; dn < 2; ++dn) {
                            const int m = m0 + dm, n = n0 + dn, g = m + n;
                            if (m < G && n < G && g < G)
                                cf[g * (g + 1) / 2 + m] = make_float2(a[4 * dm + 2 * dn], a[4 * dm + 2 * dn + 1]);
                        }
                }
            }
        }
        __syncthreads();   // T is read before the next window's chunks overwrite the A stage it aliases
        if (j + 1 < total && M % 128 != 0) {
            // T covered the padding rows of the last tile: clear them again (both planes)
            const int r0 = M - (TILES - 1) * 128;
            for (int pl = 0; pl < 2; ++pl) {
                __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(As + (size_t)(pl * TILES + (TILES - 1)) * L.stage_bytes);
                for (int e = tid; e < (128 - r0) * kCtK; e += kCtThreads)
                    tb[umma_off(r0 + e / kCtK, e % kCtK, kCtK)] = __float2bfloat16_rn(0.f);
            }
        }
        fb += fstride;
    }
    cp_async_wait(0);
    // products still in flight (only after an expired wait) complete before their tensor memory is freed
    if (!ok && tid == 0) bounded_mbar_wait(smem_u32(&mbar), lost, kCtWait);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) tmem_free(tmem, tcols);
}

namespace {

template <int TILES, bool SCORE>
cudaError_t ct_attr(int bytes) {
    return cudaFuncSetAttribute(k_coef_tc<TILES, SCORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int ct_tiles(int M) { return (M + 127) / 128; }

// Ring slots for a plan: the most (up to 4) whose layout fits shared memory, 0 if not even 2 fit.
int ct_slots(const Plan& P) {
    const int tiles = ct_tiles(P.m);
    for (int s = 4; s >= 2; --s)
        if (ct_layout(P.m, P.coef_np, P.groups, tiles, s).bytes <= (size_t)kCtSmemLimit) return s;
    return 0;
}

// The plan's geometry fits the kernel: split precision, a basis, coefficients without fields, M a multiple of
// 16 and at most 384, at least two ring slots in shared memory, the accumulators in tensor memory.
bool ct_fits(const Plan& P, const Batch& B) {
    if (P.precision != DH_PRECISION_SPLIT_BF16 || B.fields || !B.coefs || P.coef_np <= 0 || P.groups <= 0) return false;
    if (P.m % kCtQ != 0 || P.m > 384 || P.coef_np < 2 * P.groups) return false;
    return ct_slots(P) >= 2 && ct_tmem_cols(ct_tiles(P.m), P.coef_np) <= 256;
}

template <bool SCORE>
cudaError_t ct_launch(const Plan& P, const Batch& B, const BoxSrc& S, cudaStream_t st) {
    const int tiles = ct_tiles(P.m), slots = ct_slots(P);
    const CtLayout L = ct_layout(P.m, P.coef_np, P.groups, tiles, slots);
    // a persistent grid: the blocks that fit the device at once, a multiple of the polarisation count, each
    // serving one polarisation
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = tiles == 1   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coef_tc<1, SCORE>, kCtThreads, L.bytes)
                    : tiles == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coef_tc<2, SCORE>, kCtThreads, L.bytes)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coef_tc<3, SCORE>, kCtThreads, L.bytes);
    if (e != cudaSuccess) return e;
    const long long per_pol = std::min<long long>(B.count, std::max(1, sms * std::max(per_sm, 1) / P.pols));
    dim3 grid((unsigned)(per_pol * P.pols));
    switch (tiles) {
        case 1: k_coef_tc<1, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S, slots); break;
        case 2: k_coef_tc<2, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S, slots); break;
        default: k_coef_tc<3, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S, slots); break;
    }
    return cudaGetLastError();
}

}  // namespace

bool coef_tc_supported(const Plan& P, const Batch& B) {
    // the rows are copied in 16-byte pieces
    if (!ct_fits(P, B) || !B.g || (reinterpret_cast<uintptr_t>(B.g) & 15) != 0) return false;
    for (int p = 0; p < P.pols; ++p)
        if (!P.pol[p].coef_tc) return false;
    return true;
}

bool score_tc_supported(const Plan& P, const Batch& B) {
    if (!ct_fits(P, B)) return false;
    for (int p = 0; p < P.pols; ++p)
        if (!P.pol[p].score_tc) return false;
    return true;
}

cudaError_t coef_tc_init() {
    cudaError_t e;
    if ((e = ct_attr<1, false>(kCtSmemLimit))) return e;
    if ((e = ct_attr<2, false>(kCtSmemLimit))) return e;
    if ((e = ct_attr<3, false>(kCtSmemLimit))) return e;
    if ((e = ct_attr<1, true>(kCtSmemLimit))) return e;
    if ((e = ct_attr<2, true>(kCtSmemLimit))) return e;
    return ct_attr<3, true>(kCtSmemLimit);
}

cudaError_t launch_coef_tc(const Plan& P, const Batch& B, cudaStream_t st) {
    const BoxSrc none{};
    return ct_launch<false>(P, B, none, st);
}

cudaError_t launch_score_tc(const Plan& P, const Batch& B, const BoxSrc& S, cudaStream_t st) {
    return ct_launch<true>(P, B, S, st);
}

}  // namespace dhk
