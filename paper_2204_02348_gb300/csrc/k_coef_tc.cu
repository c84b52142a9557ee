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
// Data movement.  K advances in chunks of 16 window rows.  A producer thread brings each chunk (its 16 rows of
// A as FP32 and its slice of B, 128 np bytes) into one slot of a ring in shared memory with bulk asynchronous
// copies, several chunks ahead and across window boundaries.  Twelve warps split each landed chunk into
// bfloat16 hi / lo in the canonical K-major layout of an A stage (two stages: one is split while the other is
// multiplied); one thread issues the products into the window's accumulator buffer (two buffers in tensor
// memory); eight warps read each finished accumulator back with tcgen05.ld and form the coefficients (a complex
// dot product of length M per mode, eight lanes per 2 x 2 block of modes, summed in a fixed order) while the
// next window accumulates.  The roles meet only at mbarriers.
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

constexpr int kCtThreads = 704;          // 22 warps
constexpr int kCtE = 256;                // epilogue: warps 0-3 and 18-21, two per tensor-memory lane quadrant
constexpr int kCtProd = 4, kCtMma = 5;   // one warp each: the bulk copies, the products (lane 0 works)
constexpr int kCtC0 = 6 * 32;            // split: warps 6-17
constexpr int kCtC = 12 * 32;
constexpr int kCtE1 = 18;                // first warp of the epilogue's second half
constexpr int kCtQ = 16;                 // window rows per K chunk (K = 32 per chunk: real, then imaginary)
constexpr int kCtK = 2 * kCtQ;
constexpr int kCtSplit = 8;              // lanes per 2 x 2 block of modes in the second contraction
constexpr long kCtWait = 1L << 24;
constexpr int kCtSmemLimit = 227 * 1024 - 1024;
constexpr int kCtMaxSlots = 5;

struct CtLayout {
    int stage_bytes;                     // one plane of one tile of an A stage (128 rows x 32 K, bf16)
    int apitch;                          // row pitch of A in a slot (float2): M, or M + 2 for box rows (16-byte slack)
    int slot_a, slot_b, slot_bytes;      // one ring slot: 16 rows of A as float2 [16][apitch], then B [2][NP][32] bf16
    size_t a;                            // A stages [stages][2][tiles][128][32] bf16
    size_t s;                            // ring [slots]
    size_t t;                            // T [2G][M + 4] FP32, the accumulator of one window read back
    size_t mk;                           // int2 kept column range of each box row [M] (box source)
    size_t bytes;
};

__host__ __device__ inline CtLayout ct_layout(int M, int NP, int G, int tiles, int stages, int slots, bool box) {
    CtLayout L;
    L.stage_bytes = 128 * kCtK * 2;
    L.apitch = box ? M + 2 : M;
    L.slot_a = kCtQ * L.apitch * 8;
    L.slot_b = 2 * NP * kCtK * 2;
    L.slot_bytes = (L.slot_a + L.slot_b + 127) & ~127;
    L.a = 0;
    L.s = (L.a + (size_t)stages * 2 * tiles * L.stage_bytes + 1023) & ~(size_t)1023;
    L.t = L.s + (size_t)slots * L.slot_bytes;
    L.mk = L.t + (((size_t)2 * G * (M + 4) * 4 + 15) & ~(size_t)15);
    L.bytes = (L.mk + (size_t)M * 8 + 1023) & ~(size_t)1023;
    return L;
}

// Tensor-memory column stride of one tile's accumulator (NP rounded up to 32); accumulator buffers (two, so the
// epilogue reads one window while the next accumulates, when they fit the 256 columns); the columns to allocate
// (a power of two >= 32).
__host__ __device__ inline int ct_tstride(int NP) { return (NP + 31) & ~31; }
__host__ __device__ inline int ct_accs(int tiles, int NP) { return 2 * tiles * ct_tstride(NP) <= 256 ? 2 : 1; }
__host__ __device__ inline uint32_t ct_tmem_cols(int tiles, int NP) {
    uint32_t c = 32;
    while (c < (uint32_t)(ct_accs(tiles, NP) * tiles * ct_tstride(NP))) c <<= 1;
    return c;
}

}  // namespace

// Bulk asynchronous copy global -> shared (async proxy; 16-byte aligned addresses, size a multiple of 16),
// completing `bytes` on the mbarrier; and the arrival that announces those bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// Named barrier `id` over the n threads (whole warps) that use it: plain, and with an AND of a predicate.
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ bool bar_and(int id, int n, bool v) {
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// One item of a chunk: field (or box) column i = item mod M and eight consecutive rows of the chunk (half
// item / M), read from the slot's FP32 rows (element i of row r at slot[r pitch + off + i]; with a mask, box
// column i of chunk row r is kept only in [mk[r].x, mk[r].y]) and stored as bfloat16 hi and lo in the A stage
// (row i of tile i / 128; K: the eight rows' real parts at 8 (half), their imaginary parts 16 further).
// Consecutive threads take consecutive columns: the slot reads and the 16-byte stores are free of bank conflicts.
template <int TILES>
__device__ __forceinline__ void ct_convert(const float2* slot, int pitch, int off, const int2* mk, unsigned char* sa,
                                           int stage_bytes, int M, int item) {
    const int qh = item >= M, i = item - qh * M;
    __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        float2 v = slot[(8 * qh + r) * pitch + off + i];
        if (mk) {
            const int2 k = mk[8 * qh + r];
            if (i < k.x || i > k.y) v = make_float2(0.f, 0.f);
        }
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

// SCORE: the A rows are a candidate's raw box bins (BoxSrc; bins outside a row's kept range count as zero) and
// the tables its scoring tables; otherwise the x-inverse-transformed rows in B.g with the coefficient-only
// tables.  A persistent grid: every block serves one polarisation and a stride of that polarisation's windows,
// whose chunks form one stream.  Four roles meet only at mbarriers (every wait bounded):
//   producer (warp 4, lane 0)  bulk copies of chunk j into ring slot j mod slots once the slot is free;
//   split (warps 6-17)         chunk j from its slot into A stage j mod stages once the stage is free;
//   products (warp 5, lane 0)  the chunk's tcgen05 products into the window's accumulator buffer, which then
//                              frees the stage and (with the split) the slot, and after a window's last chunk
//                              marks the buffer full;
//   epilogue (warps 0-3, 18-21) each full buffer read back, released, and contracted into the coefficients.
template <int TILES, bool SCORE>
__global__ void __launch_bounds__(kCtThreads, 1) k_coef_tc(const __grid_constant__ Plan P, const __grid_constant__ Batch B,
                                                           const __grid_constant__ BoxSrc S, int stages, int slots) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mb_sfull[kCtMaxSlots], mb_sfree[kCtMaxSlots], mb_afull[2], mb_afree[2];
    __shared__ __align__(8) uint64_t mb_accf[2], mb_acce[2], mb_fin;
    __shared__ uint32_t tmem_slot;
    __shared__ int err;                   // a wait expired somewhere; no role waits any more
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = P.m, G = P.groups, NP = P.coef_np, modes = P.modes, chunks = M / kCtQ;
    const int XP = M + 4;                 // pitch of T rows (floats): rows two apart are eight banks apart
    const CtLayout L = ct_layout(M, NP, G, TILES, stages, slots, SCORE);
    const int tstride = ct_tstride(NP), accs = ct_accs(TILES, NP);
    const uint32_t tcols = ct_tmem_cols(TILES, NP);
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    const unsigned char* tab = SCORE ? pd.score_tc : pd.coef_tc;
    unsigned char* As = sm + L.a;
    float* Ts = reinterpret_cast<float*>(sm + L.t);
    int2* mk = reinterpret_cast<int2*>(sm + L.mk);
    volatile int* errp = &err;
    {
        // the A stages start zero, so rows past M of the last tile contribute nothing
        uint4* a4 = reinterpret_cast<uint4*>(As);
        for (int i = tid; i < (stages * 2 * TILES * L.stage_bytes) / 16; i += kCtThreads) a4[i] = make_uint4(0u, 0u, 0u, 0u);
        if (SCORE)
            for (int i = tid; i < M; i += kCtThreads) mk[i] = make_int2(pd.mask_lo[i], pd.mask_hi[i]);
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), tcols);
    if (tid == 0) {
        for (int k = 0; k < kCtMaxSlots; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mb_sfull[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;\n" ::"r"(smem_u32(&mb_sfree[k])));   // split + products
        }
        for (int k = 0; k < 2; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mb_afull[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mb_afree[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mb_accf[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mb_acce[k])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mb_fin)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        err = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // the zeroed stages, before any product
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    // this block's windows fb0, fb0 + fstride, ... and its stream of chunks
    const int fb0 = blockIdx.x / P.pols, fstride = gridDim.x / P.pols;
    const int nwin = fb0 < B.count ? (B.count - 1 - fb0) / fstride + 1 : 0;
    const long total = (long)nwin * chunks;
    // a wait by one thread: false once a wait anywhere has expired (then nobody waits again)
    auto wait = [&](uint64_t* mb, uint32_t parity) -> bool {
        if (*errp) return false;
        if (bounded_mbar_wait(smem_u32(mb), parity, kCtWait)) return true;
        *errp = 1;
        if (P.status) atomicOr(P.status, 2);
        return false;
    };

    if (warp == kCtProd) {
        // ================================================================ producer
        if (lane == 0) {
            const size_t wstride = SCORE ? (size_t)S.ms * S.msx : (size_t)M * M;
            uint32_t ph_free = 0u;        // parity bit per slot
            int c = 0, fb = fb0, s = 0;
            for (long j = 0; j < total; ++j) {
                if (j >= slots && !wait(&mb_sfree[s], (ph_free >> s) & 1u)) break;
                if (j >= slots) ph_free ^= 1u << s;
                const uint32_t dst = smem_u32(sm + L.s + (size_t)s * L.slot_bytes), mb = smem_u32(&mb_sfull[s]);
                if constexpr (SCORE) {
                    // 16 box rows; a row that starts 8 bytes past a 16-byte boundary is copied from 8 bytes earlier
                    // with 16 more bytes (every row of the window has the same offset: msx is even)
                    const float2* r0 = S.xs + (size_t)(fb * P.pols + pol) * wstride +
                                       (size_t)(S.qoff[pol] + kCtQ * c) * S.msx + S.poff[pol];
                    const int off = (int)((reinterpret_cast<uintptr_t>(r0) >> 3) & 1);
                    const uint32_t rb = (uint32_t)(M * 8 + 16 * off);
                    // the chunk's first and last copied elements inside the superset spectra (else no copy: the
                    // slot keeps stale values, the guard is recorded)
                    const long long e0 = (long long)(r0 - S.xs) - off;
                    const bool in = DH_IN(P.status, e0, S.xs_len, kSiteCoefTcCopy) &&
                                    DH_IN(P.status, e0 + (long long)(kCtQ - 1) * S.msx + rb / 8 - 1, S.xs_len, kSiteCoefTcCopy);
                    mbar_expect_tx(mb, (in ? (uint32_t)kCtQ * rb : 0u) + (uint32_t)L.slot_b);
                    if (in)
                        for (int r = 0; r < kCtQ; ++r)
                            bulk_g2s(dst + (uint32_t)(r * L.apitch * 8), r0 + (size_t)r * S.msx - off, rb, mb);
                } else {
                    // 16 contiguous rows of M complex values
                    const long long e0 = (long long)(fb * P.pols + pol) * wstride + (long long)(kCtQ * c) * M;
                    const bool in = DH_IN(P.status, e0 + L.slot_a / 8 - 1, B.g_len, kSiteCoefTcCopy);
                    mbar_expect_tx(mb, (uint32_t)((in ? L.slot_a : 0) + L.slot_b));
                    if (in) bulk_g2s(dst, B.g + e0, (uint32_t)L.slot_a, mb);
                }
                bulk_g2s(dst + (uint32_t)L.slot_a, tab + (size_t)c * L.slot_b, (uint32_t)L.slot_b, mb);
                if (++s == slots) s = 0;
                if (++c == chunks) {
                    c = 0;
                    fb += fstride;
                }
            }
        }
        __syncwarp();
    } else if (warp == kCtMma) {
        // ================================================================ products
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(128, NP);
            const uint32_t a_base = smem_u32(As), s_base = smem_u32(sm + L.s);
            uint32_t ph_full = 0u, ph_acce = 0u;   // parity bits per stage / per buffer
            int c = 0, w = 0, s = 0, st = 0;
            for (long j = 0; j < total; ++j) {
                const int a = w % accs;
                if (!wait(&mb_afull[st], (ph_full >> st) & 1u)) break;
                ph_full ^= 1u << st;
                if (c == 0 && w >= accs) {
                    // the epilogue has read this buffer's previous window
                    if (!wait(&mb_acce[a], (ph_acce >> a) & 1u)) break;
                    ph_acce ^= 1u << a;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t sa = a_base + (uint32_t)(st * 2 * TILES * L.stage_bytes);
                const uint32_t bh = s_base + (uint32_t)(s * L.slot_bytes + L.slot_a);
                const uint32_t bl = bh + (uint32_t)(NP * kCtK * 2);
#pragma unroll
                for (int t = 0; t < TILES; ++t) {
                    const uint32_t ahi = sa + (uint32_t)(t * L.stage_bytes), alo = sa + (uint32_t)((TILES + t) * L.stage_bytes);
                    const uint32_t d = tmem + (uint32_t)((a * TILES + t) * tstride);
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
                umma_commit(smem_u32(&mb_afree[st]));
                umma_commit(smem_u32(&mb_sfree[s]));
                if (c == chunks - 1) umma_commit(smem_u32(&mb_accf[a]));
                if (++st == stages) st = 0;
                if (++s == slots) s = 0;
                if (++c == chunks) {
                    c = 0;
                    ++w;
                }
            }
            // every product issued here is complete before the tensor memory is freed (after an expired wait some
            // may still be in flight)
            umma_commit(smem_u32(&mb_fin));
            bounded_mbar_wait(smem_u32(&mb_fin), 0u, kCtWait);
        }
        __syncwarp();
    } else if (tid >= kCtC0 && tid < kCtC0 + kCtC) {
        // ================================================================ split
        const int ct = tid - kCtC0;
        const bool lead = ct == 0;
        uint32_t ph_full = 0u, ph_free = 0u;    // parity bits per slot / per stage
        int c = 0, s = 0, st = 0;
        bool ok = true;
        for (long j = 0; j < total; ++j) {
            // the first thread waits for the chunk's copies and (for j >= stages) the stage's previous products;
            // the barrier releases the others
            bool done = true;
            if (lead) {
                done = ok && wait(&mb_sfull[s], (ph_full >> s) & 1u);
                if (j >= stages) done = done && wait(&mb_afree[st], (ph_free >> st) & 1u);
            }
            ph_full ^= 1u << s;
            if (j >= stages) ph_free ^= 1u << st;
            ok = bar_and(1, kCtC, done);
            if (ok) {
                const float2* sl = reinterpret_cast<const float2*>(sm + L.s + (size_t)s * L.slot_bytes);
                int off = 0;
                if (SCORE) off = (int)((reinterpret_cast<uintptr_t>(S.xs + (size_t)S.poff[pol]) >> 3) & 1);
                unsigned char* sa = As + (size_t)st * 2 * TILES * L.stage_bytes;
                for (int item = ct; item < 2 * M; item += kCtC)
                    ct_convert<TILES>(sl, L.apitch, off, SCORE ? mk + kCtQ * c : nullptr, sa, L.stage_bytes, M, item);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            }
            bar_sync(1, kCtC);
            if (lead && ok) {
                mbar_arrive(smem_u32(&mb_afull[st]));
                mbar_arrive(smem_u32(&mb_sfree[s]));
            }
            if (!ok) break;
            if (++st == stages) st = 0;
            if (++s == slots) s = 0;
            if (++c == chunks) c = 0;
        }
    } else {
        // ================================================================ epilogue, one window at a time
        // et: index in the group; quadrant and half: the tensor-memory lanes and the column blocks this warp reads
        const int et = warp < 4 ? tid : tid - kCtE1 * 32 + 128;
        const int quad = warp & 3, half = warp < 4 ? 0 : 1;
        uint32_t ph_accf = 0u;                 // parity bit per buffer
        bool ok = true;
        int fb = fb0;
        const float2* X = reinterpret_cast<const float2*>(tab + (size_t)chunks * L.slot_b);   // [G][M], L1/L2
        for (int w = 0; w < nwin; ++w, fb += fstride) {
            const int a = w % accs;
            bool done = true;
            if (et == 0) done = ok && wait(&mb_accf[a], (ph_accf >> a) & 1u);
            ph_accf ^= 1u << a;
            ok = bar_and(2, kCtE, done);
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // T [n'][i] for n' < 2G (lanes = the tile's columns i), NaN after an expired wait
#pragma unroll
            for (int t = 0; t < TILES; ++t) {
                const int i = t * 128 + 32 * quad + lane;
                for (int cb = 16 * half; cb < 2 * G; cb += 32) {
                    float tv[16];
                    if (ok) tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)((a * TILES + t) * tstride + cb), tv);
                    if (i < M) {
#pragma unroll
                        for (int r = 0; r < 16; ++r)
                            if (cb + r < 2 * G) Ts[(cb + r) * XP + i] = ok ? tv[r] : __int_as_float(0x7fc00000);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            bar_sync(2, kCtE);
            if (et == 0 && ok) mbar_arrive(smem_u32(&mb_acce[a]));   // the buffer may take the next window
            if (B.coefs) {
                // c_mn = sum_i X_m[i] (T_r[n][i] + i T_i[n][i]) over 2 x 2 blocks of modes (m0, m0 + 1) x (n0, n0 + 1)
                // with m0 + n0 < G, in bm-major order; eight lanes per block take i = s, s + 8, ... and are summed
                // in a fixed butterfly order
                float2* cf = B.coefs + (size_t)((B.frame0 + fb) * P.pols + pol) * modes;
                const int lb = (G - 1) / 2, nblk = (lb + 1) * (lb + 2) / 2;
                for (int b0 = 0; b0 < nblk; b0 += kCtE / kCtSplit) {
                    const int blk = b0 + et / kCtSplit, sp = et % kCtSplit;
                    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
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
                        const float2 *x0 = X + (size_t)m0 * M, *x1 = X + (size_t)m1 * M;
                        const float *r0 = Ts + n0 * XP, *i0 = Ts + (G + n0) * XP;
                        const float *r1 = Ts + n1 * XP, *i1 = Ts + (G + n1) * XP;
                        for (int i = sp; i < M; i += kCtSplit) {
                            const float2 xa = __ldg(x0 + i), xb = __ldg(x1 + i);
                            const float ta = r0[i], tb = i0[i], tc = r1[i], td = i1[i];
                            v[0] = fmaf(xa.x, ta, fmaf(-xa.y, tb, v[0]));
                            v[1] = fmaf(xa.x, tb, fmaf(xa.y, ta, v[1]));
                            v[2] = fmaf(xa.x, tc, fmaf(-xa.y, td, v[2]));
                            v[3] = fmaf(xa.x, td, fmaf(xa.y, tc, v[3]));
                            v[4] = fmaf(xb.x, ta, fmaf(-xb.y, tb, v[4]));
                            v[5] = fmaf(xb.x, tb, fmaf(xb.y, ta, v[5]));
                            v[6] = fmaf(xb.x, tc, fmaf(-xb.y, td, v[6]));
                            v[7] = fmaf(xb.x, td, fmaf(xb.y, tc, v[7]));
                        }
                    }
#pragma unroll
                    for (int o = kCtSplit / 2; o > 0; o >>= 1)
#pragma unroll
                        for (int k = 0; k < 8; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
                    if (blk < nblk && sp == 0) {
#pragma unroll
                        for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                            for (int dn = 0; dn < 2; ++dn) {
                                const int m = m0 + dm, n = n0 + dn, g = m + n;
                                if (m < G && n < G && g < G &&
                                    DH_IN(P.status, (long long)pol * modes + g * (g + 1) / 2 + m, (long long)P.pols * modes, kSiteCoefTcCoef))
                                    cf[g * (g + 1) / 2 + m] = make_float2(v[4 * dm + 2 * dn], v[4 * dm + 2 * dn + 1]);
                            }
                    }
                }
            }
            bar_sync(2, kCtE);   // T is read before the next window's readback overwrites it
        }
    }
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

// A stages and ring slots for a plan: two stages (a chunk is split while the previous one is multiplied) and as
// many slots as fit (up to five: three chunks in flight while two are split and multiplied); otherwise one stage
// with at least two slots; {0, 0} when nothing fits.
struct CtConfig {
    int stages, slots;
};
CtConfig ct_config(const Plan& P, bool box) {
    static const CtConfig order[] = {{2, 5}, {2, 4}, {1, 4}, {2, 3}, {1, 3}, {1, 2}};
    const int tiles = ct_tiles(P.m);
    for (const CtConfig& c : order)
        if (ct_layout(P.m, P.coef_np, P.groups, tiles, c.stages, c.slots, box).bytes <= (size_t)kCtSmemLimit) return c;
    return {0, 0};
}

// The plan's geometry fits the kernel: split precision, a basis, coefficients without fields, M a multiple of
// 16 and at most 384, a ring that fits shared memory, the accumulators in tensor memory.
bool ct_fits(const Plan& P, const Batch& B, bool box) {
    if (P.precision != DH_PRECISION_SPLIT_BF16 || B.fields || !B.coefs || P.coef_np <= 0 || P.groups <= 0) return false;
    if (P.m % kCtQ != 0 || P.m > 384 || P.coef_np < 2 * P.groups) return false;
    return ct_config(P, box).stages > 0 && ct_tmem_cols(ct_tiles(P.m), P.coef_np) <= 256;
}

template <bool SCORE>
cudaError_t ct_launch(const Plan& P, const Batch& B, const BoxSrc& S, cudaStream_t st) {
    const int tiles = ct_tiles(P.m);
    const CtConfig cfg = ct_config(P, SCORE);
    const CtLayout L = ct_layout(P.m, P.coef_np, P.groups, tiles, cfg.stages, cfg.slots, SCORE);
    // a persistent grid of one block per SM (the shared memory allows no more), a multiple of the polarisation
    // count, each block serving one polarisation
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int n = 148;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = n;
    }
    const long long per_pol = std::min<long long>(B.count, std::max(1, sms[dev] / P.pols));
    dim3 grid((unsigned)(per_pol * P.pols));
    switch (tiles) {
        case 1: k_coef_tc<1, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S, cfg.stages, cfg.slots); break;
        case 2: k_coef_tc<2, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S, cfg.stages, cfg.slots); break;
        default: k_coef_tc<3, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S, cfg.stages, cfg.slots); break;
    }
    return cudaGetLastError();
}

}  // namespace

bool coef_tc_supported(const Plan& P, const Batch& B) {
    // the rows are copied in bulk: 16-byte aligned; square fields only
    if (P.ny != P.n || P.my != P.m || !ct_fits(P, B, false) || !B.g || (reinterpret_cast<uintptr_t>(B.g) & 15) != 0) return false;
    for (int p = 0; p < P.pols; ++p)
        if (!P.pol[p].coef_tc) return false;
    return true;
}

bool score_tc_supported(const Plan& P, const Batch& B, const BoxSrc& S) {
    // bulk copies of the box rows: every row of a window starts at the same offset from a 16-byte boundary (an
    // even superset pitch on a 16-byte aligned base)
    if (P.ny != P.n || P.my != P.m || !ct_fits(P, B, true) || !S.xs || (reinterpret_cast<uintptr_t>(S.xs) & 15) != 0 || (S.msx & 1) != 0) return false;
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
