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
// as bfloat16 hi + lo (canonical K-major, from the plan), A = g split into bfloat16 hi + lo as it is read.
// Three products per K step (hi hi + hi lo + lo hi), FP32 accumulation in tensor memory.  K advances in chunks
// of 16 window rows through a double-buffered A stage: the block fills one stage while the tensor cores read
// the other.  The accumulator is read back by four warps with tcgen05.ld and the second contraction (one
// complex dot product of length M per mode) runs on CUDA cores in a fixed order.
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
constexpr long kCtWait = 1L << 24;

struct CtLayout {
    size_t b, a, x, md, mk, bytes;
    int stage_bytes;                     // one plane of one tile of one stage
};

__host__ __device__ inline CtLayout ct_layout(int M, int NP, int G, int modes, int tiles, int stages) {
    CtLayout L;
    L.b = 0;                                                   // bf16 [2][NP][2M]
    L.a = ((size_t)2 * NP * 2 * M * 2 + 1023) & ~(size_t)1023; // bf16 [stages][2][tiles][128][32]
    L.stage_bytes = 128 * kCtK * 2;
    L.x = L.a + (size_t)stages * 2 * tiles * L.stage_bytes;    // float2 [G][M + 1] (odd pitch: the modes of a
                                                               // half-warp read distinct banks)
    L.md = L.x + (size_t)G * (M + 1) * 8;                      // int mode_m[modes], mode_n[modes]
    L.mk = L.md + (size_t)2 * modes * 4;                       // int mask_lo[M], mask_hi[M] (box source)
    L.bytes = (L.mk + (size_t)2 * M * 4 + 1023) & ~(size_t)1023;
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

// One item of a K chunk: field column i = item mod M and eight consecutive window rows (half item / M), so
// that consecutive threads read consecutive columns and write the eight rows of one core matrix.
__device__ __forceinline__ void ct_load(const float2* g, int M, int q0, int item, float2* v) {
    const int qh = item >= M, i = item - qh * M;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = __ldg(g + (size_t)(q0 + 8 * qh + r) * M + i);
}

// The same item read from a candidate's raw box bins (w: the box's row 0, column 0; row pitch msx), zero outside
// the kept column range [mlo[q], mhi[q]] of its row: box column p takes the place of field column i.
__device__ __forceinline__ void cs_load(const float2* w, int msx, int M, int q0, int item, const int* mlo, const int* mhi,
                                        float2* v) {
    const int qh = item >= M, p = item - qh * M;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int q = q0 + 8 * qh + r;
        v[r] = (p >= mlo[q] && p <= mhi[q]) ? __ldg(w + (size_t)q * msx + p) : make_float2(0.f, 0.f);
    }
}

// The item's values as bfloat16 hi and lo parts in the stage's A planes (row i of tile i / 128; K: the eight
// rows' real parts at 8 (item & 1), their imaginary parts 16 further).
template <int TILES>
__device__ __forceinline__ void ct_store(unsigned char* sb, int stage_bytes, int M, int item, const float2* v) {
    const int qh = item >= M, i = item - qh * M;
    __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        rh[r] = __float2bfloat16_rn(v[r].x);
        ih[r] = __float2bfloat16_rn(v[r].y);
        rl[r] = __float2bfloat16_rn(v[r].x - __bfloat162float(rh[r]));
        il[r] = __float2bfloat16_rn(v[r].y - __bfloat162float(ih[r]));
    }
    const int t = i >> 7, row = i & 127;
    __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(sb + (size_t)t * stage_bytes);
    __nv_bfloat16* lo = reinterpret_cast<__nv_bfloat16*>(sb + (size_t)(TILES + t) * stage_bytes);
    *reinterpret_cast<uint4*>(hi + umma_off(row, 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(rh);
    *reinterpret_cast<uint4*>(hi + umma_off(row, kCtQ + 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(ih);
    *reinterpret_cast<uint4*>(lo + umma_off(row, 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(rl);
    *reinterpret_cast<uint4*>(lo + umma_off(row, kCtQ + 8 * qh, kCtK)) = *reinterpret_cast<const uint4*>(il);
}

// TILES: 128-row tiles of field columns (M <= 128 TILES); STAGES: A stages (2: double-buffered).  A persistent
// grid: every block serves one polarisation (its tables are staged once) and a stride of that polarisation's
// windows.  Each thread keeps the next chunk's items in registers while the current chunk is multiplied.
// SCORE: the A rows come from a candidate's raw box bins (BoxSrc) and the tables are its scoring tables;
// otherwise from the x-inverse-transformed rows in B.g with the coefficient-only tables.
template <int TILES, int STAGES, bool SCORE>
__global__ void __launch_bounds__(kCtThreads, 1) k_coef_tc(const __grid_constant__ Plan P, const __grid_constant__ Batch B,
                                                           const __grid_constant__ BoxSrc S) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = P.m, G = P.groups, NP = P.coef_np, K = 2 * M, modes = P.modes;
    const CtLayout L = ct_layout(M, NP, G, modes, TILES, STAGES);
    const uint32_t tcols = ct_tmem_cols(TILES, NP);
    const int tstride = ct_tstride(NP);
    const int pol = blockIdx.x % P.pols;
    const PolDev& pd = P.pol[pol];
    __nv_bfloat16* Ab = reinterpret_cast<__nv_bfloat16*>(sm + L.a);
    float* Ts = reinterpret_cast<float*>(sm + L.a);            // after the products: T [NP][M + 1]
    const float2* X = reinterpret_cast<const float2*>(sm + L.x);
    int* mdm = reinterpret_cast<int*>(sm + L.md);
    int* mdn = mdm + modes;
    int* mlo = reinterpret_cast<int*>(sm + L.mk);
    int* mhi = mlo + M;
    const unsigned char* tab = SCORE ? pd.score_tc : pd.coef_tc;
    {
        // the y map (both planes) and the x weights, 16 bytes at a time; the A stages start zero, so the
        // rows past M of the last tile stay zero
        const uint4* src = reinterpret_cast<const uint4*>(tab);
        uint4* dst = reinterpret_cast<uint4*>(sm + L.b);
        const int nb = (2 * NP * K * 2) / 16;
        for (int i = tid; i < nb; i += kCtThreads) dst[i] = __ldg(src + i);
        const float2* srcx = reinterpret_cast<const float2*>(tab + (size_t)2 * NP * K * 2);
        float2* dstx = reinterpret_cast<float2*>(sm + L.x);
        for (int i = tid; i < G * M; i += kCtThreads) dstx[(i / M) * (M + 1) + i % M] = __ldg(srcx + i);
        uint4* a4 = reinterpret_cast<uint4*>(sm + L.a);
        const int na = (STAGES * 2 * TILES * L.stage_bytes) / 16;
        for (int i = tid; i < na; i += kCtThreads) a4[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = tid; i < modes; i += kCtThreads) {
            mdm[i] = P.mode_m[i];
            mdn[i] = P.mode_n[i];
        }
        if (SCORE)
            for (int i = tid; i < M; i += kCtThreads) {
                mlo[i] = pd.mask_lo[i];
                mhi[i] = pd.mask_hi[i];
            }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), tcols);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t a_base = smem_u32(Ab), b_hi = smem_u32(sm + L.b), b_lo = b_hi + NP * K * 2;
    const uint32_t idesc = umma_idesc_bf16(128, NP);
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool ok = true;                       // every wait so far completed (the same in every thread)
    const int chunks = M / kCtQ, items = 2 * M;
    const int fstride = gridDim.x / P.pols;
    constexpr int IPT = 2;                // items per thread per chunk (2M <= IPT * threads)
    float2 v[IPT][8];
    // window fb's A rows: the x-inverse-transformed rows, or the candidate's box in the superset spectra
    const size_t wstride = SCORE ? (size_t)S.ms * S.msx : (size_t)M * M;
    const float2* src0 = SCORE ? S.xs + (size_t)S.qoff[pol] * S.msx + S.poff[pol] : B.g;
    auto load = [&](const float2* w, int q0, int item, float2* vv) {
        if constexpr (SCORE)
            cs_load(w, S.msx, M, q0, item, mlo, mhi, vv);
        else
            ct_load(w, M, q0, item, vv);
    };
    int fb = blockIdx.x / P.pols;
    if (fb < B.count) {
        const float2* g0 = src0 + (size_t)(fb * P.pols + pol) * wstride;
#pragma unroll
        for (int u = 0; u < IPT; ++u)
            if (tid + u * kCtThreads < items) load(g0, 0, tid + u * kCtThreads, v[u]);
    }
    for (; fb < B.count; fb += fstride) {
        const int f = B.frame0 + fb;
        const float2* g = src0 + (size_t)(fb * P.pols + pol) * wstride;
        for (int c = 0; c < chunks; ++c) {
            const int st = STAGES == 2 ? (c & 1) : 0;
            if (pending[st]) {
                // the products that read this stage earlier must be done before it is refilled; one thread
                // waits, the block barrier passes its finding (and the ordering) to the others
                const bool done = ok && (tid != 0 || bounded_mbar_wait(smem_u32(&mbar[st]), phase[st], kCtWait));
                phase[st] ^= 1u;
                pending[st] = false;
                const bool all = __syncthreads_and(done ? 1 : 0) != 0;
                if (ok && !all && tid == 0 && P.status) atomicOr(P.status, 2);
                ok = ok && all;
            }
            unsigned char* sb = sm + L.a + (size_t)st * 2 * TILES * L.stage_bytes;
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                if (tid + u * kCtThreads < items) ct_store<TILES>(sb, L.stage_bytes, M, tid + u * kCtThreads, v[u]);
            // the next chunk's items (or the next window's first chunk) in flight while this one is multiplied
            {
                const bool more = c + 1 < chunks;
                const int nfb = more ? fb : fb + fstride;
                if (nfb < B.count) {
                    const float2* gn = more ? g : src0 + (size_t)(nfb * P.pols + pol) * wstride;
#pragma unroll
                    for (int u = 0; u < IPT; ++u)
                        if (tid + u * kCtThreads < items) load(gn, more ? (c + 1) * kCtQ : 0, tid + u * kCtThreads, v[u]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0 && ok) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int q0 = c * kCtQ;
                const uint32_t sa = a_base + (uint32_t)(st * 2 * TILES * L.stage_bytes);
#pragma unroll
                for (int t = 0; t < TILES; ++t) {
                    const uint32_t ahi = sa + (uint32_t)(t * L.stage_bytes), alo = sa + (uint32_t)((TILES + t) * L.stage_bytes);
                    const uint32_t d = tmem + (uint32_t)(t * tstride);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        // this chunk's rows of part p: A columns 16 p .. 16 p + 15, B columns p M + q0 ..
                        const uint32_t ao = (uint32_t)(p * 2 * 128), bo = (uint32_t)((p * M + q0) / 8 * 128);
                        const uint64_t dah = umma_desc(ahi + ao, 128, 16 * kCtK), dal = umma_desc(alo + ao, 128, 16 * kCtK);
                        const uint64_t dbh = umma_desc(b_hi + bo, 128, 16 * K), dbl = umma_desc(b_lo + bo, 128, 16 * K);
                        umma_bf16(d, dah, dbh, idesc, (c > 0 || p > 0) ? 1u : 0u);
                        umma_bf16(d, dah, dbl, idesc, 1u);
                        umma_bf16(d, dal, dbh, idesc, 1u);
                    }
                }
                umma_commit(smem_u32(&mbar[st]));
            }
            pending[st] = ok;
        }
        // every product of this window complete
        for (int s2 = 0; s2 < STAGES; ++s2) {
            if (!pending[s2]) continue;
            const bool done = ok && (tid != 0 || bounded_mbar_wait(smem_u32(&mbar[s2]), phase[s2], kCtWait));
            phase[s2] ^= 1u;
            pending[s2] = false;
            const bool all = __syncthreads_and(done ? 1 : 0) != 0;
            if (ok && !all && tid == 0 && P.status) atomicOr(P.status, 2);
            ok = ok && all;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // T[n'][i] from tensor memory (lanes = field columns of the tile), over the A stages
        if (warp < 4) {
#pragma unroll
            for (int t = 0; t < TILES; ++t) {
                const int i = t * 128 + 32 * warp + lane;
                for (int cb = 0; cb < NP; cb += 16) {
                    float tv[16];
                    if (ok) tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t * tstride + cb), tv);
                    if (i < M) {
#pragma unroll
                        for (int r = 0; r < 16; ++r) Ts[(cb + r) * (M + 1) + i] = ok ? tv[r] : __int_as_float(0x7fc00000);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        // c_mn = sum_i X_m[i] (T_r[n][i] + i T_i[n][i]): two threads per mode (even and odd i, each in order),
        // summed in a fixed order
        if (B.coefs) {
            float2* cf = B.coefs + (size_t)(f * P.pols + pol) * modes;
            for (int k0 = 0; k0 < modes; k0 += kCtThreads / 2) {
                const int k = k0 + (tid >> 1), h = tid & 1;
                float2 acc = make_float2(0.f, 0.f);
                if (k < modes) {
                    const float2* xm = X + (size_t)mdm[k] * (M + 1);
                    const float* tr = Ts + (size_t)mdn[k] * (M + 1);
                    const float* ti = Ts + (size_t)(G + mdn[k]) * (M + 1);
                    for (int i = h; i < M; i += 2) {
                        const float2 x = xm[i];
                        const float a = tr[i], b = ti[i];
                        acc.x = fmaf(x.x, a, fmaf(-x.y, b, acc.x));
                        acc.y = fmaf(x.x, b, fmaf(x.y, a, acc.y));
                    }
                }
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
                if (k < modes && h == 0) cf[k] = acc;
            }
        }
        __syncthreads();   // T is read before the next window refills the A stages (T aliases them)
        if (fb + fstride < B.count && M % 128 != 0) {
            // the aliased stages held T: clear the padding rows of the last tile again
            const int r0 = M - (TILES - 1) * 128;
            for (int s2 = 0; s2 < STAGES; ++s2)
                for (int pl = 0; pl < 2; ++pl) {
                    __nv_bfloat16* tbh = reinterpret_cast<__nv_bfloat16*>(
                        sm + L.a + (size_t)(s2 * 2 * TILES + pl * TILES + (TILES - 1)) * L.stage_bytes);
                    for (int e = tid; e < (128 - r0) * kCtK; e += kCtThreads)
                        tbh[umma_off(r0 + e / kCtK, e % kCtK, kCtK)] = __float2bfloat16_rn(0.f);
                }
            __syncthreads();
        }
    }
    // products still in flight (only after an expired wait) complete before their tensor memory is freed
    if (!ok && tid == 0)
        for (int s2 = 0; s2 < STAGES; ++s2) bounded_mbar_wait(smem_u32(&mbar[s2]), phase[s2], kCtWait);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) tmem_free(tmem, tcols);
}

namespace {

template <int TILES, int STAGES, bool SCORE>
cudaError_t ct_attr(int bytes) {
    return cudaFuncSetAttribute(k_coef_tc<TILES, STAGES, SCORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int ct_tiles(int M) { return (M + 127) / 128; }
int ct_stages(int tiles) { return tiles <= 2 ? 2 : 1; }

}  // namespace

// The plan's geometry fits the kernel: split precision, a basis, coefficients without fields, M a multiple of
// 16 and at most 384, the tables and stages in shared memory, T within the stages, the accumulators in TMEM.
static bool ct_fits(const Plan& P, const Batch& B) {
    if (P.precision != DH_PRECISION_SPLIT_BF16 || B.fields || !B.coefs || P.coef_np <= 0 || P.groups <= 0) return false;
    if (P.m % kCtQ != 0 || P.m > 384 || 2 * P.m > 2 * kCtThreads) return false;
    const int tiles = ct_tiles(P.m);
    const CtLayout L = ct_layout(P.m, P.coef_np, P.groups, P.modes, tiles, ct_stages(tiles));
    // T [NP][M + 1] floats aliases the A stages
    const size_t ts = (size_t)P.coef_np * (P.m + 1) * 4;
    return L.bytes <= 227 * 1024 - 1024 && ts <= L.x - L.a && ct_tmem_cols(tiles, P.coef_np) <= 256;
}

bool coef_tc_supported(const Plan& P, const Batch& B) {
    if (!ct_fits(P, B)) return false;
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
    const int lim = 227 * 1024 - 1024;
    if ((e = ct_attr<1, 2, false>(lim))) return e;
    if ((e = ct_attr<2, 2, false>(lim))) return e;
    if ((e = ct_attr<3, 1, false>(lim))) return e;
    if ((e = ct_attr<1, 2, true>(lim))) return e;
    if ((e = ct_attr<2, 2, true>(lim))) return e;
    return ct_attr<3, 1, true>(lim);
}

namespace {

template <bool SCORE>
cudaError_t ct_launch(const Plan& P, const Batch& B, const BoxSrc& S, cudaStream_t st) {
    const int tiles = ct_tiles(P.m), stages = ct_stages(tiles);
    const CtLayout L = ct_layout(P.m, P.coef_np, P.groups, P.modes, tiles, stages);
    // a persistent grid: the blocks that fit the device at once (shared memory allows one or two per SM), a
    // multiple of the polarisation count, each serving one polarisation
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = tiles == 1   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coef_tc<1, 2, SCORE>, kCtThreads, L.bytes)
                    : tiles == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coef_tc<2, 2, SCORE>, kCtThreads, L.bytes)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coef_tc<3, 1, SCORE>, kCtThreads, L.bytes);
    if (e != cudaSuccess) return e;
    const long long per_pol = std::min<long long>(B.count, std::max(1, sms * std::max(per_sm, 1) / P.pols));
    dim3 grid((unsigned)(per_pol * P.pols));
    switch (tiles) {
        case 1: k_coef_tc<1, 2, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S); break;
        case 2: k_coef_tc<2, 2, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S); break;
        default: k_coef_tc<3, 1, SCORE><<<grid, kCtThreads, L.bytes, st>>>(P, B, S); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_coef_tc(const Plan& P, const Batch& B, cudaStream_t st) {
    const BoxSrc none{};
    return ct_launch<false>(P, B, none, st);
}

cudaError_t launch_score_tc(const Plan& P, const Batch& B, const BoxSrc& S, cudaStream_t st) {
    return ct_launch<true>(P, B, S, st);
}

}  // namespace dhk
