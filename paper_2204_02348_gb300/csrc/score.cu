// Alignment-candidate scoring: total captured power of every frame under every candidate setting (the
// quantity the guide's AutoAlign search maximises while it perturbs tilt, defocus and waist).
//
// The forward transform does not depend on the candidate except through which bins its box selects, so it
// runs once per frame on a superset box that covers every candidate's box:
//   k_ypass  (generic path, with the superset rows)  -> r1s[q][x]   (Ms x N per window)
//   k_xfwd   x transform of the superset rows, keep the superset columns -> xs[q][c] (Ms x Msx, raw DFT bins)
// and then, per candidate, only the candidate-specific work runs:
//   k_xinv_sel  gather the candidate's M x M box from xs, apply its circular mask and beam-centre phase,
//               x inverse transform                                     -> g[q][i]
//   k_yinv / k_yinv_tc  y inverse transform, correction, HG overlap with the candidate's tables -> coefficients
//   k_power     P[b][s] = sum over pols and modes of |c|^2, fixed-order warp reduction.
// Candidates whose boxes do not fit one superset of at most N rows and columns fall back to the full path.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fft.cuh"
#include "runtime.hpp"

namespace dhk {

constexpr int kSThreads = 256;

// power[(frame0 + b) * count + s0 + s] = sum over pols and modes of |c|^2 for the candidates s0 .. s0 + ns - 1 of a
// chunk (coefficients of candidate s at frame slot b: coefs[(s * cstride + b) * per_frame ...], frame index
// relative to the chunk), one warp per (frame, candidate), summed in a fixed order.
__global__ void k_power(const float2* __restrict__ coefs, int per_frame, int frame0, int frames, int ns, int s0,
                        int cstride, float* __restrict__ power, int count) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= frames * ns) return;
    const int s = w / frames, b = w - s * frames;
    const float2* c = coefs + ((size_t)s * cstride + b) * per_frame;
    float acc = 0.f;
    for (int k = lane; k < per_frame; k += 32) acc = fmaf(c[k].x, c[k].x, fmaf(c[k].y, c[k].y, acc));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) power[(size_t)(frame0 + b) * count + s0 + s] = acc;
}

struct Superset {
    int ms, msx;                  // superset rows and columns
    int klx[DH_MAX_POLS];         // first superset column bin (unwrapped)
};

// x transform of R superset rows per block; keeps the superset columns in natural order.
__global__ void __launch_bounds__(kSThreads, 2) k_xfwd(const __grid_constant__ Plan P, const __grid_constant__ Superset S,
                                                       const float2* __restrict__ r1s, float2* __restrict__ xs, int count,
                                                       int logr, int logn, long long r1s_len, long long xs_len) {
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int R = 1 << logr, es = R + 1, N = P.n;
    const int pol = blockIdx.y, q0 = blockIdx.x * R;
    for (int fb = blockIdx.z; fb < count; fb += gridDim.z) {
        const float2* src = r1s + (size_t)(fb * P.pols + pol) * S.ms * N;
        // eight independent loads in flight per thread before their shared-memory stores
        for (int i0 = tid; i0 < R * N; i0 += 8 * nthr) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                const int q = q0 + (idx >> logn);
                v[u] = (idx < R * N && q < S.ms &&
                        DH_IN(P.status, (long long)(fb * P.pols + pol) * S.ms * N + (long long)q * N + (idx & (N - 1)), r1s_len, kSiteScore))
                           ? src[(size_t)q * N + (idx & (N - 1))] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                if (idx < R * N) smem[(idx & (N - 1)) * es + (idx >> logn)] = v[u];
            }
        }
        __syncthreads();
        fft_run<false>(smem, N, P.rad_n, P.nrad_n, logr, es, P.tw_fwd_n, tid, nthr);
        float2* dst = xs + (size_t)(fb * P.pols + pol) * S.ms * S.msx;
        for (int idx = tid; idx < R * S.msx; idx += nthr) {
            const int row = idx / S.msx, c = idx - row * S.msx;
            const int q = q0 + row;
            if (q < S.ms) {
                const int kx = (S.klx[pol] + c) & (N - 1);
                if (DH_IN(P.status, (long long)(fb * P.pols + pol) * S.ms * S.msx + (long long)q * S.msx + c, xs_len, kSiteScore))
                    dst[(size_t)q * S.msx + c] = smem[P.pos_n[kx] * es + row];
            }
        }
        __syncthreads();
    }
}

// One candidate: gather its box from the superset, mask and phase it, x inverse transform.
// MR0 MR1 MR2: the radix plan of M fixed at compile time (then 16 rows per block, logr = 4), or MR0 = 0 for
// the runtime plan.
template <int MR0, int MR1, int MR2>
__global__ void __launch_bounds__(kSThreads, MR0 == 0 ? 2 : 4) k_xinv_sel(const __grid_constant__ Plan P, const __grid_constant__ Superset S,
                                                           const float2* __restrict__ xs, float2* __restrict__ g,
                                                           int count, int qoff0, int qoff1, int poff0, int poff1, int logr,
                                                           long long xs_len, long long g_len) {
    extern __shared__ float2 smem[];   // [M][R + 1] tile, then the phase and mask tables
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int R = 1 << logr, es = R + 1, M = P.m;
    const int pol = blockIdx.y, q0 = blockIdx.x * R;
    const int qoff = pol ? qoff1 : qoff0, poff = pol ? poff1 : poff0;
    const PolDev& pd = P.pol[pol];
    float2* phx = smem + (size_t)M * es;         // [M] beam-centre phase along x
    float2* phy = phx + M;                       // [R] along y, this block's box rows
    int* mlo = reinterpret_cast<int*>(phy + R);  // [R] kept column range of this block's box rows
    int* mhi = mlo + R;
    for (int i = tid; i < M; i += nthr) phx[i] = pd.phase_x[i];
    for (int i = tid; i < R; i += nthr) {
        const bool in = q0 + i < M;
        phy[i] = in ? pd.phase_y[q0 + i] : make_float2(0.f, 0.f);
        mlo[i] = in ? pd.mask_lo[q0 + i] : 1;
        mhi[i] = in ? pd.mask_hi[q0 + i] : 0;
    }
    __syncthreads();
    for (int fb = blockIdx.z; fb < count; fb += gridDim.z) {
        const float2* src = xs + (size_t)(fb * P.pols + pol) * S.ms * S.msx;
        // eight independent loads in flight per thread before their shared-memory stores
        for (int i0 = tid; i0 < R * M; i0 += 8 * nthr) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                const int row = idx / M, p = idx - row * M;
                const int q = q0 + row;
                v[u] = make_float2(0.f, 0.f);
                if (idx < R * M && q < M && p >= mlo[row] && p <= mhi[row] &&
                    DH_IN(P.status, (long long)(fb * P.pols + pol) * S.ms * S.msx + (long long)(qoff + q) * S.msx + poff + p, xs_len,
                          kSiteScore))
                    v[u] = src[(size_t)(qoff + q) * S.msx + poff + p];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = i0 + u * nthr;
                if (idx < R * M) {
                    const int row = idx / M, p = idx - row * M;
                    const int q = q0 + row;
                    float2 w = make_float2(0.f, 0.f);
                    if (q < M && p >= mlo[row] && p <= mhi[row]) w = cmul(cmul(v[u], phx[p]), phy[row]);
                    smem[plan_pos<MR0, MR1, MR2>(P.pos_m, p) * es + row] = w;
                }
            }
        }
        __syncthreads();
        if constexpr (MR0 == 0)
            fft_run<true>(smem, M, P.rad_m, P.nrad_m, logr, es, P.tw_inv_m, tid, nthr);
        else
            ifft_static<MR0, MR1, MR2, 16, 17, kSThreads>(smem, P.tw_inv_m, tid);
        float2* dst = g + (size_t)(fb * P.pols + pol) * M * M;
        for (int idx = tid; idx < R * M; idx += nthr) {
            const int row = idx / M, i = idx - row * M;
            const int q = q0 + row;
            if (q < M && DH_IN(P.status, (long long)(fb * P.pols + pol) * M * M + (long long)q * M + i, g_len, kSiteScore))
                dst[(size_t)q * M + i] = smem[i * es + row];
        }
        __syncthreads();
    }
}

cudaError_t score_init() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_xfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024))) return e;
    if ((e = cudaFuncSetAttribute(k_xinv_sel<0, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024))) return e;
    return cudaFuncSetAttribute(k_xinv_sel<16, 11, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace dhk

using namespace dh;

namespace {

int ilog2i(int v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

}  // namespace

extern "C" int dh_score_settings(dh_handle h, const void* d_frames, int dtype, int batch, const dh_setting* settings,
                                 int count, float* d_power, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    if (!d_frames || !settings || !d_power) return fail(DH_ERROR_NULLPOINTER, "null pointer");
    if (count < 1) return fail(DH_ERROR_INVALIDARGUMENT, "candidate count must be >= 1");
    if (dtype != DH_DTYPE_U16 && dtype != DH_DTYPE_F32) return fail(DH_ERROR_INVALIDARGUMENT, "bad dtype");
    if (batch < 1) batch = 1;
    int rc = ensure_plan(H);
    if (rc) return rc;
    if (H->plan.modes == 0) return fail(DH_ERROR_INVALIDARGUMENT, "scoring needs a basis (group count > 0)");
    if (H->plan.ny != H->plan.n || H->plan.my != H->plan.m)
        return fail(DH_ERROR_INVALIDDIMENSION, "candidate scoring needs a square window and field");
    static bool score_ready[64] = {false};
    if (H->device >= 0 && H->device < 64 && !score_ready[H->device]) {
        cudaError_t e = dhk::score_init();
        if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
        score_ready[H->device] = true;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // candidate plans: geometry and tables of every candidate, validated before any work is queued, uploaded into
    // the handle's candidate area with one copy; the call returns once its work is done, so the next call may
    // overwrite the area
    std::vector<dhk::Plan> plans;
    std::vector<Geometry> geos(count);
    std::vector<Tables> tabs(count);
    auto cleanup = [&]() { cudaStreamSynchronize(st); };
    for (int s = 0; s < count; ++s) {
        std::string why;
        rc = build_geometry_candidate(H->s, settings[s], &geos[s], &why);
        if (rc) return fail(rc, "candidate " + std::to_string(s) + ": " + why);
    }
    build_tables_many(H->s, geos, &tabs, H->s.precision == DH_PRECISION_SPLIT_BF16);
    rc = upload_plans(H, geos, tabs, &plans);
    if (rc) return rc;
    const dhk::Plan& P0 = H->plan;
    const int N = P0.n, M = P0.m, pols = P0.pols;
    const int per_frame = pols * P0.modes;
    // superset box over all candidates, per polarisation
    dhk::Superset S{};
    int kly_min[DH_MAX_POLS] = {0, 0};
    int ms = M, msx = M;
    for (int p = 0; p < pols; ++p) {
        int ylo = geos[0].pol[p].ax[1].klo, yhi = ylo, xlo = geos[0].pol[p].ax[0].klo, xhi = xlo;
        for (const Geometry& g : geos) {
            ylo = std::min(ylo, g.pol[p].ax[1].klo);
            yhi = std::max(yhi, g.pol[p].ax[1].klo);
            xlo = std::min(xlo, g.pol[p].ax[0].klo);
            xhi = std::max(xhi, g.pol[p].ax[0].klo);
        }
        kly_min[p] = ylo;
        S.klx[p] = xlo;
        ms = std::max(ms, M + (yhi - ylo));
        msx = std::max(msx, M + (xhi - xlo));
    }
    // an even column count: every superset row then starts on the same 16-byte phase, as the scoring
    // contraction's bulk copies need (the extra column is one more DFT bin, never read)
    msx += msx & 1;
    S.ms = ms;
    S.msx = msx;
    const bool superset = ms <= N && msx <= N;
    dhk::StageTimer* tm = H->timer();
    if (!superset) {
        // one candidate at a time through the full generic path, coefficients for the whole batch
        const size_t per_frame_scratch = split_window_bytes(P0) * pols;
        const int chunk = chunk_frames(per_frame_scratch, pols, batch, H->device);
        const size_t spectra_bytes = (per_frame_scratch * chunk + 255) & ~(size_t)255;
        rc = ensure_scratch(H, spectra_bytes + (size_t)batch * per_frame * sizeof(float2));
        if (rc) {
            cleanup();
            return rc;
        }
        float2* coefs = (float2*)((char*)H->d_scratch + spectra_bytes);   // [batch][pols * modes]
        for (int s = 0; s < count && rc == DH_SUCCESS; ++s) {
            rc = run_split(plans[s], H->d_scratch, per_frame_scratch * chunk, d_frames, dtype, batch, nullptr, nullptr,
                           coefs, st, tm);
            if (rc) break;
            if (tm) tm->start(st);
            dhk::k_power<<<(batch + 7) / 8, 256, 0, st>>>(coefs, per_frame, 0, batch, 1, s, batch, d_power, count);
            if (tm) tm->stop(st, "k_power");
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_fail(e, "power");
        }
        cleanup();
        return rc;
    }
    // per frame: the superset spectra plus every candidate's coefficients
    const size_t per_frame_scratch = ((size_t)ms * N + (size_t)ms * msx + (size_t)M * M) * sizeof(float2) * pols;
    const size_t per_frame_coefs = (size_t)count * per_frame * sizeof(float2);
    const int chunk = chunk_frames(per_frame_scratch + per_frame_coefs, pols, batch, H->device);
    // superset rows, superset spectra and candidate x-inverse rows, each region starting on a 256-byte boundary
    const size_t r1s_bytes = ((size_t)chunk * pols * ms * N * sizeof(float2) + 255) & ~(size_t)255;
    // 256 bytes of slack: a box row copied with 16 bytes of alignment slack may end 8 bytes past the spectra
    const size_t xs_bytes = ((size_t)chunk * pols * ms * msx * sizeof(float2) + 256 + 255) & ~(size_t)255;
    const size_t spectra_bytes = (r1s_bytes + xs_bytes + (size_t)chunk * pols * M * M * sizeof(float2) + 255) & ~(size_t)255;
    rc = ensure_scratch(H, spectra_bytes + per_frame_coefs * chunk);
    if (rc) {
        cleanup();
        return rc;
    }
    float2* coefs = (float2*)((char*)H->d_scratch + spectra_bytes);   // [count][chunk][pols * modes]
    auto power = [&](int f0, int n) -> int {
        const int warps = n * count, per_block = 8;
        if (tm) tm->start(st);
        dhk::k_power<<<(warps + per_block - 1) / per_block, 32 * per_block, 0, st>>>(coefs, per_frame, f0, n, count, 0,
                                                                                  chunk, d_power, count);
        if (tm) tm->stop(st, "k_power");
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? DH_SUCCESS : cuda_fail(e, "power");
    };
    float2* r1s = (float2*)H->d_scratch;
    float2* xs = (float2*)((char*)H->d_scratch + r1s_bytes);
    float2* gbuf = (float2*)((char*)H->d_scratch + r1s_bytes + xs_bytes);
    dhk::Plan Psup = P0;                 // the y pass extracts the superset rows
    Psup.m = ms;
    Psup.my = ms;
    for (int p = 0; p < pols; ++p) Psup.pol[p].kly = kly_min[p];
    const int logr = (N >= 512) ? 4 : 5;
    const int R = 1 << logr;
    for (int f0 = 0; f0 < batch && rc == DH_SUCCESS; f0 += chunk) {
        const int n = std::min(chunk, batch - f0);
        const int zf = std::min(n, 65535);
        dhk::Batch B{};
        B.src = d_frames;
        B.dtype = dtype;
        B.frame0 = f0;
        B.count = n;
        B.r1 = r1s;
        B.r1_len = (long long)(r1s_bytes / sizeof(float2));
        cudaError_t e = dhk::launch_ypass(Psup, B, st, tm);
        if (e == cudaSuccess) {
            dim3 gx((ms + R - 1) / R, pols, zf);
            if (tm) tm->start(st);
            dhk::k_xfwd<<<gx, dhk::kSThreads, (size_t)N * (R + 1) * sizeof(float2), st>>>(P0, S, r1s, xs, n, logr, ilog2i(N),
                (long long)(r1s_bytes / sizeof(float2)), (long long)(xs_bytes / sizeof(float2)));
            if (tm) tm->stop(st, "k_xfwd");
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "superset transform");
            break;
        }
        for (int s = 0; s < count && rc == DH_SUCCESS; ++s) {
            const dhk::Plan& Pc = plans[s];
            int qo[2] = {0, 0}, po[2] = {0, 0};
            for (int p = 0; p < pols; ++p) {
                qo[p] = Pc.pol[p].kly - kly_min[p];
                po[p] = Pc.pol[p].klx - S.klx[p];
            }
            dhk::Batch Bc{};
            Bc.src = d_frames;
            Bc.dtype = dtype;
            Bc.frame0 = f0;
            Bc.count = n;
            Bc.g = gbuf;
            Bc.g_len = (long long)chunk * pols * M * M;
            // the last kernel writes frame f at (f * pols + pol) * modes: shift so frame f0 lands at slot 0
            Bc.coefs = coefs + (size_t)s * chunk * per_frame - (size_t)f0 * per_frame;
            cudaError_t e = cudaSuccess;
            const dhk::BoxSrc box{xs, ms, msx, {qo[0], qo[1]}, {po[0], po[1]}, (long long)(xs_bytes / sizeof(float2))};
            if (dhk::score_tc_supported(Pc, Bc, box)) {
                // split-BF16: one contraction straight from the candidate's box in the superset spectra
                if (tm) tm->start(st);
                e = dhk::launch_score_tc(Pc, Bc, box, st);
                if (tm) tm->stop(st, "k_score_tc");
            } else {
                dim3 gi((M + R - 1) / R, pols, zf);
                if (tm) tm->start(st);
                // the large configuration's field size (176 = 16 11) runs with its inverse plan fixed at compile time
                if (M == 176 && R == 16 && Pc.nrad_m == 2 && Pc.rad_m[0] == 16 && Pc.rad_m[1] == 11)
                    dhk::k_xinv_sel<16, 11, 1><<<gi, dhk::kSThreads, ((size_t)M * (R + 1) + M + 2 * R) * sizeof(float2), st>>>(
                        Pc, S, xs, gbuf, n, qo[0], qo[1], po[0], po[1], logr, (long long)(xs_bytes / sizeof(float2)),
                        (long long)chunk * pols * M * M);
                else
                    dhk::k_xinv_sel<0, 0, 0><<<gi, dhk::kSThreads, ((size_t)M * (R + 1) + M + 2 * R) * sizeof(float2), st>>>(
                        Pc, S, xs, gbuf, n, qo[0], qo[1], po[0], po[1], logr, (long long)(xs_bytes / sizeof(float2)),
                        (long long)chunk * pols * M * M);
                if (tm) tm->stop(st, "k_xinv_sel");
                e = cudaGetLastError();
                if (e == cudaSuccess) e = dhk::launch_last(Pc, Bc, st, tm);
            }
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "candidate");
                break;
            }
        }
        if (rc == DH_SUCCESS) rc = power(f0, n);
    }
    cleanup();
    return rc;
}
