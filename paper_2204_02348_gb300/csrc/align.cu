// Fine-alignment search (user guide, digHoloAutoAlign: the "fine alignment tweaking stage"; goal: captured
// power, i.e. insertion loss).  A compass search over every polarisation's tilt (x, y), defocus and waist:
// each iteration scores the centre and the 8 P stencil points (one parameter moved by -step or +step, waist
// steps relative) in one dh_score_settings call, sums each candidate's power over the batch on the GPU
// (k_colsum, fixed order, FP64), moves to the best stencil point when it beats the centre (ties: lowest index)
// and otherwise halves every step.  The search is host orchestration around the GPU scoring path.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "runtime.hpp"

namespace dhk {
namespace {

constexpr int kSumThreads = 256;

// sums[s] = sum_b power[b][s] (power [batch][count] float), fixed order
__global__ void __launch_bounds__(kSumThreads) k_colsum(const float* __restrict__ power, int batch, int count,
                                                        double* __restrict__ sums) {
    __shared__ double red[kSumThreads];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < batch; b += kSumThreads) acc += (double)power[(size_t)b * count + s];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kSumThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[s] = red[0];
}

}  // namespace
}  // namespace dhk

namespace dh {

static void stencil(const dh_setting& c, int pols, const double st[3], std::vector<dh_setting>* out) {
    out->clear();
    out->push_back(c);
    for (int p = 0; p < pols; ++p)
        for (int par = 0; par < 4; ++par)
            for (int k = 0; k < 2; ++k) {
                const double sgn = k == 0 ? -1.0 : 1.0;
                dh_setting v = c;
                if (par < 2)
                    v.tilt_deg[p][par] += sgn * st[0];
                else if (par == 2)
                    v.defocus[p] += sgn * st[1];
                else
                    v.waist[p] *= 1.0 + sgn * st[2];
                out->push_back(v);
            }
}

}  // namespace dh

using namespace dh;

extern "C" int dh_get_alignment(dh_handle h, dh_setting* out) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    if (!out) return fail(DH_ERROR_NULLPOINTER, "out is null");
    std::lock_guard<std::mutex> lk(H->mu);
    for (int p = 0; p < DH_MAX_POLS; ++p) {
        out->tilt_deg[p][0] = H->s.tilt_deg[p][0];
        out->tilt_deg[p][1] = H->s.tilt_deg[p][1];
        out->defocus[p] = H->s.defocus[p];
        out->waist[p] = H->s.waist[p];
    }
    return DH_SUCCESS;
}

extern "C" int dh_auto_align(dh_handle h, const void* d_frames, int dtype, int batch, const double* steps,
                             const double* min_steps, int max_iter, double* power, int* iterations, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    if (!d_frames) return fail(DH_ERROR_NULLPOINTER, "frames pointer is null");
    if (batch < 1) batch = 1;
    const double def_steps[3] = {0.02, 0.1, 0.05}, def_min[3] = {2e-4, 1e-3, 5e-4};
    double st[3], lo[3];
    for (int i = 0; i < 3; ++i) {
        st[i] = steps ? steps[i] : def_steps[i];
        lo[i] = min_steps ? min_steps[i] : def_min[i];
        if (!(st[i] > 0.0) || !(lo[i] > 0.0)) return fail(DH_ERROR_INVALIDARGUMENT, "steps must be positive");
    }
    dh_setting cur{};
    int pols = 1, groups = 0;
    {
        std::lock_guard<std::mutex> lk(H->mu);
        pols = H->s.pols;
        groups = H->s.groups;
        for (int p = 0; p < DH_MAX_POLS; ++p) {
            cur.tilt_deg[p][0] = H->s.tilt_deg[p][0];
            cur.tilt_deg[p][1] = H->s.tilt_deg[p][1];
            cur.defocus[p] = H->s.defocus[p];
            cur.waist[p] = H->s.waist[p];
        }
    }
    if (groups < 1) return fail(DH_ERROR_INVALIDARGUMENT, "alignment needs a basis (group count > 0)");
    const int count = 1 + 8 * pols;
    cudaStream_t cs = (cudaStream_t)stream;
    float* d_power = nullptr;
    double* d_sums = nullptr;
    cudaError_t e = cudaMalloc(&d_power, (size_t)batch * count * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_sums, count * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(d_power);
        return fail(DH_ERROR_MEMORYALLOCATION, std::string("alignment scratch: ") + cudaGetErrorString(e));
    }
    std::vector<dh_setting> cand;
    std::vector<double> sums(count);
    double best = 0.0;
    int it = 0, rc = DH_SUCCESS;
    while (it < max_iter && (st[0] >= lo[0] || st[1] >= lo[1] || st[2] >= lo[2])) {
        stencil(cur, pols, st, &cand);
        rc = dh_score_settings(h, d_frames, dtype, batch, cand.data(), count, d_power, stream);
        if (rc) break;
        dhk::k_colsum<<<count, dhk::kSumThreads, 0, cs>>>(d_power, batch, count, d_sums);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(sums.data(), d_sums, count * sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "alignment power sums");
            break;
        }
        ++it;
        int k = 0;
        for (int s = 1; s < count; ++s)
            if (sums[s] > sums[k]) k = s;
        best = sums[0];
        if (sums[k] > sums[0]) {
            cur = cand[k];
            best = sums[k];
        } else {
            for (double& v : st) v *= 0.5;
        }
    }
    cudaFree(d_power);
    cudaFree(d_sums);
    if (rc) return rc;
    for (int p = 0; p < pols && rc == DH_SUCCESS; ++p) {
        rc = dh_set_tilt(h, 0, p, cur.tilt_deg[p][0]);
        if (!rc) rc = dh_set_tilt(h, 1, p, cur.tilt_deg[p][1]);
        if (!rc) rc = dh_set_defocus(h, p, cur.defocus[p]);
        if (!rc) rc = dh_set_basis(h, p, cur.waist[p], groups);
    }
    if (power) *power = best;
    if (iterations) *iterations = it;
    return rc;
}
