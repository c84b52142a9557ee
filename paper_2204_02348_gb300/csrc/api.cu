// extern "C" entry points declared in include/digholo.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/digholo.h"
#include "kernels.cuh"
#include "plan.hpp"
#include "runtime.hpp"

namespace dh {

static thread_local std::string g_err = "no error";

int fail(int code, const std::string& why) {
    g_err = why;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    std::string s = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(DH_ERROR_CUDA, s);
}

// ------------------------------------------------------------------------------------------- handles

static std::mutex g_handles_mu;
static std::vector<std::unique_ptr<Handle>> g_handles;

Handle* get_handle(dh_handle h) {
    std::lock_guard<std::mutex> lk(g_handles_mu);
    if (h < 0 || h >= (int)g_handles.size() || !g_handles[h]) return nullptr;
    return g_handles[h].get();
}

static void release_device(Handle* H) {
    release_pipe(H);
    if (H->d_blob || H->d_scratch || H->d_hg || H->d_cand) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (H->device >= 0 && H->device != cur) cudaSetDevice(H->device);
        if (H->d_blob) cudaFree(H->d_blob);
        if (H->d_scratch) cudaFree(H->d_scratch);
        if (H->d_hg) cudaFree(H->d_hg);
        if (H->d_cand) cudaFree(H->d_cand);
        if (H->device >= 0 && H->device != cur && cur >= 0) cudaSetDevice(cur);
    }
    H->d_blob = nullptr;
    H->d_scratch = nullptr;
    H->scratch_bytes = 0;
    H->d_hg = nullptr;
    H->hg_bytes = 0;
    H->d_cand = nullptr;
    H->cand_bytes = 0;
    H->device = -1;
}

// ------------------------------------------------------------------------------------------- plan upload

struct Blob {
    std::vector<unsigned char> bytes;
    size_t put(const void* p, size_t n) {
        size_t off = (bytes.size() + 255) & ~(size_t)255;
        bytes.resize(off + std::max(n, (size_t)1));
        if (n) std::memcpy(bytes.data() + off, p, n);
        return off;
    }
};

static std::vector<int> pos_table(int len, const std::vector<int>& rad) {
    // position of frequency k after DIF passes with these radices (first pass first)
    std::vector<int> pos(len);
    for (int k = 0; k < len; ++k) {
        int p = 0, s = len, rem = k;
        for (int r : rad) {
            s /= r;
            p += (rem % r) * s;
            rem /= r;
        }
        pos[k] = p;
    }
    return pos;
}

// The host image of a plan's device tables, with each table's offset in it.
struct PlanImage {
    Blob b;
    size_t o_twn = 0, o_twm = 0, o_pn = 0, o_pm = 0, o_mm = 0, o_mn = 0, o_st = 0, o_bt = 0;
    size_t o_twny = 0, o_twmy = 0, o_pny = 0, o_pmy = 0;
    size_t o_pol[DH_MAX_POLS][13] = {};
};

static int build_plan_image(const Geometry& g, const Tables& t, PlanImage* im) {
    if ((int)t.radix_n.size() > dhk::kMaxRadices || (int)t.radix_m.size() > dhk::kMaxRadices ||
        (int)t.radix_ny.size() > dhk::kMaxRadices || (int)t.radix_my.size() > dhk::kMaxRadices)
        return fail(DH_ERROR_INVALIDDIMENSION, "too many radix passes");
    Blob& b = im->b;
    im->o_twn = b.put(t.tw_fwd_n.data(), t.tw_fwd_n.size() * 4);
    im->o_twm = b.put(t.tw_inv_m.data(), t.tw_inv_m.size() * 4);
    std::vector<int> pn = pos_table(g.n, t.radix_n), pm = pos_table(g.m, t.radix_m);
    im->o_pn = b.put(pn.data(), pn.size() * 4);
    im->o_pm = b.put(pm.data(), pm.size() * 4);
    if (g.square()) {
        im->o_twny = im->o_twn;
        im->o_twmy = im->o_twm;
        im->o_pny = im->o_pn;
        im->o_pmy = im->o_pm;
    } else {
        im->o_twny = b.put(t.tw_fwd_ny.data(), t.tw_fwd_ny.size() * 4);
        im->o_twmy = b.put(t.tw_inv_my.data(), t.tw_inv_my.size() * 4);
        std::vector<int> pny = pos_table(g.ny, t.radix_ny), pmy = pos_table(g.my, t.radix_my);
        im->o_pny = b.put(pny.data(), pny.size() * 4);
        im->o_pmy = b.put(pmy.data(), pmy.size() * 4);
    }
    im->o_mm = b.put(t.mode_m.data(), t.mode_m.size() * 4);
    im->o_mn = b.put(t.mode_n.data(), t.mode_n.size() * 4);
    const int zero_status[4] = {0, 0, 0, 0};
    im->o_st = b.put(zero_status, sizeof zero_status);
    im->o_bt = b.put(t.basis_tt.data(), t.basis_tt.size() * 4);
    for (int p = 0; p < g.pols; ++p) {
        const PolTables& pt = t.pol[p];
        im->o_pol[p][0] = b.put(pt.mask_lo.data(), pt.mask_lo.size() * 4);
        im->o_pol[p][1] = b.put(pt.mask_hi.data(), pt.mask_hi.size() * 4);
        im->o_pol[p][2] = b.put(pt.phase_x.data(), pt.phase_x.size() * 4);
        im->o_pol[p][3] = b.put(pt.phase_y.data(), pt.phase_y.size() * 4);
        im->o_pol[p][4] = b.put(pt.corr_x.data(), pt.corr_x.size() * 4);
        im->o_pol[p][5] = b.put(pt.corr_y.data(), pt.corr_y.size() * 4);
        im->o_pol[p][6] = b.put(pt.hg_x.data(), pt.hg_x.size() * 4);
        im->o_pol[p][7] = b.put(pt.hg_y.data(), pt.hg_y.size() * 4);
        im->o_pol[p][8] = b.put(pt.hgy_tc.data(), pt.hgy_tc.size() * 2);
        im->o_pol[p][9] = b.put(pt.cal.data(), pt.cal.size() * 4);
        im->o_pol[p][10] = b.put(pt.pr.data(), pt.pr.size());
        im->o_pol[p][11] = b.put(pt.coef_tc.data(), pt.coef_tc.size());
        im->o_pol[p][12] = b.put(pt.score_tc.data(), pt.score_tc.size());
    }
    return DH_SUCCESS;
}

// The kernel plan of an image uploaded at device address `base`.
static void plan_from_image(const Settings& s, const Geometry& g, const Tables& t, const PlanImage& im,
                            unsigned char* base, dhk::Plan* out) {
    dhk::Plan& P = *out;
    std::memset(&P, 0, sizeof P);
    P.n = g.n;
    P.m = g.m;
    P.groups = g.groups;
    P.modes = g.modes;
    P.pols = g.pols;
    P.width = s.width;
    P.height = s.height;
    P.precision = s.precision;
    P.tc_np = tc_rows(g.groups);
    P.nrad_n = (int)t.radix_n.size();
    P.nrad_m = (int)t.radix_m.size();
    for (int i = 0; i < P.nrad_n; ++i) P.rad_n[i] = t.radix_n[i];
    for (int i = 0; i < P.nrad_m; ++i) P.rad_m[i] = t.radix_m[i];
    P.tw_fwd_n = (const float2*)(base + im.o_twn);
    P.tw_inv_m = (const float2*)(base + im.o_twm);
    P.pos_n = (const int*)(base + im.o_pn);
    P.pos_m = (const int*)(base + im.o_pm);
    P.ny = g.ny;
    P.my = g.my;
    P.nrad_ny = (int)t.radix_ny.size();
    P.nrad_my = (int)t.radix_my.size();
    for (int i = 0; i < P.nrad_ny; ++i) P.rad_ny[i] = t.radix_ny[i];
    for (int i = 0; i < P.nrad_my; ++i) P.rad_my[i] = t.radix_my[i];
    P.tw_fwd_ny = (const float2*)(base + im.o_twny);
    P.tw_inv_my = (const float2*)(base + im.o_twmy);
    P.pos_ny = (const int*)(base + im.o_pny);
    P.pos_my = (const int*)(base + im.o_pmy);
    P.mode_m = (const int*)(base + im.o_mm);
    P.mode_n = (const int*)(base + im.o_mn);
    P.status = (int*)(base + im.o_st);
    P.modes_out = g.modes_out;
    P.basis_tt = t.basis_tt.empty() ? nullptr : (const float2*)(base + im.o_bt);
    for (int p = 0; p < g.pols; ++p) {
        dhk::PolDev& pd = P.pol[p];
        pd.ox = g.pol[p].ax[0].origin;
        pd.oy = g.pol[p].ax[1].origin;
        pd.klx = g.pol[p].ax[0].klo;
        pd.kly = g.pol[p].ax[1].klo;
        pd.mask_lo = (const int*)(base + im.o_pol[p][0]);
        pd.mask_hi = (const int*)(base + im.o_pol[p][1]);
        pd.phase_x = (const float2*)(base + im.o_pol[p][2]);
        pd.phase_y = (const float2*)(base + im.o_pol[p][3]);
        pd.corr_x = (const float2*)(base + im.o_pol[p][4]);
        pd.corr_y = (const float2*)(base + im.o_pol[p][5]);
        pd.hg_x = (const float*)(base + im.o_pol[p][6]);
        pd.hg_y = (const float*)(base + im.o_pol[p][7]);
        pd.hgy_tc = t.pol[p].hgy_tc.empty() ? nullptr : (const uint16_t*)(base + im.o_pol[p][8]);
        pd.cal = t.pol[p].cal.empty() ? nullptr : (const float*)(base + im.o_pol[p][9]);
        pd.pr = t.pol[p].pr.empty() ? nullptr : base + im.o_pol[p][10];
        pd.coef_tc = t.pol[p].coef_tc.empty() ? nullptr : base + im.o_pol[p][11];
        pd.score_tc = t.pol[p].score_tc.empty() ? nullptr : base + im.o_pol[p][12];
    }
    P.coef_np = 0;
    bool coef_all = g.pols > 0;
    for (int p = 0; p < g.pols; ++p) coef_all = coef_all && !t.pol[p].coef_tc.empty();
    if (coef_all) P.coef_np = t.pol[0].coef_np;
}

int upload_plan(const Settings& s, const Geometry& g, const Tables& t, void** out_blob, dhk::Plan* out) {
    PlanImage im;
    int rc = build_plan_image(g, t, &im);
    if (rc) return rc;
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, im.b.bytes.size());
    if (e != cudaSuccess) return fail(DH_ERROR_MEMORYALLOCATION, std::string("plan tables: ") + cudaGetErrorString(e));
    e = cudaMemcpy(d, im.b.bytes.data(), im.b.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "plan upload");
    }
    plan_from_image(s, g, t, im, (unsigned char*)d, out);
    *out_blob = d;
    return DH_SUCCESS;
}

int upload_plans(Handle* H, const std::vector<Geometry>& geos, const std::vector<Tables>& tabs,
                 std::vector<dhk::Plan>* plans) {
    const size_t n = geos.size();
    std::vector<PlanImage> ims(n);
    std::vector<size_t> at(n);
    size_t total = 0;
    for (size_t i = 0; i < n; ++i) {
        int rc = build_plan_image(geos[i], tabs[i], &ims[i]);
        if (rc) return rc;
        at[i] = total;
        total = (total + ims[i].b.bytes.size() + 255) & ~(size_t)255;
    }
    if (total > H->cand_bytes) {
        if (H->d_cand) cudaFree(H->d_cand);
        H->d_cand = nullptr;
        H->cand_bytes = 0;
        cudaError_t e = cudaMalloc(&H->d_cand, total);
        if (e != cudaSuccess) {
            H->d_cand = nullptr;
            return fail(DH_ERROR_MEMORYALLOCATION, std::string("candidate plan tables: ") + cudaGetErrorString(e));
        }
        H->cand_bytes = total;
    }
    std::vector<unsigned char> all(total, 0);
    for (size_t i = 0; i < n; ++i) std::memcpy(all.data() + at[i], ims[i].b.bytes.data(), ims[i].b.bytes.size());
    cudaError_t e = cudaMemcpy(H->d_cand, all.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "candidate plan upload");
    plans->resize(n);
    for (size_t i = 0; i < n; ++i) {
        plan_from_image(H->s, geos[i], tabs[i], ims[i], (unsigned char*)H->d_cand + at[i], &(*plans)[i]);
        // candidates report waits and guards through the handle's own status block
        if (H->plan.status) (*plans)[i].status = H->plan.status;
    }
    return DH_SUCCESS;
}

int init_device_once(int dev) {
    static std::mutex mu;
    static bool inited[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && inited[dev]) return DH_SUCCESS;
    cudaError_t e = dhk::split_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = dhk::tc_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = dhk::coef_tc_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = fused_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = fused_pr_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = fused_g_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = fused256_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    e = dhk::basis_init();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    if (dev >= 0 && dev < 64) inited[dev] = true;
    return DH_SUCCESS;
}

int ensure_plan(Handle* H) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (!H->dirty && H->device == dev && H->d_blob) return DH_SUCCESS;
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    tune_refresh(H, g);
    Tables t;
    build_tables(H->s, g, &t);
    rc = init_device_once(dev);
    if (rc) return rc;
    if (H->device != dev) release_device(H);
    void* blob = nullptr;
    dhk::Plan P;
    rc = upload_plan(H->s, g, t, &blob, &P);
    if (rc) return rc;
    if (H->d_blob) cudaFree(H->d_blob);
    H->d_blob = blob;
    H->plan = P;
    H->device = dev;
    H->geo = g;
    H->tab = t;
    H->dirty = false;
    return DH_SUCCESS;
}

int ensure_scratch(Handle* H, size_t bytes) {
    if (H->scratch_bytes >= bytes) return DH_SUCCESS;
    if (H->d_scratch) cudaFree(H->d_scratch);
    H->d_scratch = nullptr;
    H->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&H->d_scratch, bytes);
    if (e != cudaSuccess) {
        H->d_scratch = nullptr;
        return fail(DH_ERROR_MEMORYALLOCATION, std::string("scratch: ") + cudaGetErrorString(e));
    }
    H->scratch_bytes = bytes;
    return DH_SUCCESS;
}

int chunk_frames(size_t per_frame_bytes, int pols, int batch, int device, size_t target) {
    static int sms[64] = {0};
    int n = 148;
    if (device >= 0 && device < 64) {
        if (!sms[device]) cudaDeviceGetAttribute(&sms[device], cudaDevAttrMultiProcessorCount, device);
        if (sms[device] > 0) n = sms[device];
    }
    const size_t per = std::max<size_t>(per_frame_bytes, 1);
    size_t frames = ((size_t)8 * n + pols - 1) / pols;
    frames = std::max(frames, target / per);
    frames = std::min(frames, std::max<size_t>(1, kScratchCap / per));
    return (int)std::max<size_t>(1, std::min<size_t>(frames, (size_t)batch));
}

size_t split_window_bytes(const dhk::Plan& P) { return ((size_t)P.my * P.n + (size_t)P.my * P.m) * sizeof(float2); }

// ------------------------------------------------------------------------------------------- profiler

cudaEvent_t Profiler::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Profiler::start(cudaStream_t s) {
    open = take();
    cudaEventRecord(open, s);
}

void Profiler::stop(cudaStream_t s, const char* kernel) {
    cudaEvent_t b = take();
    cudaEventRecord(b, s);
    pending.push_back(Rec{kernel, open, b});
    open = nullptr;
}

int Profiler::resolve() {
    for (Rec& r : pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "profile events");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        size_t i = 0;
        while (i < names.size() && names[i] != r.name) ++i;
        if (i == names.size()) {
            names.push_back(r.name);
            launches.push_back(0);
            total_ms.push_back(0.0);
        }
        launches[i] += 1;
        total_ms[i] += ms;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
    return DH_SUCCESS;
}

void Profiler::reset() {
    resolve();
    names.clear();
    launches.clear();
    total_ms.clear();
}

Profiler::~Profiler() {
    for (Rec& r : pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

size_t basis_scratch_bytes(const dhk::Plan& P) {
    return P.basis_tt ? (size_t)P.pols * P.modes * sizeof(float2) : 0;
}

// The output-basis transform after the HG overlap: the path writes HG coefficients to `hg`, k_basis writes
// the caller's coefficients.
static int finish_basis(const dhk::Plan& P, void* hg, void* coefs, int batch, cudaStream_t st,
                        dhk::StageTimer* timer) {
    cudaError_t e = dhk::launch_basis(P, (const float2*)hg, (float2*)coefs, batch * P.pols, st, timer);
    return e == cudaSuccess ? DH_SUCCESS : cuda_fail(e, "basis transform launch");
}

// Point *coefs at the handle's HG-coefficient scratch when an output-basis transform follows; returns the
// caller's buffer in *out.
static int basis_target(Handle* H, int batch, void** coefs, void** out) {
    const dhk::Plan& P = H->plan;
    *out = *coefs;
    if (!*coefs || !P.basis_tt) return DH_SUCCESS;
    const size_t need = basis_scratch_bytes(P) * batch;
    if (H->hg_bytes < need) {
        if (H->d_hg) cudaFree(H->d_hg);
        H->d_hg = nullptr;
        H->hg_bytes = 0;
        cudaError_t e = cudaMalloc(&H->d_hg, need);
        if (e != cudaSuccess) {
            H->d_hg = nullptr;
            return fail(DH_ERROR_MEMORYALLOCATION, std::string("basis scratch: ") + cudaGetErrorString(e));
        }
        H->hg_bytes = need;
    }
    *coefs = H->d_hg;
    return DH_SUCCESS;
}

int process(Handle* H, const void* frames, int dtype, int batch, void* window, void* fields, void* coefs,
            cudaStream_t st) {
    if (!frames) return fail(DH_ERROR_NULLPOINTER, "frames pointer is null");
    if (dtype != DH_DTYPE_U16 && dtype != DH_DTYPE_F32) return fail(DH_ERROR_INVALIDARGUMENT, "dtype must be DH_DTYPE_U16 or DH_DTYPE_F32");
    if (batch < 1) batch = 1;
    int rc = ensure_plan(H);
    if (rc) return rc;
    const dhk::Plan& P = H->plan;
    if (P.modes == 0) coefs = nullptr;
    void* out = nullptr;
    rc = basis_target(H, batch, &coefs, &out);
    if (rc) return rc;
    if (fused_allowed(H, P) && !window && fused_frames_ok(P, frames, dtype)) {
        rc = launch_fused_path(H, P, frames, dtype, batch, fields, coefs, st, H->timer());
    } else {
        const size_t per_frame = split_window_bytes(P) * P.pols;
        const int chunk = chunk_frames(per_frame, P.pols, batch, H->device,
                                       H->chunk_mb > 0 ? (size_t)H->chunk_mb << 20 : kScratchTarget);
        rc = ensure_scratch(H, per_frame * chunk);
        if (rc) return rc;
        rc = run_split(P, H->d_scratch, H->scratch_bytes, frames, dtype, batch, window, fields, coefs, st, H->timer());
    }
    if (rc || out == coefs) return rc;
    return finish_basis(P, coefs, out, batch, st, H->timer());
}

// Batch averaging on the generic path: per chunk of averaging groups, the forward kernels fill the
// x-inverse-transformed windows of every member, k_avg_dot / k_avg_sum form the phase-aligned means, and the
// last kernel transforms and decomposes one window per group.
int process_avg(Handle* H, const void* frames, int dtype, int batch, int avg, int mode, void* fields, void* coefs,
                cudaStream_t st) {
    if (!frames) return fail(DH_ERROR_NULLPOINTER, "frames pointer is null");
    if (dtype != DH_DTYPE_U16 && dtype != DH_DTYPE_F32) return fail(DH_ERROR_INVALIDARGUMENT, "dtype must be DH_DTYPE_U16 or DH_DTYPE_F32");
    if (mode != DH_AVGMODE_SEQUENTIAL && mode != DH_AVGMODE_INTERLACED && mode != DH_AVGMODE_SEQUENTIALSWEEP)
        return fail(DH_ERROR_INVALIDARGUMENT, "avg_mode must be DH_AVGMODE_SEQUENTIAL, _INTERLACED or _SEQUENTIALSWEEP");
    if (avg > DH_MAX_AVG_COUNT) return fail(DH_ERROR_INVALIDDIMENSION, "avg_count exceeds DH_MAX_AVG_COUNT");
    if (batch < 1) batch = 1;
    if (avg <= 1) return process(H, frames, dtype, batch, nullptr, fields, coefs, st);
    int rc = ensure_plan(H);
    if (rc) return rc;
    const dhk::Plan& P = H->plan;
    if (P.modes == 0) coefs = nullptr;
    void* out = nullptr;
    rc = basis_target(H, batch, &coefs, &out);
    if (rc) return rc;
    const long long elems = (long long)P.pols * P.my * P.m;
    const int slices = dhk::avg_slices(elems);
    // 128 x 128 windows: the fused kernel's forward-only mode writes each member's window and its inverse-only
    // mode reconstructs the group means (no r1 scratch); otherwise the generic forward kernels
    const bool fused = fused_allowed(H, P) && use_fused(P) && fused_frames_ok(P, frames, dtype);
    // per member frame: its window (fused) or the generic path's r1 and window
    const size_t member = fused ? (size_t)elems * sizeof(float2) : split_window_bytes(P) * P.pols;
    const size_t per_group = (size_t)avg * member + (size_t)elems * sizeof(float2) + (size_t)avg * slices * sizeof(float2);
    // groups per chunk: enough member windows for several waves of the forward kernels, about the L2-sized
    // scratch target, at most the scratch cap and the grid limit
    int dev_sms = 148;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, H->device);
    size_t groups = std::max<size_t>(((size_t)8 * dev_sms + (size_t)avg * P.pols - 1) / ((size_t)avg * P.pols),
                                     kScratchTarget / per_group);
    groups = std::min(groups, std::max<size_t>(1, kScratchCap / per_group));
    groups = std::min<size_t>(std::min<size_t>(groups, (size_t)batch), 65535);
    const int chunk = (int)std::max<size_t>(1, groups);
    rc = ensure_scratch(H, per_group * chunk);
    if (rc) return rc;
    // scratch: [r1 of every member (generic path only)] [member windows] [group means] [inner-product partials]
    float2* r1 = (float2*)H->d_scratch;
    float2* gbuf = fused ? r1 : r1 + (size_t)chunk * avg * P.pols * P.my * P.n;
    float2* mean = gbuf + (size_t)chunk * avg * elems;
    float2* part = mean + (size_t)chunk * elems;
    if ((size_t)((part + (size_t)chunk * avg * slices) - r1) * sizeof(float2) > H->scratch_bytes)
        return fail(DH_ERROR_ERROR, "averaging scratch layout exceeds the reservation");
    dhk::StageTimer* tm = H->timer();
    for (int g0 = 0; g0 < batch; g0 += chunk) {
        const int n = std::min(chunk, batch - g0);
        dhk::Batch B{};
        B.src = frames;
        B.dtype = dtype;
        B.r1 = r1;
        B.r1_len = fused ? 0 : (long long)chunk * avg * P.pols * P.my * P.n;
        long long mstride, gstride;
        cudaError_t e = cudaSuccess;
        const int total = batch * avg;
        if (mode == DH_AVGMODE_INTERLACED) {
            // member j of groups [g0, g0 + n) is the contiguous frame range [j batch + g0, j batch + g0 + n)
            for (int j = 0; j < avg && e == cudaSuccess; ++j) {
                if (fused) {
                    rc = launch_fused(H, P, frames, dtype, total, j * batch + g0, n, dhk::kModeForward, nullptr,
                                      gbuf + (size_t)j * n * elems, nullptr, nullptr, st, tm);
                    if (rc) return rc;
                } else {
                    B.frame0 = j * batch + g0;
                    B.count = n;
                    B.g = gbuf + (size_t)j * n * elems;
                    B.g_len = (long long)chunk * avg * elems - (long long)j * n * elems;
                    e = dhk::launch_forward(P, B, st, tm);
                }
            }
            mstride = (long long)n * elems;
            gstride = elems;
        } else {
            if (fused) {
                rc = launch_fused(H, P, frames, dtype, total, g0 * avg, n * avg, dhk::kModeForward, nullptr, gbuf,
                                  nullptr, nullptr, st, tm);
                if (rc) return rc;
            } else {
                B.frame0 = g0 * avg;
                B.count = n * avg;
                B.g = gbuf;
                B.g_len = (long long)chunk * avg * elems;
                e = dhk::launch_forward(P, B, st, tm);
            }
            mstride = elems;
            gstride = (long long)avg * elems;
        }
        const dhk::AvgExtents X{P.status, (long long)chunk * avg * elems, (long long)chunk * avg * slices,
                                (long long)chunk * elems};
        if (e == cudaSuccess) e = dhk::launch_avg(gbuf, part, mean, n, avg, elems, mstride, gstride, X, st, tm);
        if (e == cudaSuccess && fused) {
            rc = launch_fused(H, P, nullptr, dtype, 0, g0, n, dhk::kModeInverse, mean, nullptr, fields, coefs, st, tm);
            if (rc) return rc;
            continue;
        }
        if (e == cudaSuccess) {
            dhk::Batch L{};
            L.src = frames;
            L.dtype = dtype;
            L.frame0 = g0;
            L.count = n;
            L.g = mean;
            L.g_len = (long long)chunk * elems;
            L.fields = (float2*)fields;
            L.coefs = (float2*)coefs;
            e = dhk::launch_last(P, L, st, tm);
        }
        if (e != cudaSuccess) return cuda_fail(e, "averaging launch");
    }
    if (out == coefs) return DH_SUCCESS;
    return finish_basis(P, coefs, out, batch, st, tm);
}

int process_with(Handle* H, const void* frames, int dtype, int batch, void* fields, void* coefs, void* scratch,
                 size_t scratch_bytes, cudaStream_t st) {
    return process_plan(H, H->plan, frames, dtype, batch, fields, coefs, scratch, scratch_bytes, st);
}

int process_plan(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                 void* scratch, size_t scratch_bytes, cudaStream_t st) {
    if (P.modes == 0) coefs = nullptr;
    void* out = coefs;
    if (coefs && P.basis_tt) {
        // the HG coefficients take the end of the scratch
        const size_t need = basis_scratch_bytes(P) * batch;
        if (scratch_bytes < need) return fail(DH_ERROR_MEMORYALLOCATION, "scratch smaller than the basis transform needs");
        scratch_bytes -= need;
        coefs = (unsigned char*)scratch + scratch_bytes;
    }
    int rc;
    if (fused_allowed(H, P) && fused_frames_ok(P, frames, dtype))
        rc = launch_fused_path(H, P, frames, dtype, batch, fields, coefs, st, nullptr);
    else
        rc = run_split(P, scratch, scratch_bytes, frames, dtype, batch, nullptr, fields, coefs, st, nullptr);
    if (rc || out == coefs) return rc;
    return finish_basis(P, coefs, out, batch, st, nullptr);
}

void window_rows(const dhk::Plan& P, int* row0, int* rows) {
    int lo = P.height, hi = 0;
    for (int p = 0; p < P.pols; ++p) {
        lo = std::min(lo, P.pol[p].oy);
        hi = std::max(hi, P.pol[p].oy + P.ny);   // the window is N_y rows high
    }
    *row0 = lo;
    *rows = hi - lo;
}

int run_split(const dhk::Plan& P, void* scratch, size_t scratch_bytes, const void* frames, int dtype, int batch,
              void* window, void* fields, void* coefs, cudaStream_t st, dhk::StageTimer* timer) {
    const size_t per_frame = split_window_bytes(P) * P.pols;
    const int chunk = (int)std::min<size_t>((size_t)batch, scratch_bytes / per_frame);
    if (chunk < 1) return fail(DH_ERROR_MEMORYALLOCATION, "scratch smaller than one frame");
    float2* r1 = (float2*)scratch;
    float2* g = r1 + (size_t)chunk * P.pols * P.my * P.n;
    for (int f0 = 0; f0 < batch; f0 += chunk) {
        dhk::Batch B;
        B.src = frames;
        B.dtype = dtype;
        B.frame0 = f0;
        B.count = std::min(chunk, batch - f0);
        B.r1 = r1;
        B.g = g;
        B.r1_len = (long long)chunk * P.pols * P.my * P.n;
        B.g_len = (long long)chunk * P.pols * P.my * P.m;
        B.window = (float2*)window;
        B.fields = (float2*)fields;
        B.coefs = (float2*)coefs;
        cudaError_t e = dhk::launch_split(P, B, st, timer);
        if (e != cudaSuccess) return cuda_fail(e, "launch");
    }
    return DH_SUCCESS;
}

}  // namespace dh

using namespace dh;

#define GET_HANDLE(h)                                                     \
    Handle* H = get_handle(h);                                            \
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");      \
    std::lock_guard<std::mutex> lk(H->mu)

extern "C" {

const char* dh_last_error(void) { return g_err.c_str(); }

int dh_create(dh_handle* out) {
    if (!out) return fail(DH_ERROR_NULLPOINTER, "out is null");
    std::lock_guard<std::mutex> lk(g_handles_mu);
    g_handles.emplace_back(new Handle());
    *out = (dh_handle)(g_handles.size() - 1);
    return DH_SUCCESS;
}

int dh_destroy(dh_handle h) {
    std::unique_ptr<Handle> owned;
    {
        std::lock_guard<std::mutex> lk(g_handles_mu);
        if (h < 0 || h >= (int)g_handles.size() || !g_handles[h]) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
        owned = std::move(g_handles[h]);
    }
    std::lock_guard<std::mutex> lk(owned->mu);
    if (owned->d_blob || owned->d_scratch || owned->d_hg) cudaDeviceSynchronize();
    release_device(owned.get());
    return DH_SUCCESS;
}

int dh_set_frame(dh_handle h, int width, int height, int pol_count, double pixel_size) {
    GET_HANDLE(h);
    if (width <= 0 || height <= 0) return fail(DH_ERROR_INVALIDDIMENSION, "frame width and height must be positive");
    if (pol_count < 1 || pol_count > DH_MAX_POLS) return fail(DH_ERROR_INVALIDPOLARISATION, "polarisation count must be 1 or 2");
    if (!(pixel_size > 0.0) || !std::isfinite(pixel_size)) return fail(DH_ERROR_INVALIDARGUMENT, "pixel size must be positive");
    H->s.width = width;
    H->s.height = height;
    H->s.pols = pol_count;
    H->s.pixel = pixel_size;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_wavelength(dh_handle h, double wavelength) {
    GET_HANDLE(h);
    if (!(wavelength > 0.0) || !std::isfinite(wavelength)) return fail(DH_ERROR_INVALIDARGUMENT, "wavelength must be positive");
    H->s.wavelength = wavelength;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_fft_window(dh_handle h, int nx, int ny, int* set_nx, int* set_ny) {
    GET_HANDLE(h);
    const int fx = (nx / 16) * 16, fy = (ny / 16) * 16;
    if (fx <= 0 || fy <= 0) return fail(DH_ERROR_INVALIDDIMENSION, "window size must be at least 16");
    if (fx > DH_MAX_WINDOW || (fx & (fx - 1)) || fy > DH_MAX_WINDOW || (fy & (fy - 1)))
        return fail(DH_ERROR_INVALIDDIMENSION, "window sizes must be powers of two up to 1024");
    H->s.n = fx;
    H->s.ny = fy;
    H->dirty = true;
    if (set_nx) *set_nx = fx;
    if (set_ny) *set_ny = fy;
    return DH_SUCCESS;
}

int dh_set_beam_centre(dh_handle h, int axis, int pol, double centre) {
    GET_HANDLE(h);
    if (axis < 0 || axis > 1) return fail(DH_ERROR_INVALIDAXIS, "axis must be 0 (x) or 1 (y)");
    if (pol < 0 || pol >= DH_MAX_POLS) return fail(DH_ERROR_INVALIDPOLARISATION, "polarisation must be 0 or 1");
    if (!std::isfinite(centre)) return fail(DH_ERROR_INVALIDARGUMENT, "beam centre must be finite");
    H->s.centre[pol][axis] = centre;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_fourier_window_radius(dh_handle h, double radius_deg) {
    GET_HANDLE(h);
    if (!(radius_deg > 0.0) || !std::isfinite(radius_deg)) return fail(DH_ERROR_INVALIDARGUMENT, "window radius must be positive");
    H->s.radius_deg = radius_deg;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_ifft_size(dh_handle h, int mx, int my) {
    GET_HANDLE(h);
    for (int v : {mx, my})
        if (v < 0 || (v > 0 && (v % 16 || v > DH_MAX_FIELD || radix_plan(v).empty())))
            return fail(DH_ERROR_INVALIDDIMENSION,
                        "field sizes must be 0 or multiples of 16 up to 512 with a 19-smooth odd part");
    H->s.m_req = mx;
    H->s.my_req = my;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_tilt(dh_handle h, int axis, int pol, double tilt_deg) {
    GET_HANDLE(h);
    if (axis < 0 || axis > 1) return fail(DH_ERROR_INVALIDAXIS, "axis must be 0 (x) or 1 (y)");
    if (pol < 0 || pol >= DH_MAX_POLS) return fail(DH_ERROR_INVALIDPOLARISATION, "polarisation must be 0 or 1");
    if (!std::isfinite(tilt_deg)) return fail(DH_ERROR_INVALIDARGUMENT, "tilt must be finite");
    H->s.tilt_deg[pol][axis] = tilt_deg;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_defocus(dh_handle h, int pol, double dioptre) {
    GET_HANDLE(h);
    if (pol < 0 || pol >= DH_MAX_POLS) return fail(DH_ERROR_INVALIDPOLARISATION, "polarisation must be 0 or 1");
    if (!std::isfinite(dioptre)) return fail(DH_ERROR_INVALIDARGUMENT, "defocus must be finite");
    H->s.defocus[pol] = dioptre;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_basis(dh_handle h, int pol, double waist, int group_count) {
    GET_HANDLE(h);
    if (pol < 0 || pol >= DH_MAX_POLS) return fail(DH_ERROR_INVALIDPOLARISATION, "polarisation must be 0 or 1");
    if (group_count < 0 || group_count > DH_MAX_GROUPS) return fail(DH_ERROR_INVALIDDIMENSION, "group count must be in 0..32");
    if (!(waist > 0.0) || !std::isfinite(waist)) return fail(DH_ERROR_INVALIDDIMENSION, "waist must be positive");
    H->s.waist[pol] = waist;
    H->s.groups = group_count;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_fill_factor_correction(dh_handle h, int enabled) {
    GET_HANDLE(h);
    H->s.fill_factor = enabled != 0;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_precision(dh_handle h, int precision) {
    GET_HANDLE(h);
    if (precision != DH_PRECISION_FP32 && precision != DH_PRECISION_SPLIT_BF16)
        return fail(DH_ERROR_INVALIDARGUMENT, "precision must be DH_PRECISION_FP32 or DH_PRECISION_SPLIT_BF16");
    H->s.precision = precision;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_ref_calibration(dh_handle h, const uint16_t* cal, int wavelength_count, int width, int height) {
    GET_HANDLE(h);
    H->dirty = true;
    if (!cal || wavelength_count < 1 || width < 1 || height < 1) {
        H->s.cal_on = 0;   // as the guide specifies: an invalid calibration disables the calibration
        return fail(cal ? DH_ERROR_INVALIDARGUMENT : DH_ERROR_NULLPOINTER, "invalid reference calibration; calibration disabled");
    }
    const size_t px = (size_t)width * height;
    uint16_t top = 0;
    for (size_t i = 0; i < px * wavelength_count; ++i) top = std::max(top, cal[i]);
    if (top == 0) {
        H->s.cal_on = 0;
        return fail(DH_ERROR_INVALIDARGUMENT, "reference calibration is all zero; calibration disabled");
    }
    H->s.cal.assign(cal, cal + px);
    H->s.cal_w = width;
    H->s.cal_h = height;
    H->s.cal_max = (double)top;
    H->s.cal_on = 1;
    return DH_SUCCESS;
}

int dh_set_ref_calibration_enabled(dh_handle h, int enabled) {
    GET_HANDLE(h);
    if (enabled && H->s.cal.empty()) return fail(DH_ERROR_INVALIDARGUMENT, "no reference calibration has been set");
    H->s.cal_on = enabled != 0;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_basis_type(dh_handle h, int basis) {
    GET_HANDLE(h);
    if (basis != DH_BASIS_HG && basis != DH_BASIS_LG && basis != DH_BASIS_CUSTOM)
        return fail(DH_ERROR_INVALIDARGUMENT, "basis must be DH_BASIS_HG, DH_BASIS_LG or DH_BASIS_CUSTOM");
    H->s.basis = basis;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_basis_transform(dh_handle h, int modes_in, int modes_out, const void* transform) {
    GET_HANDLE(h);
    if (!transform) return fail(DH_ERROR_NULLPOINTER, "transform is null");
    if (modes_in < 1 || modes_out < 1 || (long long)modes_in * modes_out > (1ll << 24))
        return fail(DH_ERROR_INVALIDDIMENSION, "transform dimensions must be >= 1 with modes_in * modes_out <= 2^24");
    const float* t = (const float*)transform;
    H->s.custom.assign(t, t + (size_t)2 * modes_in * modes_out);
    H->s.custom_in = modes_in;
    H->s.custom_out = modes_out;
    H->s.basis = DH_BASIS_CUSTOM;
    H->dirty = true;
    return DH_SUCCESS;
}

int dh_set_variant(dh_handle h, int variant) {
    GET_HANDLE(h);
    if (variant < DH_VARIANT_AUTO || variant > DH_VARIANT_FUSED_GROUPS)
        return fail(DH_ERROR_INVALIDARGUMENT,
                    "variant must be one of DH_VARIANT_AUTO, _FUSED, _FUSED_PRUNED, _GENERIC, _FUSED_GROUPS");
    H->variant = variant;
    return DH_SUCCESS;
}

int dh_get_variant(dh_handle h, int* variant) {
    GET_HANDLE(h);
    if (!variant) return fail(DH_ERROR_NULLPOINTER, "variant is null");
    int rc = ensure_plan(H);
    if (rc) return rc;
    *variant = resolve_variant(H, H->plan, true);
    return DH_SUCCESS;
}

int dh_get_output_dims(dh_handle h, int* m, int* modes, double* dx) {
    GET_HANDLE(h);
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    if (m) *m = g.m;
    if (modes) *modes = g.modes_out;
    if (dx) *dx = g.dx;
    return DH_SUCCESS;
}

int dh_get_field_dims(dh_handle h, int* mx, int* my, double* dx, double* dy) {
    GET_HANDLE(h);
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    if (mx) *mx = g.m;
    if (my) *my = g.my;
    if (dx) *dx = g.dx;
    if (dy) *dy = g.dy;
    return DH_SUCCESS;
}

int dh_get_axes(dh_handle h, int pol, double* x, double* y) {
    GET_HANDLE(h);
    if (!x || !y) return fail(DH_ERROR_NULLPOINTER, "axis arrays are null");
    if (pol < 0 || pol >= H->s.pols) return fail(DH_ERROR_INVALIDPOLARISATION, "no such polarisation");
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    for (int i = 0; i < g.m; ++i) x[i] = (double)(i - g.m / 2) * g.dx;
    for (int j = 0; j < g.my; ++j) y[j] = (double)(j - g.my / 2) * g.dy;
    return DH_SUCCESS;
}

int dh_process_batch(dh_handle h, const void* d_frames, int dtype, int batch, void* d_fields, void* d_coefs,
                     void* stream) {
    GET_HANDLE(h);
    return process(H, d_frames, dtype, batch, nullptr, d_fields, d_coefs, (cudaStream_t)stream);
}

int dh_process_batch_window(dh_handle h, const void* d_frames, int dtype, int batch, void* d_window,
                            void* d_fields, void* d_coefs, void* stream) {
    GET_HANDLE(h);
    if (!d_window) return fail(DH_ERROR_NULLPOINTER, "window pointer is null");
    return process(H, d_frames, dtype, batch, d_window, d_fields, d_coefs, (cudaStream_t)stream);
}

int dh_process_batch_avg(dh_handle h, const void* d_frames, int dtype, int batch, int avg_count, int avg_mode,
                         void* d_fields, void* d_coefs, void* stream) {
    GET_HANDLE(h);
    return process_avg(H, d_frames, dtype, batch, avg_count, avg_mode, d_fields, d_coefs, (cudaStream_t)stream);
}

int dh_set_profiling(dh_handle h, int enable) {
    GET_HANDLE(h);
    H->prof.reset();
    H->prof.on = enable != 0;
    return DH_SUCCESS;
}

int dh_get_profile(dh_handle h, int max_kernels, char* names, long long* launches, double* total_ms, int* count) {
    GET_HANDLE(h);
    if (!count) return fail(DH_ERROR_NULLPOINTER, "count is null");
    int rc = H->prof.resolve();
    if (rc) return rc;
    const int n = (int)H->prof.names.size();
    *count = n;
    for (int i = 0; i < n && i < max_kernels; ++i) {
        if (names) {
            std::strncpy(names + 64 * i, H->prof.names[i].c_str(), 63);
            names[64 * i + 63] = 0;
        }
        if (launches) launches[i] = H->prof.launches[i];
        if (total_ms) total_ms[i] = H->prof.total_ms[i];
    }
    return DH_SUCCESS;
}

}  // extern "C"
