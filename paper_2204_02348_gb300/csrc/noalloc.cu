// dh_process_batch_noalloc: the generic reconstruction path without any device allocation.
//
// Callers that own all device memory themselves (a framework's caching allocator, a serving process that has
// already divided a fixed HBM budget) or that run an acquisition loop which must not stall cannot let a library
// call cudaMalloc / cudaFree: those calls synchronise the device and can fail in the middle of a run.  This
// entry point serves them.  It runs the same three kernels as dh_process_batch, but both its plan tables and
// its scratch live in one array of static device memory defined below, so nothing is allocated per call.
//
// The array is 16 MiB: 1 MiB for the plan tables (uploaded by each call with a stream-ordered copy) and
// 15 MiB of scratch (the per-frame spectra between the kernels; the batch is processed in chunks that fit).
// The overlap is always the FP32 one (the split-BF16 tables are not packed), so the handle's precision
// setting does not apply here.  Every GPU that loads the library holds the array until the process exits.
// All calls share it and it keeps the last call's contents; nothing in it has to start at zero, because every
// table entry and every scratch element is written before it is read within the same call (the status block at
// the start of the table area is part of each call's table upload, so it starts every call at zero).  Calls that
// overlap on the GPU (queued on different streams, or from different threads without ordering) race on the
// array: serialise them on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.hpp"

namespace {
constexpr size_t kNoallocBytes = 16ull << 20;
constexpr size_t kNoallocTableBytes = 1ull << 20;
constexpr size_t kNoallocScratchBytes = kNoallocBytes - kNoallocTableBytes;
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_area[kNoallocBytes];

namespace dh {
namespace {

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device, looked up once per device (with that device
// current) and cached; also sets the kernels' shared-memory attribute for that device.
int noalloc_area(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(DH_ERROR_INVALIDARGUMENT, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_area);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        e = dhk::split_init();
        if (e == cudaSuccess) e = dhk::basis_init();
        if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
        g_noalloc_addr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_addr[dev];
    return DH_SUCCESS;
}

struct Packer {
    std::vector<unsigned char> bytes;
    size_t put(const void* p, size_t n) {
        const size_t off = (bytes.size() + 255) & ~(size_t)255;
        bytes.resize(off + (n ? n : 1));
        if (n) std::memcpy(bytes.data() + off, p, n);
        return off;
    }
};

std::vector<int> digit_reversed_positions(int len, const std::vector<int>& rad) {
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

// Host image of the plan tables plus the kernel plan pointing into the device copy at `dev_tables`.
int pack_plan(const Settings& s, const Geometry& g, const Tables& t, unsigned char* dev_tables, Packer* pk,
              dhk::Plan* out) {
    if ((int)t.radix_n.size() > dhk::kMaxRadices || (int)t.radix_m.size() > dhk::kMaxRadices ||
        (int)t.radix_ny.size() > dhk::kMaxRadices || (int)t.radix_my.size() > dhk::kMaxRadices)
        return fail(DH_ERROR_INVALIDDIMENSION, "too many radix passes");
    // the status block first (offset 0 of the table area): zero in every call's upload, so it reports the last call
    const int zero_status[4] = {0, 0, 0, 0};
    const size_t o_st = pk->put(zero_status, sizeof zero_status);
    const size_t o_twn = pk->put(t.tw_fwd_n.data(), t.tw_fwd_n.size() * 4);
    const size_t o_twm = pk->put(t.tw_inv_m.data(), t.tw_inv_m.size() * 4);
    const std::vector<int> pn = digit_reversed_positions(g.n, t.radix_n);
    const std::vector<int> pm = digit_reversed_positions(g.m, t.radix_m);
    const size_t o_pn = pk->put(pn.data(), pn.size() * 4);
    const size_t o_pm = pk->put(pm.data(), pm.size() * 4);
    // the y axis' transforms: the x ones for square geometries, their own tables otherwise
    size_t o_twny = o_twn, o_twmy = o_twm, o_pny = o_pn, o_pmy = o_pm;
    if (!g.square()) {
        o_twny = pk->put(t.tw_fwd_ny.data(), t.tw_fwd_ny.size() * 4);
        o_twmy = pk->put(t.tw_inv_my.data(), t.tw_inv_my.size() * 4);
        const std::vector<int> pny = digit_reversed_positions(g.ny, t.radix_ny);
        const std::vector<int> pmy = digit_reversed_positions(g.my, t.radix_my);
        o_pny = pk->put(pny.data(), pny.size() * 4);
        o_pmy = pk->put(pmy.data(), pmy.size() * 4);
    }
    const size_t o_mm = pk->put(t.mode_m.data(), t.mode_m.size() * 4);
    const size_t o_mn = pk->put(t.mode_n.data(), t.mode_n.size() * 4);
    const size_t o_bt = pk->put(t.basis_tt.data(), t.basis_tt.size() * 4);
    dhk::Plan& P = *out;
    std::memset(&P, 0, sizeof P);
    P.n = g.n;
    P.m = g.m;
    P.groups = g.groups;
    P.modes = g.modes;
    P.pols = g.pols;
    P.width = s.width;
    P.height = s.height;
    // The static table area holds no tensor-core B operand, so this path always runs the FP32 overlap,
    // whatever precision the handle asks for; a split-BF16 plan here would have no B tiles to read.
    P.precision = DH_PRECISION_FP32;
    P.nrad_n = (int)t.radix_n.size();
    P.nrad_m = (int)t.radix_m.size();
    for (int i = 0; i < P.nrad_n; ++i) P.rad_n[i] = t.radix_n[i];
    for (int i = 0; i < P.nrad_m; ++i) P.rad_m[i] = t.radix_m[i];
    P.tw_fwd_n = (const float2*)(dev_tables + o_twn);
    P.tw_inv_m = (const float2*)(dev_tables + o_twm);
    P.pos_n = (const int*)(dev_tables + o_pn);
    P.pos_m = (const int*)(dev_tables + o_pm);
    P.ny = g.ny;
    P.my = g.my;
    P.nrad_ny = (int)t.radix_ny.size();
    P.nrad_my = (int)t.radix_my.size();
    for (int i = 0; i < P.nrad_ny; ++i) P.rad_ny[i] = t.radix_ny[i];
    for (int i = 0; i < P.nrad_my; ++i) P.rad_my[i] = t.radix_my[i];
    P.tw_fwd_ny = (const float2*)(dev_tables + o_twny);
    P.tw_inv_my = (const float2*)(dev_tables + o_twmy);
    P.pos_ny = (const int*)(dev_tables + o_pny);
    P.pos_my = (const int*)(dev_tables + o_pmy);
    P.mode_m = (const int*)(dev_tables + o_mm);
    P.mode_n = (const int*)(dev_tables + o_mn);
    P.modes_out = g.modes_out;
    P.basis_tt = t.basis_tt.empty() ? nullptr : (const float2*)(dev_tables + o_bt);
    P.status = (int*)(dev_tables + o_st);
    for (int p = 0; p < g.pols; ++p) {
        const PolTables& pt = t.pol[p];
        dhk::PolDev& pd = P.pol[p];
        pd.ox = g.pol[p].ax[0].origin;
        pd.oy = g.pol[p].ax[1].origin;
        pd.klx = g.pol[p].ax[0].klo;
        pd.kly = g.pol[p].ax[1].klo;
        pd.mask_lo = (const int*)(dev_tables + pk->put(pt.mask_lo.data(), pt.mask_lo.size() * 4));
        pd.mask_hi = (const int*)(dev_tables + pk->put(pt.mask_hi.data(), pt.mask_hi.size() * 4));
        pd.phase_x = (const float2*)(dev_tables + pk->put(pt.phase_x.data(), pt.phase_x.size() * 4));
        pd.phase_y = (const float2*)(dev_tables + pk->put(pt.phase_y.data(), pt.phase_y.size() * 4));
        pd.corr_x = (const float2*)(dev_tables + pk->put(pt.corr_x.data(), pt.corr_x.size() * 4));
        pd.corr_y = (const float2*)(dev_tables + pk->put(pt.corr_y.data(), pt.corr_y.size() * 4));
        pd.hg_x = (const float*)(dev_tables + pk->put(pt.hg_x.data(), pt.hg_x.size() * 4));
        pd.hg_y = (const float*)(dev_tables + pk->put(pt.hg_y.data(), pt.hg_y.size() * 4));
        const size_t o_cal = pk->put(pt.cal.data(), pt.cal.size() * 4);
        pd.cal = pt.cal.empty() ? nullptr : (const float*)(dev_tables + o_cal);
    }
    if (pk->bytes.size() > kNoallocTableBytes)
        return fail(DH_ERROR_INVALIDDIMENSION, "plan tables of this geometry exceed the 1 MiB static table area");
    return DH_SUCCESS;
}

}  // namespace

int* noalloc_status_block(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    return reinterpret_cast<int*>(g_noalloc_addr[dev]);   // offset 0 of the table area, once the array is set up
}

}  // namespace dh

using namespace dh;

extern "C" int dh_process_batch_noalloc(dh_handle h, const void* d_frames, int dtype, int batch, void* d_fields,
                                        void* d_coefs, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    if (!d_frames) return fail(DH_ERROR_NULLPOINTER, "frames pointer is null");
    if (dtype != DH_DTYPE_U16 && dtype != DH_DTYPE_F32)
        return fail(DH_ERROR_INVALIDARGUMENT, "dtype must be DH_DTYPE_U16 or DH_DTYPE_F32");
    if (batch < 1) batch = 1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* area = nullptr;
    int rc = noalloc_area(dev, &area);
    if (rc) return rc;
    Geometry g;
    std::string why;
    rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    Tables t;
    build_tables(H->s, g, &t);
    Packer pk;
    dhk::Plan P;
    rc = pack_plan(H->s, g, t, area, &pk, &P);
    if (rc) return rc;
    if (P.modes == 0) d_coefs = nullptr;
    const size_t hg_frame = d_coefs ? basis_scratch_bytes(P) : 0;
    const size_t per_frame = split_window_bytes(P) * P.pols + hg_frame;
    if (per_frame > kNoallocScratchBytes) {
        return fail(DH_ERROR_INVALIDDIMENSION, "one frame of this geometry needs " + std::to_string(per_frame) +
                                                   " bytes of scratch; the static scratch holds " +
                                                   std::to_string(kNoallocScratchBytes));
    }
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemcpyAsync(area, pk.bytes.data(), pk.bytes.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "plan table upload");
    unsigned char* scratch = area + kNoallocTableBytes;
    if (!hg_frame)
        return run_split(P, scratch, kNoallocScratchBytes, d_frames, dtype, batch, nullptr, d_fields, d_coefs, st,
                         nullptr);
    // output-basis transform: chunks whose HG coefficients sit at the end of the static scratch
    const int chunk = (int)std::min<size_t>((size_t)batch, kNoallocScratchBytes / per_frame);
    const size_t frame_bytes = (size_t)P.width * P.height * (dtype == DH_DTYPE_U16 ? 2 : 4);
    const size_t field_bytes = (size_t)P.pols * P.my * P.m * sizeof(float2);
    const size_t coef_bytes = (size_t)P.pols * P.modes_out * sizeof(float2);
    float2* hg = (float2*)(scratch + kNoallocScratchBytes - (size_t)chunk * hg_frame);
    for (int f0 = 0; f0 < batch; f0 += chunk) {
        const int n = std::min(chunk, batch - f0);
        rc = run_split(P, scratch, kNoallocScratchBytes - (size_t)chunk * hg_frame,
                       (const unsigned char*)d_frames + f0 * frame_bytes, dtype, n, nullptr,
                       d_fields ? (unsigned char*)d_fields + f0 * field_bytes : nullptr, hg, st, nullptr);
        if (rc) return rc;
        e = dhk::launch_basis(P, hg, (float2*)((unsigned char*)d_coefs + f0 * coef_bytes), n * P.pols, st, nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "basis transform launch");
    }
    return DH_SUCCESS;
}
