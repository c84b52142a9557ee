// Host-buffer entry point: the paper's processing call takes frames in host memory (digHoloSetBatch /
// digHoloSetBatchUint16 with a host pointer, then digHoloProcessBatch) and returns fields and coefficients in
// host memory.  dh_process_batch_host does the same on the GPU with the copies hidden behind the kernels:
// the batch is cut into chunks that cycle over kSlots streams, each with its own device staging buffers, so
// the host-to-device copy of one chunk, the reconstruction of the previous one and the device-to-host copy of
// the one before that run at the same time (the two copy directions use separate copy engines).  Only the frame
// rows that hold the polarisation windows are copied (one strided copy per chunk), and the kernels run with a
// copy of the plan whose frame height and window rows are those of the cropped frames.  The asynchronous entry
// returns once everything is queued, so that the next batch's uploads start behind this one's downloads: each
// internal stream keeps its own staging slot from call to call, and a call whose slot layout differs from the
// last one first waits for the streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "runtime.hpp"

namespace dh {

namespace {

constexpr int kSlots = 4;
constexpr size_t kAlign = 256;
constexpr size_t kSlotCap = 256ull << 20;   // device bytes per slot
constexpr int kMinChunk = 32;                // frames
constexpr int kChunksTarget = 4;             // chunks per batch when the batch is large enough

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

}  // namespace

struct HostPipe {
    int device = -1;
    cudaStream_t st[kSlots] = {};
    cudaEvent_t start = nullptr;
    cudaEvent_t done[kSlots] = {};
    unsigned char* buf = nullptr;
    size_t bytes = 0;
    size_t slot = 0;                  // staging bytes per stream of the last call (its layout)
};

void release_pipe(Handle* H) {
    HostPipe* p = H->pipe;
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (p->device >= 0 && p->device != cur) cudaSetDevice(p->device);
    for (int s = 0; s < kSlots; ++s) {
        if (p->st[s]) cudaStreamSynchronize(p->st[s]);
    }
    if (p->buf) cudaFree(p->buf);
    for (int s = 0; s < kSlots; ++s) {
        if (p->st[s]) cudaStreamDestroy(p->st[s]);
        if (p->done[s]) cudaEventDestroy(p->done[s]);
    }
    if (p->start) cudaEventDestroy(p->start);
    if (p->device >= 0 && p->device != cur && cur >= 0) cudaSetDevice(cur);
    delete p;
    H->pipe = nullptr;
}

static int ensure_pipe(Handle* H, size_t bytes) {
    if (H->pipe && H->pipe->device != H->device) release_pipe(H);
    if (!H->pipe) {
        HostPipe* p = new HostPipe();
        p->device = H->device;
        H->pipe = p;
        cudaError_t e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
        for (int s = 0; s < kSlots && e == cudaSuccess; ++s) {
            e = cudaStreamCreateWithFlags(&p->st[s], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            release_pipe(H);
            return cuda_fail(e, "host pipeline streams");
        }
    }
    HostPipe* p = H->pipe;
    if (p->bytes >= bytes) return DH_SUCCESS;
    for (int s = 0; s < kSlots; ++s) cudaStreamSynchronize(p->st[s]);
    if (p->buf) cudaFree(p->buf);
    p->buf = nullptr;
    p->bytes = 0;
    cudaError_t e = cudaMalloc(&p->buf, bytes);
    if (e != cudaSuccess) {
        p->buf = nullptr;
        return fail(DH_ERROR_MEMORYALLOCATION, std::string("host pipeline buffers: ") + cudaGetErrorString(e));
    }
    p->bytes = bytes;
    return DH_SUCCESS;
}

static int process_host(Handle* H, const void* h_frames, int dtype, int batch, void* h_fields, void* h_coefs,
                        cudaStream_t caller, bool wait) {
    if (!h_frames) return fail(DH_ERROR_NULLPOINTER, "frames pointer is null");
    if (dtype != DH_DTYPE_U16 && dtype != DH_DTYPE_F32)
        return fail(DH_ERROR_INVALIDARGUMENT, "dtype must be DH_DTYPE_U16 or DH_DTYPE_F32");
    if (batch < 1) batch = 1;
    int rc = ensure_plan(H);
    if (rc) return rc;
    const dhk::Plan& P = H->plan;
    if (P.modes == 0) h_coefs = nullptr;
    const size_t esz = dtype == DH_DTYPE_U16 ? 2 : 4;
    int row0 = 0, rows = 0;
    window_rows(P, &row0, &rows);
    dhk::Plan Pc = P;                      // the plan of the cropped frames
    Pc.height = rows;
    for (int p = 0; p < P.pols; ++p) Pc.pol[p].oy -= row0;
    const size_t full = (size_t)P.width * P.height * esz;
    const size_t frame = (size_t)P.width * rows * esz;
    const size_t field = h_fields ? (size_t)P.pols * P.my * P.m * sizeof(float2) : 0;
    const size_t coef = h_coefs ? (size_t)P.pols * P.modes_out * sizeof(float2) : 0;
    // staged frames start 256-byte aligned, so the row pitch alone decides whether the fused path applies
    const bool fused = fused_allowed(H, P) && fused_layout_ok(P, dtype);
    const size_t scratch = (fused ? 0 : split_window_bytes(P) * P.pols) + (coef ? basis_scratch_bytes(P) : 0);
    const size_t per_frame = frame + field + coef + scratch;
    if (align_up(frame) + align_up(field) + align_up(coef) + align_up(scratch) > kSlotCap)
        return fail(DH_ERROR_MEMORYALLOCATION, "one frame of this geometry exceeds the host pipeline's slot size");
    int chunk = std::max(kMinChunk, (batch + kChunksTarget - 1) / kChunksTarget);
    chunk = (int)std::min<size_t>((size_t)chunk, std::max<size_t>(1, kSlotCap / per_frame));
    chunk = std::min(chunk, batch);
    size_t b_frames, b_fields, b_coefs, b_scratch, slot;
    for (;; --chunk) {
        b_frames = align_up(chunk * frame);
        b_fields = align_up(chunk * field);
        b_coefs = align_up(chunk * coef);
        b_scratch = align_up(chunk * scratch);
        slot = b_frames + b_fields + b_coefs + b_scratch;
        if (slot <= kSlotCap || chunk == 1) break;
    }
    const int slots = std::min(kSlots, (batch + chunk - 1) / chunk);
    rc = ensure_pipe(H, slot * slots);
    if (rc) return rc;
    HostPipe* p = H->pipe;
    if (p->slot != slot) {
        // stream s stages its chunks at s * slot: with another slot size the regions of different streams would
        // overlap the work of earlier calls still in flight
        for (int s = 0; s < kSlots; ++s) cudaStreamSynchronize(p->st[s]);
        p->slot = slot;
    }
    // order the pipeline after the work already queued on the caller's stream
    cudaError_t e = cudaEventRecord(p->start, caller);
    for (int s = 0; s < slots && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(p->st[s], p->start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "host pipeline ordering");
    for (int k = 0, f0 = 0; f0 < batch && rc == DH_SUCCESS; ++k, f0 += chunk) {
        const int s = k % slots;
        const int n = std::min(chunk, batch - f0);
        cudaStream_t st = p->st[s];
        unsigned char* base = p->buf + (size_t)s * slot;
        unsigned char* d_frames = base;
        unsigned char* d_fields = field ? base + b_frames : nullptr;
        unsigned char* d_coefs = coef ? base + b_frames + b_fields : nullptr;
        unsigned char* d_scratch = scratch ? base + b_frames + b_fields + b_coefs : nullptr;
        // rows [row0, row0 + rows) of each of the chunk's frames, packed
        e = cudaMemcpy2DAsync(d_frames, frame, (const unsigned char*)h_frames + (size_t)f0 * full + (size_t)row0 * P.width * esz,
                              full, frame, n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "frames upload");
            break;
        }
        rc = process_plan(H, Pc, d_frames, dtype, n, d_fields, d_coefs, d_scratch, b_scratch, st);
        if (rc) break;
        if (d_fields) {
            e = cudaMemcpyAsync((unsigned char*)h_fields + (size_t)f0 * field, d_fields, (size_t)n * field,
                                cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "fields download");
        }
        if (d_coefs && rc == DH_SUCCESS) {
            e = cudaMemcpyAsync((unsigned char*)h_coefs + (size_t)f0 * coef, d_coefs, (size_t)n * coef,
                                cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "coefficients download");
        }
    }
    // the asynchronous entry leaves the completion to dh_process_batch_host_wait (a wait of the caller's stream
    // would order the next call's first upload after this call's last download)
    if (!wait) return rc;
    // the caller's stream waits for the pipeline; the call returns when the results are in host memory
    for (int s = 0; s < slots; ++s) {
        cudaEventRecord(p->done[s], p->st[s]);
        cudaStreamWaitEvent(caller, p->done[s], 0);
    }
    for (int s = 0; s < slots; ++s) {
        e = cudaStreamSynchronize(p->st[s]);
        if (e != cudaSuccess && rc == DH_SUCCESS) rc = cuda_fail(e, "host pipeline");
    }
    return rc;
}

}  // namespace dh

using namespace dh;

extern "C" int dh_process_batch_host(dh_handle h, const void* h_frames, int dtype, int batch, void* h_fields,
                                     void* h_coefs, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    return process_host(H, h_frames, dtype, batch, h_fields, h_coefs, (cudaStream_t)stream, true);
}

extern "C" int dh_process_batch_host_async(dh_handle h, const void* h_frames, int dtype, int batch, void* h_fields,
                                           void* h_coefs, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    return process_host(H, h_frames, dtype, batch, h_fields, h_coefs, (cudaStream_t)stream, false);
}

extern "C" int dh_process_batch_host_wait(dh_handle h) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    HostPipe* p = H->pipe;
    if (!p) return DH_SUCCESS;
    int rc = DH_SUCCESS;
    for (int s = 0; s < kSlots; ++s) {
        const cudaError_t e = p->st[s] ? cudaStreamSynchronize(p->st[s]) : cudaSuccess;
        if (e != cudaSuccess && rc == DH_SUCCESS) rc = cuda_fail(e, "host pipeline");
    }
    return rc;
}
