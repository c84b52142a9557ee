// Handle state and the host-side helpers shared by the entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "plan.hpp"

namespace dh {

// Frames per launch chunk of the generic path: enough windows for several waves of its one-block-per-window
// kernels (at least 8 per SM), at least what fits 48 MB (the chunk then stays in the 129 MB L2 between its
// kernels), and at most 1 GiB of scratch.
constexpr size_t kScratchTarget = 48ull << 20;
constexpr size_t kScratchCap = 1ull << 30;
int chunk_frames(size_t per_frame_bytes, int pols, int batch, int device, size_t target = kScratchTarget);

// Records a CUDA event pair around every kernel launch of a handle while enabled; totals per kernel name.
struct Profiler : dhk::StageTimer {
    bool on = false;
    struct Rec {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    cudaEvent_t open = nullptr;
    std::vector<std::string> names;
    std::vector<long long> launches;
    std::vector<double> total_ms;
    cudaEvent_t take();
    void start(cudaStream_t s) override;
    void stop(cudaStream_t s, const char* kernel) override;
    int resolve();   // wait for pending events, fold them into the totals
    void reset();
    ~Profiler() override;
};

// Kernel variants a handle can be held to (the values of DH_VARIANT_* in digholo.h).
constexpr int kVariantAuto = 0, kVariantFusedLegacy = 1, kVariantFusedPruned = 2, kVariantGeneric = 3,
              kVariantFusedGroups = 4;

struct HostPipe;   // streams and staging buffers of dh_process_batch_host (host.cu)

struct Handle {
    std::mutex mu;
    Settings s;
    bool dirty = true;
    int device = -1;
    Geometry geo{};
    Tables tab;
    void* d_blob = nullptr;       // plan tables (device)
    dhk::Plan plan{};
    void* d_scratch = nullptr;    // generic-path scratch (device)
    size_t scratch_bytes = 0;
    void* d_hg = nullptr;         // HG coefficients ahead of an output-basis transform (device)
    size_t hg_bytes = 0;
    void* d_cand = nullptr;       // plan tables of the candidates of a scoring call (device, reused by later calls)
    size_t cand_bytes = 0;
    HostPipe* pipe = nullptr;     // host-buffer pipeline, created on first use
    int variant = 0;              // kernel variant (DH_VARIANT_*): 0 lets the library (or its tuner) choose
    int tuned = 0;                // the tuner's variant for the current settings (0: none)
    int chunk_mb = 0;             // the tuner's generic-path scratch target per chunk, MiB (0: kScratchTarget)
    std::string tune_key;         // geometry key the tuning above belongs to
    bool tune_set = false;        // the tuning was set for tune_key (dh_set_tuning / dh_autotune), not looked up
    std::string tune_path;        // JSON cache file (dh_set_tuning_cache), empty when none
    std::map<std::string, dh_tuning> tune_cache;   // choices per geometry key
    Profiler prof;
    dhk::StageTimer* timer() { return prof.on ? &prof : nullptr; }
};

// Free the host-buffer pipeline of a handle (streams, events, device buffers).
void release_pipe(Handle* H);

// Tuner (tune.cpp): the geometry key of settings, and the tuning in effect for it: applied to the handle
// (variant, chunk target, radix plan in the settings) whenever the plan is rebuilt.
std::string tuning_key(const Settings& s, const Geometry& g);
void tune_refresh(Handle* H, const Geometry& g);

int fail(int code, const std::string& why);
int cuda_fail(cudaError_t e, const char* where);
Handle* get_handle(dh_handle h);
int ensure_plan(Handle* H);
int ensure_scratch(Handle* H, size_t bytes);
size_t split_window_bytes(const dhk::Plan& P);
// Upload the tables of a geometry to a fresh device blob and fill the kernel plan that points into it.
int upload_plan(const Settings& s, const Geometry& g, const Tables& t, void** out_blob, dhk::Plan* out);
// Upload the tables of several geometries (with the handle's settings) into the handle's candidate area, one
// copy for all, growing the area as needed, and fill their kernel plans.  The area is reused by the next call:
// the caller's work that reads it must be complete by then.
int upload_plans(Handle* H, const std::vector<Geometry>& geos, const std::vector<Tables>& tabs,
                 std::vector<dhk::Plan>* plans);
// Queue the generic three-kernel path for frames [0, batch) with the given plan and scratch.
int run_split(const dhk::Plan& P, void* scratch, size_t scratch_bytes, const void* frames, int dtype, int batch,
              void* window, void* fields, void* coefs, cudaStream_t st, dhk::StageTimer* timer);

// Fused single-kernel path for 128 x 128 windows (k_fused.cu).
bool use_fused(const dhk::Plan& P);
// Fused single-kernel path for 256 x 256 windows with 96 x 96 fields, uint16 frames, FP32 overlap (k_fused256.cu).
bool use_fused256(const dhk::Plan& P);
cudaError_t fused256_init();
int launch_fused256(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                    cudaStream_t st, dhk::StageTimer* timer);
// The variant a call runs (dh_set_variant's rules; `aligned`: the frames suit tensor copies).
int resolve_variant(const Handle* H, const dhk::Plan& P, bool aligned);
// use_fused, unless the handle's variant resolves to the generic path.
bool fused_allowed(const Handle* H, const dhk::Plan& P);
// The fused kernels stage windows with tensor copies: the frames need a 16-byte aligned base and row pitch (and,
// for the 256 x 256 kernel, uint16 pixels).  fused_layout_ok: the pitch and pixel rule alone (frames staged
// 256-byte aligned by the library itself).
bool fused_frames_ok(const dhk::Plan& P, const void* frames, int dtype);
bool fused_layout_ok(const dhk::Plan& P, int dtype);
// The variant rules and the fused paths' dispatch live in dispatch.cu.
cudaError_t fused_init();
int launch_fused_path(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields,
                      void* coefs, cudaStream_t st, dhk::StageTimer* timer);
// The fused kernel in one of its modes (0 whole path, 1 forward only: windows to win_out [count][pol][M][M],
// 2 inverse only: windows from win_in) over frames [frame0, frame0 + count) of an array of `total` frames;
// outputs and windows are indexed from frame0 (outputs) or 0 (windows).
int launch_fused(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int total, int frame0, int count,
                 int mode, const float2* win_in, float2* win_out, void* fields, void* coefs, cudaStream_t st,
                 dhk::StageTimer* timer);

// Column-pruned fused path (k_fused_pr.cu): 128 x 128 windows, 64 x 64 fields, FP32 overlap, whole path only;
// used by launch_fused_path when the plan carries its table block.
bool use_fused_pr(const dhk::Plan& P);
cudaError_t fused_pr_init();
int launch_fused_pr(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                    cudaStream_t st, dhk::StageTimer* timer);

// Status block of the allocation-free path on device dev (the start of its static array; nullptr until the first
// call on that device set the array up).
int* noalloc_status_block(int dev);

// Group-transform fused path (k_fused_g.cu): 128 x 128 windows, 64 x 64 fields, FP32 overlap, whole path only.
bool use_fused_g(const dhk::Plan& P);
cudaError_t fused_g_init();
int launch_fused_g(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                   cudaStream_t st, dhk::StageTimer* timer);

// HG coefficient bytes per frame that an output-basis transform needs as scratch (0 for the HG basis).
size_t basis_scratch_bytes(const dhk::Plan& P);

// Queue one batch with the handle's uploaded plan and caller-provided scratch (used by the serving loop,
// where concurrent requests of one handle must not share the handle's scratch).  With an output-basis
// transform the last batch * basis_scratch_bytes of the scratch hold the HG coefficients.  No profiling.
int process_with(Handle* H, const void* frames, int dtype, int batch, void* fields, void* coefs, void* scratch,
                 size_t scratch_bytes, cudaStream_t st);
// As process_with, with a copy of the handle's plan (the host pipeline's row-cropped frames).
int process_plan(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields, void* coefs,
                 void* scratch, size_t scratch_bytes, cudaStream_t st);
// Rows [row0, row0 + rows) of a frame that hold every polarisation's window.
void window_rows(const dhk::Plan& P, int* row0, int* rows);

}  // namespace dh
