// Parameter blocks shared by the host launch code and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/digholo.h"

namespace dhk {

constexpr int kMaxRadices = 6;

// What one launch of the fused 128 x 128 kernel runs: the whole path, only the forward part (the masked window
// written to memory), or only the inverse part (the window read from memory).  Batch averaging combines the
// two split modes around the averaging kernels.
constexpr int kModeFull = 0, kModeForward = 1, kModeInverse = 2;

// Device tables of one polarisation (all pointers into the plan's device blob).
struct PolDev {
    int ox, oy;              // window origin in the frame
    int klx, kly;            // first box bin along x and y (unwrapped)
    const int* mask_lo;      // [M] first kept column of box row q
    const int* mask_hi;      // [M] last kept column of box row q
    const float2* phase_x;   // [M] (-1)^klo exp(-2 pi i (klo+p) eps / N) / N
    const float2* phase_y;   // [M]
    const float2* corr_x;    // [M] (-1)^i residual-tilt and defocus phase
    const float2* corr_y;    // [M]
    const float* hg_x;       // [G][M] u_g(x'_i) dx'
    const float* hg_y;       // [G][M]
    const uint16_t* hgy_tc;  // [2][NP][M] bf16 hi / lo of hg_y, tensor-core core-matrix layout
    const float* cal;        // nullable [N][N] reference-calibration factor over the window
    const unsigned char* pr; // nullable table block of the column-pruned fused kernel (fused_pr.hpp)
};

struct Plan {
    int n, m, groups, modes, pols;
    int width, height;
    int precision;           // DH_PRECISION_*
    int tc_np;               // rows of the tensor-core B operand (16 or 32)
    int nrad_n, nrad_m;
    int rad_n[kMaxRadices];
    int rad_m[kMaxRadices];
    const float2* tw_fwd_n;  // [N]
    const float2* tw_inv_m;  // [M]
    const int* pos_n;        // [N] position of frequency k after the forward DIF passes
    const int* pos_m;        // [M] position of index k for the inverse DIT input
    const int* mode_m;       // [modes]
    const int* mode_n;       // [modes]
    int modes_out;           // coefficients per polarisation in the output basis
    const float2* basis_tt;  // nullable [modes][modes_out]: transposed HG -> output-basis matrix (null: HG)
    int* status;             // nullable device status word: bit 0 set when a bounded wait expired
    PolDev pol[DH_MAX_POLS];
};

// One launch of the generic path over frames [frame0, frame0 + frames).
struct Batch {
    const void* src;         // frames [B][H][W] uint16 or float32
    int dtype;
    int frame0, count;       // frames [frame0, frame0 + count) of this launch
    float2* r1;              // scratch [frames][pol][M][N]: y-transformed box rows
    float2* g;               // scratch [frames][pol][M][M]: x-inverse-transformed rows
    float2* window;          // nullable [B][pol][M][M] masked window (natural order)
    float2* fields;          // nullable [B][pol][M][M]
    float2* coefs;           // nullable [B][pol][modes]
};

// Optional per-kernel device timing: start() before and stop() after every launch, on the launch stream.
struct StageTimer {
    virtual void start(cudaStream_t s) = 0;
    virtual void stop(cudaStream_t s, const char* kernel) = 0;
    virtual ~StageTimer() {}
};

// Launchers of the generic three-kernel path (k_split.cu).  Return cudaGetLastError().
cudaError_t launch_split(const Plan& plan, const Batch& batch, cudaStream_t stream, StageTimer* timer);
// k_ypass + k_xpass (window spectrum to x-inverse-transformed rows in batch.g) and the last kernel on their
// own (candidate scoring and batch averaging reuse them).
cudaError_t launch_forward(const Plan& plan, const Batch& batch, cudaStream_t stream, StageTimer* timer);
cudaError_t launch_ypass(const Plan& plan, const Batch& batch, cudaStream_t stream, StageTimer* timer);
cudaError_t launch_last(const Plan& plan, const Batch& batch, cudaStream_t stream, StageTimer* timer);
// Shared-memory opt-in, once per process and device.
cudaError_t split_init();
cudaError_t score_init();

// Output-basis transform (basis.cu): out[v][k] = sum_l T[k][l] hg[v][l] over `vectors` coefficient vectors
// (frames x polarisations) of plan.modes HG coefficients each; out holds plan.modes_out per vector.
cudaError_t launch_basis(const Plan& plan, const float2* hg, float2* out, int vectors, cudaStream_t stream,
                         StageTimer* timer);
cudaError_t basis_init();

// Batch averaging (k_avg.cu): phase-aligned mean of the x-inverse-transformed windows of each averaging
// group.  g holds groups x members windows of E = pols * M * M elements, member j of group gi at element
// offset gi * gstride + j * mstride; out receives [groups][E]; part is scratch of groups * members * slices.
int avg_slices(long long elems);
cudaError_t launch_avg(const float2* g, float2* part, float2* out, int groups, int members, long long elems,
                       long long mstride, long long gstride, cudaStream_t stream, StageTimer* timer);

// Split-BF16 tensor-core variant of the last generic kernel (k_overlap_tc.cu).
bool tc_supported(const Plan& plan);
cudaError_t tc_init();
cudaError_t launch_yinv_tc(const Plan& plan, const Batch& batch, cudaStream_t stream);

}  // namespace dhk
