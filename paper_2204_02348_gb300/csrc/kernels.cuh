// Parameter blocks shared by the host launch code and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/digholo.h"
#include "check.cuh"

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
    const unsigned char* coef_tc;   // nullable coefficient-only tensor-core tables: the y map as bf16 hi / lo
                                    // chunks of 16 window rows ([hi][lo] x [coef_np][32], canonical K-major),
                                    // then float2 X[G][M]
    const unsigned char* score_tc;  // nullable scoring tables, the same layout: phased y map over the raw box
                                    // rows, then float2 Xh[G][M] over the raw box columns
};

struct Plan {
    int n, m, groups, modes, pols;   // n, m: window and field size along x
    int ny, my;              // window and field size along y (n, m for square geometries)
    int width, height;
    int precision;           // DH_PRECISION_*
    int tc_np;               // rows of the tensor-core B operand (16 or 32)
    int coef_np;             // rows of the coefficient-only contraction's B operand (2G rounded up to 16), 0: none
    int nrad_n, nrad_m;
    int rad_n[kMaxRadices];
    int rad_m[kMaxRadices];
    const float2* tw_fwd_n;  // [N]
    const float2* tw_inv_m;  // [M]
    const int* pos_n;        // [N] position of frequency k after the forward DIF passes
    const int* pos_m;        // [M] position of index k for the inverse DIT input
    // the y axis' transforms (the generic kernels' y passes read these; equal to the x ones when square)
    int nrad_ny, nrad_my;
    int rad_ny[kMaxRadices];
    int rad_my[kMaxRadices];
    const float2* tw_fwd_ny; // [N_y]
    const float2* tw_inv_my; // [M_y]
    const int* pos_ny;       // [N_y]
    const int* pos_my;       // [M_y]
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
    long long r1_len;        // elements of the r1 scratch region (the bounds-checked build tests against them)
    long long g_len;         // elements of the g scratch region
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
// X: the status block and the element extents of g, part and out (tested by the bounds-checked build).
struct AvgExtents {
    int* status;
    long long g_len, part_len, out_len;
};
int avg_slices(long long elems);
cudaError_t launch_avg(const float2* g, float2* part, float2* out, int groups, int members, long long elems,
                       long long mstride, long long gstride, const AvgExtents& X, cudaStream_t stream,
                       StageTimer* timer);

// Coefficient-only split-BF16 last kernel (k_coef_tc.cu): the y transform, correction and y overlap as one
// tensor-core contraction of the x-inverse-transformed rows; for batches without fields.
bool coef_tc_supported(const Plan& plan, const Batch& batch);
cudaError_t coef_tc_init();
cudaError_t launch_coef_tc(const Plan& plan, const Batch& batch, cudaStream_t stream);

// Where an alignment candidate's box sits in the superset spectra of candidate scoring: window w (frame slot
// times pols plus polarisation) at xs + w ms msx, box row q and column p of polarisation pol at
// (qoff[pol] + q) msx + poff[pol] + p (raw DFT bins, before mask and phases).
struct BoxSrc {
    const float2* xs;
    int ms, msx;
    int qoff[DH_MAX_POLS], poff[DH_MAX_POLS];
    long long xs_len;        // elements of the superset spectra (tested by the bounds-checked build)
};
// The same contraction reading a candidate's box bins straight from the superset spectra, with the candidate's
// scoring tables (PolDev::score_tc): the x inverse transform is folded into the x weights, so no x-inverse
// kernel runs.  Coefficients of frame slot b at batch.coefs[(b pols + pol) modes] (batch.frame0 0).
bool score_tc_supported(const Plan& plan, const Batch& batch, const BoxSrc& src);
cudaError_t launch_score_tc(const Plan& plan, const Batch& batch, const BoxSrc& src, cudaStream_t stream);

// Split-BF16 tensor-core variant of the last generic kernel (k_overlap_tc.cu).
bool tc_supported(const Plan& plan);
cudaError_t tc_init();
cudaError_t launch_yinv_tc(const Plan& plan, const Batch& batch, cudaStream_t stream);

}  // namespace dhk
