/*
 * digholo.h - C ABI of the GB300 (sm_103a) batched off-axis hologram reconstruction library.
 *
 * The library implements digHolo's processing pipeline (user guide v1.0, "digHolo processing pipeline"):
 *   1. cut the FFT window around each polarisation's beam centre and Fourier transform it;
 *   2. select the off-axis term inside a circular Fourier window centred on the reference tilt, shift it
 *      to the origin, inverse transform it at the window's reduced size, and remove the reference's
 *      residual tilt and defocus;
 *   3. project the reconstructed field onto a Hermite-Gaussian basis.
 * Every step runs as hand-written CUDA kernels on the caller's stream; there is no CPU fallback.
 *
 * Conventions (the user guide leaves these open; the same readings are used throughout):
 *   - frames are row-major [batch][height][width], x fastest; pixel (i, j) is centred at (i px, j px);
 *   - window origin o = round_half_away(c / px) - N/2 per axis, c the beam centre in metres;
 *   - angles map to bins linearly: kappa = theta_rad * N * px / lambda, r = w_c,rad * N * px / lambda;
 *   - the kept bins form an M x M box starting at round_half_away(kappa) - M/2, masked by the circle
 *     ((k - kappa)/r)^2 summed over both axes <= 1 and by the real-to-complex half plane 0 <= k_x <= N/2;
 *   - fields are complex64 [batch][pol][M][M] sampled at x'_i = (i - M/2) N px / M from the beam centre,
 *     E = (1/N^2) sum_q F(k0+q) exp(2 pi i q.x'/(N px)) exp(-2 pi i (kappa-k0).x'/(N px)) exp(-i pi D |x'|^2/lambda);
 *   - coefficients are complex64 [batch][pol][modes], polarisation-blocked ("HHHHHVVVVV", as
 *     digHoloBasisGetCoefs lays them out); modes HG(m, n) with m + n < G, ordered by group g = m + n, then m
 *     ascending; c_mn = dx' dy' sum_ij u_m(x'_i) u_n(y'_j) E_ji with L2-normalised real u_n (other bases:
 *     dh_set_basis_type).
 *
 * Ownership: every device pointer passed in (frames, fields, coefficients, powers) is owned by the caller and
 * must stay valid until the work queued on the given stream has finished.  The library owns only its plan
 * tables and scratch, which it allocates on the current device when a plan is first used after a change.
 * Units follow the guide's "units" module: metres, dioptre, degrees.
 *
 * Error behaviour: every function returns one of the DH_* codes below (numeric values as the guide's
 * DIGHOLO_ERROR_* codes, plus DH_ERROR_TIMEOUT and DH_ERROR_CUDA).  dh_last_error() returns a thread-local
 * description of the most recent failure.  A failed call leaves the handle's settings unchanged.
 */
#ifndef DIGHOLO_GB300_H
#define DIGHOLO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes ("Error codes" module of the guide; 12 and 13 are added here). */
#define DH_SUCCESS 0
#define DH_ERROR_ERROR 1
#define DH_ERROR_INVALIDHANDLE 2
#define DH_ERROR_NULLPOINTER 3
#define DH_ERROR_INVALIDDIMENSION 5
#define DH_ERROR_INVALIDPOLARISATION 6
#define DH_ERROR_INVALIDAXIS 7
#define DH_ERROR_INVALIDARGUMENT 8
#define DH_ERROR_MEMORYALLOCATION 9
#define DH_ERROR_TIMEOUT 12
#define DH_ERROR_CUDA 13

/* Frame pixel types (digHoloSetBatch takes float32, digHoloSetBatchUint16 takes uint16). */
#define DH_DTYPE_U16 0
#define DH_DTYPE_F32 1

/* Arithmetic of the modal overlap: plain FP32 on CUDA cores, or BF16 tensor-core MMA with FP32 accumulation
 * and a hi/lo split of both operands (three products per term). */
#define DH_PRECISION_FP32 0
#define DH_PRECISION_SPLIT_BF16 1

/* Kernel variants of the reconstruction (dh_set_variant).  The guide's counterpart is the FFTW planning mode
 * (digHoloConfigSetFFTWPlanMode), which chooses how a transform is computed without changing its result. */
#define DH_VARIANT_AUTO 0           /* the library's choice, or the tuner's (dh_autotune) */
#define DH_VARIANT_FUSED 1          /* single-kernel path, window stays on chip: 128 x 128 windows, and 256 x 256
                                     * windows with 96 x 96 fields and uint16 frames */
#define DH_VARIANT_FUSED_PRUNED 2   /* single-kernel path transforming only the columns the window keeps */
#define DH_VARIANT_GENERIC 3        /* three-kernel path through library scratch (any window size) */
#define DH_VARIANT_FUSED_GROUPS 4   /* single-kernel path, every 1-D transform inside one 8-thread group, the x
                                     * transforms only on the box rows the window touches */

/* Coefficient bases (digHoloConfigSetBasisType): the field is always projected onto the HG modes; LG and
 * custom coefficients are a matrix applied to the HG coefficients. */
#define DH_BASIS_HG 0
#define DH_BASIS_LG 1
#define DH_BASIS_CUSTOM 2

/* Transfer-matrix metrics (DIGHOLO_METRIC_*, same indices). */
#define DH_METRIC_IL 0
#define DH_METRIC_MDL 1
#define DH_METRIC_DIAG 2
#define DH_METRIC_SNRAVG 3
#define DH_METRIC_DIAGBEST 4
#define DH_METRIC_DIAGWORST 5
#define DH_METRIC_SNRBEST 6
#define DH_METRIC_SNRWORST 7
#define DH_METRIC_SNRMG 8
#define DH_METRIC_COUNT 9
#define DH_MAX_METRIC_SIZE 1024

/* Largest sizes the kernels accept. */
#define DH_MAX_POLS 2
#define DH_MAX_WINDOW 1024
#define DH_MAX_FIELD 512
#define DH_MAX_GROUPS 32
#define DH_MAX_AVG_COUNT 4096

/* Averaging modes ("Averaging modes" module): where the avg_count frames of averaging group g sit. */
#define DH_AVGMODE_SEQUENTIAL 0        /* frames g avg_count + j: [A A A B B B] */
#define DH_AVGMODE_INTERLACED 1        /* frames j batch + g: [A B A B A B] */
#define DH_AVGMODE_SEQUENTIALSWEEP 2   /* blocks of wavelength sweeps; one wavelength here, so as SEQUENTIAL */

typedef int dh_handle;

/* Create a handle with default settings (digHoloCreate).  *out receives the handle index. */
int dh_create(dh_handle* out);

/* Release a handle and its device tables and scratch (digHoloDestroy).  Synchronises the device. */
int dh_destroy(dh_handle h);

/* Description of the last error raised on this thread (never NULL). */
const char* dh_last_error(void);

/* Frame geometry ("Frame buffer" module): width and height in pixels (positive), polarisation count 1 or 2
 * (the two components sit on opposite halves of the frame width), pixel pitch in metres (> 0).
 * Returns DH_ERROR_INVALIDDIMENSION, DH_ERROR_INVALIDPOLARISATION or DH_ERROR_INVALIDARGUMENT. */
int dh_set_frame(dh_handle h, int width, int height, int pol_count, double pixel_size);

/* Operating wavelength in metres, > 0 (digHoloConfigSetWavelengthCentre). */
int dh_set_wavelength(dh_handle h, double wavelength);

/* FFT window size (digHoloConfigSetfftWindowSize), per axis.  Values are floored to a multiple of 16 as the
 * guide's DIGHOLO_PIXEL_QUANTA rule says; each must then be a power of two 16..1024 (DH_ERROR_INVALIDDIMENSION
 * otherwise).  Non-square windows (nx != ny) run the generic three-kernel path with the FP32 overlap (the fused,
 * split-BF16 and candidate-scoring paths serve square windows and fields).  *set_nx / *set_ny (nullable) receive
 * the sizes actually set. */
int dh_set_fft_window(dh_handle h, int nx, int ny, int* set_nx, int* set_ny);

/* Beam centre of one axis (0 = x, 1 = y) and polarisation, metres (digHoloConfigSetBeamCentre). */
int dh_set_beam_centre(dh_handle h, int axis, int pol, double centre);

/* Radius w_c of the circular Fourier window, degrees, > 0 (digHoloConfigSetFourierWindowRadius). */
int dh_set_fourier_window_radius(dh_handle h, double radius_deg);

/* Reduced field size per axis (IFFT resolution mode 1).  0 selects the guide's rule M = 16 ceil(2 r / 16) with r
 * the window radius in that axis' bins (the FFT [IFFT] table of the Benchmarks section); otherwise a positive
 * multiple of 16 up to min(N, 512) of that axis whose odd part has prime factors <= 19.  Fields are
 * [M_y][M_x]. */
int dh_set_ifft_size(dh_handle h, int mx, int my);

/* Reference tilt of one axis and polarisation, degrees (digHoloConfigSetTilt): the position of the
 * off-axis term in Fourier space. */
int dh_set_tilt(dh_handle h, int axis, int pol, double tilt_deg);

/* Reference defocus of one polarisation, dioptre (digHoloConfigSetDefocus). */
int dh_set_defocus(dh_handle h, int pol, double dioptre);

/* Hermite-Gaussian basis (digHoloConfigSetBasisWaist, digHoloConfigSetBasisGroupCount): waist in metres (> 0)
 * of polarisation pol, and the group count G (0..DH_MAX_GROUPS, shared by both polarisations; G = 0 means no
 * modal decomposition and no coefficients). */
int dh_set_basis(dh_handle h, int pol, double waist, int group_count);

/* Fill-factor correction (digHoloConfigSetFillFactorCorrectionEnabled): when enabled (nonzero) the frames are
 * taken to come from pixels with a 100 % fill factor, and the kept Fourier bins are divided by the pixel
 * response sinc(k/N) = sin(pi k/N) / (pi k/N) of both axes (k the unwrapped bin) before the inverse transform.
 * Off by default. */
int dh_set_fill_factor_correction(dh_handle h, int enabled);

/* Coefficient basis (digHoloConfigSetBasisType; "Modal decomposition" module): DH_BASIS_HG, DH_BASIS_LG or
 * DH_BASIS_CUSTOM.  The field is always decomposed in the separable HG basis; the other bases are a matrix T
 * applied to each polarisation's HG coefficients on the GPU, c_out[k] = sum_l T[k][l] c_HG[l], FP32.
 *   - LG: modes LG_p^l with group N = 2p + |l| < G, ordered by group, then l ascending (-N, -N+2, ..., N);
 *     LG_p^l(r, phi) = sqrt(2 p! / (pi (p+|l|)!)) / w (sqrt(2) r / w)^|l| L_p^|l|(2 r^2/w^2) exp(-r^2/w^2)
 *     exp(i l phi) with L the generalised Laguerre polynomial, and c_pl = <LG_p^l | E>.  The matrix is built in
 *     FP64 from the closed-form HG-LG relation; G modes per group, so the count equals the HG count.
 *   - custom: the matrix set by dh_set_basis_transform.  Selecting DH_BASIS_CUSTOM before any matrix was set
 *     computes HG coefficients, as the guide states.
 * Returns DH_ERROR_INVALIDARGUMENT for other values.  dh_get_output_dims reports the coefficient count of the
 * selected basis; dh_score_settings always scores the HG coefficients. */
int dh_set_basis_type(dh_handle h, int basis);

/* Custom basis (digHoloConfigSetBasisTypeCustom): copies the host complex64 matrix transform
 * [modes_out][modes_in] (row-major, interleaved re/im) and selects DH_BASIS_CUSTOM.  Columns beyond the HG mode
 * count of the current G are unused; HG modes beyond modes_in contribute nothing.  1 <= modes_in, modes_out
 * and modes_in * modes_out <= 2^24, else DH_ERROR_INVALIDDIMENSION; NULL transform gives DH_ERROR_NULLPOINTER. */
int dh_set_basis_transform(dh_handle h, int modes_in, int modes_out, const void* transform);

/* Reference-wave calibration (digHoloConfigSetRefCalibrationIntensity): cal is a host uint16 array of
 * wavelength_count frames [height][width], the measured intensity of the reference wave alone (any exposure).
 * It is normalised by its maximum over all its pixels and frames, and every frame is multiplied pixel by pixel
 * by sqrt(max / cal) = 1 / (relative reference amplitude) before the transform (0 where cal = 0), which removes
 * a non-uniform reference amplitude from the off-axis term.  One wavelength is processed here, so the first
 * calibration frame is used.  The array is copied; the calibration is enabled.  width x height must equal the
 * frame size when a batch is processed (DH_ERROR_INVALIDDIMENSION otherwise).  As in the guide, an invalid
 * call (cal NULL: DH_ERROR_NULLPOINTER; a count or size < 1, or an all-zero array: DH_ERROR_INVALIDARGUMENT)
 * disables the calibration: the one exception to "a failed call leaves the settings unchanged". */
int dh_set_ref_calibration(dh_handle h, const uint16_t* cal, int wavelength_count, int width, int height);

/* Enable (nonzero) or disable the reference calibration last set (digHoloConfigSetRefCalibrationEnabled);
 * enabling without one gives DH_ERROR_INVALIDARGUMENT. */
int dh_set_ref_calibration_enabled(dh_handle h, int enabled);

/* Overlap arithmetic (the transforms are FP32 either way): DH_PRECISION_FP32, or DH_PRECISION_SPLIT_BF16, the
 * y contraction of the HG overlap on the tensor cores with bfloat16 hi + lo parts of the field and of the basis
 * (hi hi + hi lo + lo hi, FP32 accumulation); coefficients then agree with the FP32 ones to about 1e-5
 * relative.  Any other value gives DH_ERROR_INVALIDARGUMENT. */
int dh_set_precision(dh_handle h, int precision);

/* Hold the handle to one kernel variant (DH_VARIANT_*), as the guide's FFTW planning mode
 * (digHoloConfigSetFFTWPlanMode) selects how transforms are computed; every variant computes the same
 * reconstruction to rounding.  A variant that does not apply to the current settings (a fused variant for a
 * window other than 128 x 128 or 256 x 256 with 96 x 96 fields (the latter: uint16 frames, at most 16 HG
 * groups), the pruned and the group variants outside 128 x 128 windows with 64 x 64 fields and the FP32 overlap
 * (the pruned one also needs at most 48 kept columns), or frames whose base or row pitch is not 16-byte
 * aligned) falls back to the next one that does (pruned or groups -> fused -> generic).  DH_VARIANT_AUTO (the
 * default) takes the tuner's choice when one exists for these settings, else the fused variant where it
 * applies and the generic one elsewhere.  Unknown values give DH_ERROR_INVALIDARGUMENT. */
int dh_set_variant(dh_handle h, int variant);

/* The variant that dh_process_batch runs for the current settings and aligned frames (the fallbacks and the
 * tuner's choice resolved); validates the settings like dh_get_output_dims. */
int dh_get_variant(dh_handle h, int* variant);

/* ---------------------------------------------------------------------------------------------- autotuner
 * The guide lets FFTW plan its transforms (digHoloConfigSetFFTWPlanMode: estimate ... exhaustive) and keeps
 * the plans in a wisdom file (digHoloFFTWWisdomFilename) so later runs skip the search.  Here the choices are
 * the kernel variant, the generic path's chunk size (frames per launch, which decides whether the spectra stay
 * in L2 between its kernels) and the radix plan of the M-point inverse transforms.  dh_autotune times every
 * candidate on the caller's frames and keeps the fastest; the choices are stored per geometry key in a JSON
 * cache file, the analogue of the wisdom file.  Every candidate computes the same reconstruction to rounding. */

#define DH_MAX_RADICES 6

typedef struct dh_tuning {
    int variant;                     /* DH_VARIANT_* (DH_VARIANT_AUTO: the library's default) */
    int chunk_mb;                    /* generic path: scratch target per launch chunk in MiB (0: default 48) */
    int nradix;                      /* radix plan of the field size M, first pass first (0: the default plan) */
    int radix[DH_MAX_RADICES];       /* each radix in {2, 3, 4, 5, 7, 8, 11, 13, 16, 17, 19}, product M */
} dh_tuning;

/* Geometry key the tuner files choices under (field size, window, groups, polarisations, frame size,
 * precision, basis), as a NUL-terminated string in buf (at most len bytes, 128 suffice).  Host only. */
int dh_tuning_key(dh_handle h, char* buf, int len);

/* The candidates dh_autotune times for the current settings, in its order (host only): at most max entries
 * written to out, their number to *count (may exceed max).  For 128 x 128 windows: the group variant where it
 * applies, the fused variant, the pruned one where it applies, and the generic path; otherwise the generic path at chunk targets 24, 48 and
 * 96 MiB with the default radix plan of M and up to three alternatives (the reversed plan, other power-of-two
 * factorisations). */
int dh_tuning_candidates(dh_handle h, dh_tuning* out, int max, int* count);

/* Hold the handle to one tuning (NULL: back to the defaults and the cache).  The radix plan is validated
 * (DH_ERROR_INVALIDARGUMENT unless its radices are supported and multiply to M); a changed plan re-uploads the
 * tables on the next call.  The tuning stays while the geometry key is unchanged. */
int dh_set_tuning(dh_handle h, const dh_tuning* t);

/* The tuning in effect for the current settings: the one set or chosen for this key, else the cache's entry,
 * else zeros (defaults).  Host only. */
int dh_get_tuning(dh_handle h, dh_tuning* out);

/* Load tuning choices from a JSON cache file and remember the path (dh_autotune writes its choices back to
 * it).  A missing file is an empty cache; a malformed one gives DH_ERROR_INVALIDARGUMENT and leaves the
 * handle's cache unchanged.  NULL forgets the path and the loaded choices. */
int dh_set_tuning_cache(dh_handle h, const char* path);

/* Time every candidate of dh_tuning_candidates on these frames (one untimed run, then `reps` runs between
 * CUDA events on `stream`, reps < 1 taken as 3), keep the fastest (the first on ties), record it under the
 * geometry key (and in the cache file when one is set) and run it once more, so that d_fields / d_coefs
 * (as for dh_process_batch) hold its results on return.  Synchronises the device; uses the handle's own
 * scratch.  Changes no GPU setting. */
int dh_autotune(dh_handle h, const void* d_frames, int dtype, int batch, void* d_fields, void* d_coefs, void* stream,
                int reps);

/* Validate the settings and report the output geometry: field size M_x (equal to M_y for square fields),
 * number of coefficients per polarisation in the selected basis, and the field sample pitch dx' = N_x px / M_x
 * in metres.  Any pointer may be NULL.  Returns DH_ERROR_INVALIDARGUMENT when a polarisation's window leaves
 * the frame, its tilt centre leaves the half plane 0 < kappa_x <= N_x/2, or a field size exceeds its window. */
int dh_get_output_dims(dh_handle h, int* m, int* modes, double* dx);

/* The field's size and sample pitch along both axes (dh_get_output_dims' validation): fields are [M_y][M_x]
 * complex64 per polarisation, dx' = N_x px / M_x, dy' = N_y px / M_y.  Any pointer may be NULL. */
int dh_get_field_dims(dh_handle h, int* mx, int* my, double* dx, double* dy);

/* Field axes of one polarisation in metres from its beam centre (digHoloGetFields' x and y): host arrays of
 * at least M_x (x) and M_y (y) doubles. */
int dh_get_axes(dh_handle h, int pol, double* x, double* y);

/* Reconstruct a batch (digHoloProcessBatch).  d_frames: device array [batch][height][width] of uint16 or
 * float32 (dtype); d_fields (nullable): device complex64 [batch][pol][M][M]; d_coefs (nullable, ignored when
 * G = 0): device complex64 [batch][pol][modes].  batch < 1 is treated as 1 (digHoloConfigSetBatchCount).
 * Asynchronous on stream (a cudaStream_t, NULL = legacy default stream); the plan tables are uploaded on
 * the first call after a settings change, which synchronises the device once.  Geometries that take the
 * generic multi-kernel path keep the spectra between their kernels in scratch owned by the handle, one
 * buffer per handle: calls on one handle queued on different streams race on it, so queue them on one stream
 * (or use one handle per stream). */
int dh_process_batch(dh_handle h, const void* d_frames, int dtype, int batch, void* d_fields, void* d_coefs,
                     void* stream);

/* Host-buffer variant of dh_process_batch, as the guide's own processing call works on frames in host memory
 * (digHoloSetBatch / digHoloSetBatchUint16, then digHoloProcessBatch).  h_frames: host [batch][height][width]
 * uint16 or float32; h_fields (nullable): host complex64 [batch][pol][M][M]; h_coefs (nullable, ignored when
 * G = 0): host complex64 [batch][pol][modes].  The batch is cut into chunks that cycle over four internal
 * streams with their own device staging buffers (at most 256 MiB each, owned by the handle and kept for the
 * next call), so that host-to-device copies, reconstruction and device-to-host copies of consecutive chunks
 * overlap; only the frame rows that hold the polarisation windows are copied to the device.  The kernels and
 * results are those of dh_process_batch.  The work starts after the work already
 * queued on stream; the call returns when the outputs are in host memory (stream then also waits for it).
 * Page-locked host buffers are needed for the copies to overlap; pageable ones work but copy synchronously. */
int dh_process_batch_host(dh_handle h, const void* h_frames, int dtype, int batch, void* h_fields, void* h_coefs,
                          void* stream);

/* dh_process_batch_host that returns once the copies and kernels are queued, for streams of batches: the next
 * call's uploads then start while this call's downloads run.  The work starts after the work already queued on
 * stream; the outputs of every call made so far are in host memory when dh_process_batch_host_wait returns.
 * Until then h_frames must stay unchanged and valid, h_fields / h_coefs must not be read, and the handle's
 * settings must not change.  Calls on one handle run chunk by chunk in call order, so consecutive calls may
 * reuse the same host buffers.  Page-locked host buffers are needed for the call to return before the copies
 * complete (pageable ones copy synchronously). */
int dh_process_batch_host_async(dh_handle h, const void* h_frames, int dtype, int batch, void* h_fields,
                                void* h_coefs, void* stream);

/* Wait for every dh_process_batch_host_async call made on the handle: returns DH_SUCCESS once their outputs are
 * in host memory, or the CUDA error of the pipeline (DH_ERROR_CUDA). */
int dh_process_batch_host_wait(dh_handle h);

/* As dh_process_batch, and also writes the Fourier window that is inverse transformed for every (frame, pol)
 * (digHoloGetFourierPlaneWindow): d_window complex64 [batch][pol][M][M] with
 * d_window[q][p] = mask(p, q) (-1)^(p+q) F(k0x - M/2 + p, k0y - M/2 + q) / N^2, F the window spectrum in the
 * conventions above (the (-1)^(p+q) factor centres the inverse transform on the beam centre).  This entry
 * always takes the generic multi-kernel path. */
int dh_process_batch_window(dh_handle h, const void* d_frames, int dtype, int batch, void* d_window,
                            void* d_fields, void* d_coefs, void* stream);

/* Averaged reconstruction (digHoloSetBatchAvg / digHoloSetBatchAvgUint16 followed by digHoloProcessBatch).
 * d_frames holds batch * avg_count frames laid out as avg_mode says; the frames of each averaging group are
 * Fourier transformed and windowed, the kept window of member j is multiplied by the unit phasor
 * a_j = conj(d_j) / |d_j| with d_j = sum over polarisations and kept bins of conj(W_0) W_j (a_0 = 1; a_j = 1
 * when d_j = 0), so that it is in phase with the group's first member, and the aligned windows are averaged,
 * (1/avg_count) sum_j a_j W_j (after the fill-factor correction when it is enabled).  One inverse transform,
 * correction and decomposition per group follow: d_fields [batch][pol][M][M], d_coefs [batch][pol][modes] as
 * for dh_process_batch.  batch < 1 and avg_count < 1 are treated as 1 (avg_count = 1 is dh_process_batch);
 * avg_count > DH_MAX_AVG_COUNT gives DH_ERROR_INVALIDDIMENSION and an unknown avg_mode
 * DH_ERROR_INVALIDARGUMENT.  Always takes the generic multi-kernel path; asynchronous on stream. */
int dh_process_batch_avg(dh_handle h, const void* d_frames, int dtype, int batch, int avg_count, int avg_mode,
                         void* d_fields, void* d_coefs, void* stream);

/* Allocation-free variant of dh_process_batch.  The paper has no counterpart (digHolo allocates its own
 * buffers).  It exists for callers that cannot let a library allocate device memory while they process: code
 * whose device memory belongs to another allocator (a framework's caching pool, a serving process that has
 * already divided a fixed HBM budget) and acquisition loops that must not stall, since cudaMalloc / cudaFree
 * synchronise the device and can fail in the middle of a run.  It runs the generic kernels of dh_process_batch
 * with the same arguments, outputs and error codes, always with the FP32 overlap (a handle set to
 * DH_PRECISION_SPLIT_BF16 still gets FP32 coefficients here), but takes its plan tables and scratch from
 * one 16 MiB array of static device memory (1 MiB of tables, 15 MiB of scratch) that every GPU loading the
 * library holds until the process exits; it calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current and sets the kernels' shared-memory attribute; make that first call before any stream
 *     capture.
 *   - Each call uploads its plan tables with a copy ordered on `stream` (which first waits for the work
 *     already queued on that stream), then processes the batch in chunks that fit the scratch.
 *   - Geometries whose tables exceed 1 MiB, or whose single frame needs more than 15 MiB of scratch, are
 *     rejected with DH_ERROR_INVALIDDIMENSION (the supported limits, N <= 1024 and M <= 512, fit; an
 *     output-basis matrix counts against the tables: the LG matrix fits up to G = 16 at every supported size).
 *   - All calls share the array, which keeps the last call's contents; nothing in it needs to start at zero
 *     (every element is written before it is read within a call).  Calls that overlap on the GPU (different
 *     streams, or threads without ordering) race on the array: serialise them on one stream.
 *   - Its status block is the first 16 bytes of the array's table area, zeroed by each call's table upload
 *     (so it reflects the last call); dh_get_device_status and dh_get_check_record fold it into their reports
 *     on any handle.  Its kernels contain no bounded waits: only the bounds-checked build's guards set it. */
int dh_process_batch_noalloc(dh_handle h, const void* d_frames, int dtype, int batch, void* d_fields, void* d_coefs,
                             void* stream);

/* One alignment candidate for dh_score_settings: per polarisation tilt (x, y) in degrees, defocus in
 * dioptre and basis waist in metres. */
typedef struct dh_setting {
    double tilt_deg[DH_MAX_POLS][2];
    double defocus[DH_MAX_POLS];
    double waist[DH_MAX_POLS];
} dh_setting;

/* Total captured power of every frame under every candidate (the quantity the guide's AutoAlign search
 * maximises): d_power device float32 [batch][count], P[b][s] = sum_pol sum_modes |c_{b,pol,s}|^2, with each
 * candidate's own tilt, defocus and waist and the handle's other settings.  settings: host array of count
 * candidates (count >= 1).  Fields are not written. */
int dh_score_settings(dh_handle h, const void* d_frames, int dtype, int batch, const dh_setting* settings,
                      int count, float* d_power, void* stream);

/* Transfer-matrix metrics of a coefficient batch (digHoloAutoAlignCalcMetrics; AutoAlign metric defines).
 * d_coefs: device complex64 [batch][pol][modes] as this handle writes them (modes as dh_get_output_dims
 * reports); row b of the transfer matrix A is batch element b, its columns are the pol x modes coefficients.
 * metrics: host double[DH_METRIC_COUNT], all in dB (10 log10):
 *   IL = mean eigenvalue of the Gram matrix (the smaller of A A^H, A^H A: the squared singular values),
 *   MDL = largest / smallest of them (eigenvalues below 1e-12 of the largest count as 0: MDL = +inf),
 *   DIAG = sum_i |X_ii|^2, SNRAVG = diagonal / off-diagonal power, DIAGBEST / DIAGWORST = largest / smallest
 *   |X_ii|^2, SNRBEST / SNRWORST = largest / smallest row ratio |X_ii|^2 / sum_{j != i} |X_ij|^2, SNRMG = as
 *   SNRAVG with every coupling inside one mode group of one polarisation counted as signal (row i and column
 *   i taken as the same mode); X = A, or A A^H when mul_conj_trans is nonzero
 *   (digHoloConfigSetAutoAlignBasisMulConjTrans); the diagonal has min(rows, columns) elements.  Zero power
 *   gives -inf, a zero denominator +inf; SNRMG is -FLT_MAX ("not calculated", as the guide) for a custom basis.
 * eigenvalues (nullable): host double[min(batch, pol x modes)], the Gram eigenvalues (unsorted).
 * The Gram products and the eigenvalues (parallel cyclic Jacobi, at most 40 sweeps) run in FP64 on the GPU;
 * min(batch, pol x modes) and, with mul_conj_trans, batch must be <= DH_MAX_METRIC_SIZE
 * (DH_ERROR_INVALIDDIMENSION).  FP64 is slow on this GPU: about 10 ms at 100 rows, seconds at 1024.
 * Synchronous: allocates scratch, queues on stream and waits. */
int dh_calc_metrics(dh_handle h, const void* d_coefs, int batch, int mul_conj_trans, double* metrics,
                    double* eigenvalues, void* stream);

/* Current alignment settings of every polarisation (digHoloConfigGetTilt / GetDefocus / GetBasisWaist) into
 * *out (host). */
int dh_get_alignment(dh_handle h, dh_setting* out);

/* Fine-alignment search (digHoloAutoAlign's tweak stage; goal: captured power / insertion loss).  Starting from
 * the handle's tilt, defocus and waist, each iteration scores with dh_score_settings the centre and, for every
 * polarisation and parameter (tilt x, tilt y, defocus, waist), the settings with that parameter moved by -step
 * and +step (candidates in that order; waist steps relative, w (1 -/+ step)); it moves to the candidate with the
 * largest power summed over the batch (FP64 sum on the GPU) when that beats the centre (ties: first candidate),
 * and otherwise halves every step.  It stops when every step is below its minimum or after max_iter scorings,
 * and writes the final settings to the handle.  steps / min_steps: host double[3] (tilt degrees, defocus
 * dioptre, relative waist); NULL gives {0.02, 0.1, 0.05} / {2e-4, 1e-3, 5e-4}.  power (nullable): the final
 * total power; iterations (nullable): scorings run.  Synchronous. */
int dh_auto_align(dh_handle h, const void* d_frames, int dtype, int batch, const double* steps,
                  const double* min_steps, int max_iter, double* power, int* iterations, void* stream);


/* ------------------------------------------------------------------------------------------------------------
 * Serving loop (continuous batching).  The guide's library processes one batch per call on the caller's thread;
 * this server accepts requests at any time from any thread, admits each as soon as a stream slot is free and
 * its device memory fits a fixed HBM budget, and overlaps admitted requests on the device.  Plans (bases,
 * twiddles, masks) stay resident on the device per geometry handle.
 *
 * A request names a configured handle (its geometry and settings, which must not change while the request is
 * pending), host frames [batch][height][width] and optional host outputs (fields [batch][pol][M][M] and
 * coefficients [batch][pol][modes], complex64).  Pinned host memory gives asynchronous copies.  A request
 * larger than the budget is processed in consecutive frame chunks inside its reservation; a request whose
 * single frame does not fit is rejected at submission with DH_ERROR_MEMORYALLOCATION.  Results do not depend
 * on which other requests share the device (the kernels are deterministic and requests never share memory).
 * ------------------------------------------------------------------------------------------------------------ */
typedef struct dh_server_s* dh_server;

typedef struct dh_request {
    dh_handle geometry;        /* configured handle */
    const void* h_frames;      /* host frames */
    int dtype;                 /* DH_DTYPE_U16 or DH_DTYPE_F32 */
    int batch;                 /* frames, >= 1 */
    void* h_fields;            /* nullable host output */
    void* h_coefs;             /* nullable host output */
} dh_request;

typedef struct dh_stats {
    long long submitted, completed, failed, frames;
    double p50_ms, p99_ms, max_ms;   /* submit-to-completion latency of completed requests */
    double frames_per_s;             /* frames completed / (last completion - first submission) */
    size_t budget_bytes, peak_bytes; /* HBM budget and the largest reservation total seen */
    int max_inflight, peak_inflight;
    double wait_p50_ms, wait_p99_ms;     /* submission to admission */
    double kernel_p50_ms, kernel_p99_ms; /* device time of a request's own kernels (CUDA events around them) */
    double span_p50_ms, span_p99_ms;     /* device time from a request's first copy to its last on its stream */
    double kernel_ms_total;              /* sum of every completed request's kernel time */
    long long bypassed;                  /* admissions of a request past an earlier one that did not fit */
} dh_stats;

/* Create a server on the current device with an HBM budget in bytes (reserved with one allocation; 0 is
 * allowed and then admits nothing) and at most max_inflight concurrently processed requests (1..64, one
 * stream each).  Admission takes queued requests in arrival order; a request that does not fit the free
 * budget lets later ones that do fit go first, until it has waited DH_SERVER_MAX_WAIT_MS or been passed
 * DH_SERVER_MAX_BYPASS times, after which nothing is admitted before it. */
#define DH_SERVER_MAX_WAIT_MS 25
#define DH_SERVER_MAX_BYPASS 8
int dh_server_create(size_t hbm_budget, int max_inflight, dh_server* out);
/* Admission policy of a server: a request that does not fit may be passed by later ones until it has been
 * passed max_bypass times or has waited max_wait_ms (defaults DH_SERVER_MAX_BYPASS and DH_SERVER_MAX_WAIT_MS);
 * max_bypass = 0 admits strictly in arrival order.  Negative values give DH_ERROR_INVALIDARGUMENT. */
int dh_server_set_admission(dh_server s, int max_bypass, int max_wait_ms);
/* Queue a request; *ticket identifies it.  Validation errors are returned here. */
int dh_server_submit(dh_server s, const dh_request* r, uint64_t* ticket);
/* Wait for a request to finish (timeout_ms < 0: no limit).  Returns the request's own status, or
 * DH_ERROR_TIMEOUT when the wait ran out (the request keeps running). */
int dh_server_wait(dh_server s, uint64_t ticket, int timeout_ms);
/* Counters and latency percentiles of the server so far. */
int dh_server_stats(dh_server s, dh_stats* out);
/* Finish in-flight requests, fail queued ones, release the budget and the streams. */
int dh_server_destroy(dh_server s);

/* Failure detection.  Every wait inside a kernel (tensor-copy and tensor-core mbarriers) is bounded; when a
 * bound runs out the kernel writes NaN outputs for the affected windows, sets a bit in the handle's device
 * status word (bit 0: a staged-window copy did not arrive; bit 1: a tensor-core product did not complete) and
 * returns, leaving the context usable.  dh_get_device_status synchronises with the device, returns the word in
 * *status and clears it.  dh_check_bounded_wait runs the same bounded wait on an mbarrier that nothing ever
 * completes, with `limit` tries, and reports in *expired whether the limit ran out (1) as it must. */
int dh_get_device_status(dh_handle h, int* status);
int dh_check_bounded_wait(long long limit, int* expired);

/* Bounds-checked build (the paper has no counterpart; it stands in for a device memory checker).
 * libdigholo_gb300_checked.so is the same library compiled with DH_CHECKED:
 * before every guarded global-memory access of the reconstruction kernels (scratch regions against the extent
 * the host carved for them, outputs against the batch layout, 16-byte vector accesses against their alignment)
 * it tests the offset, skips the access when the test fails and records the failure instead of touching memory
 * outside the buffer: bit 2 of the device status word (dh_get_device_status), and the first failing guard site
 * with its offset and extent (low 32 bits each), which dh_get_check_record returns and clears (site 0: none;
 * sites are numbered in csrc/check.cuh).  In the normal build the guards compile away and the record stays 0.
 * dh_checked_build reports which build is loaded (1: checked).  dh_check_bounds_probe runs one guard at an
 * offset one past its extent, with no memory access behind it in either build: in the checked build it
 * records site 99 (offset 4, extent 4); in the normal build nothing. */
#define DH_STATUS_WAIT_COPY 1
#define DH_STATUS_WAIT_MMA 2
#define DH_STATUS_BOUNDS 4
int dh_get_check_record(dh_handle h, int* site, int* offset, int* extent);
int dh_checked_build(int* checked);
int dh_check_bounds_probe(dh_handle h);

/* Per-kernel device timing (the analogue of digHoloBenchmark's per-stage rates).  While enabled, every kernel
 * the handle launches is bracketed by a CUDA event pair recorded on the launch stream.  dh_set_profiling
 * clears the totals.  dh_get_profile waits for the recorded events and reports, per kernel, its name
 * (names: max_kernels slots of 64 chars, nullable), number of launches and total milliseconds since the last
 * reset; *count receives the number of distinct kernels (may exceed max_kernels). */
int dh_set_profiling(dh_handle h, int enable);
int dh_get_profile(dh_handle h, int max_kernels, char* names, long long* launches, double* total_ms, int* count);

#ifdef __cplusplus
}
#endif

#endif /* DIGHOLO_GB300_H */
