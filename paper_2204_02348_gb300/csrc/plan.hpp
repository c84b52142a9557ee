// Host-side plan of one handle: settings, validation, FP64 geometry and the device tables derived from them.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>
#include <cstdint>

#include "../../include/digholo.h"

namespace dh {

// Settings exactly as the caller gave them (guide modules "Frame buffer", "Window sizes", "Wavelength",
// "Alignment", "Modal decomposition").
struct Settings {
    int width = 0, height = 0, pols = 1;
    double pixel = 20e-6;
    double wavelength = 1565e-9;
    int n = 128;                         // FFT window along x
    int ny = 128;                        // FFT window along y
    double centre[DH_MAX_POLS][2] = {{0, 0}, {0, 0}};
    double radius_deg = 0.0;
    int m_req = 0;                       // field size along x; 0: the guide's size rule
    int my_req = 0;                      // field size along y; 0: the guide's size rule
    double tilt_deg[DH_MAX_POLS][2] = {{0, 0}, {0, 0}};
    double defocus[DH_MAX_POLS] = {0, 0};
    double waist[DH_MAX_POLS] = {100e-6, 100e-6};
    int groups = 0;
    int precision = DH_PRECISION_FP32;
    int fill_factor = 0;                 // divide the window by the pixel response sinc(k/N) per axis
    int basis = DH_BASIS_HG;             // coefficient basis (custom falls back to HG until a matrix is set)
    int custom_in = 0, custom_out = 0;   // custom transform dimensions (modes in x modes out)
    std::vector<float> custom;           // custom transform, complex [custom_out][custom_in], interleaved re/im
    int cal_on = 0;                      // reference calibration enabled
    int cal_w = 0, cal_h = 0;            // calibration frame size
    double cal_max = 0.0;                // maximum over every calibration frame
    std::vector<uint16_t> cal;           // first calibration frame [cal_h][cal_w] (the single wavelength)
    std::vector<int> radix_m;            // radix plan of M chosen by the tuner (empty: radix_plan(M))
};

// Geometry of one axis of one polarisation (all FP64, computed as the conventions in digholo.h state).
struct AxisGeom {
    int origin;      // frame index of window pixel 0
    double eps;      // round_half_away(c/px) - c/px, the sub-pixel offset of the window grid
    double kappa;    // tilt in bins
    int k0;          // box centre bin
    int klo;         // first box bin, k0 - M/2
};

struct PolGeom {
    AxisGeom ax[2];
    double r;        // window radius in bins along x (the radius in angle times N_x px / lambda)
    double ry;       // the same along y (N_y px / lambda)
    double defocus, waist;
};

struct Geometry {
    int n, m, groups, modes, pols;   // n, m: window and field size along x
    int ny, my;      // window and field size along y (equal to n, m for square geometries)
    double dy;       // field pitch along y, N_y px / M_y
    int basis;       // effective basis: DH_BASIS_HG, DH_BASIS_LG or DH_BASIS_CUSTOM
    int modes_out;   // coefficients per polarisation in that basis (0 when G = 0)
    double dx;       // field pitch along x, N_x px / M_x
    bool square() const { return n == ny && m == my; }
    PolGeom pol[DH_MAX_POLS];
};

// Per-polarisation host tables in the layouts the kernels read (FP64 arithmetic, stored FP32).
struct PolTables {
    std::vector<float> phase_x, phase_y;   // complex [M]: (-1)^klo exp(-2 pi i (klo+p) eps / N) / N
    std::vector<float> corr_x, corr_y;     // complex [M]: (-1)^i exp(-2 pi i (kappa-k0)(i-M/2)/M) exp(-i pi D x'^2/lambda)
    std::vector<int> mask_lo, mask_hi;     // [M] per box row q: kept columns p in [lo, hi] (empty if lo > hi)
    std::vector<float> hg_x, hg_y;         // [G][M]: u_g(x'_i) dx'
    // split-BF16 tensor-core operand: u_n(y'_j) dy' as bf16 hi then lo, each [NP][M] in the K-major core-matrix
    // layout (8 rows x 8 values per 128-byte core; core (nb, kb) at (nb * M/8 + kb) * 128 bytes); rows n >= G zero
    std::vector<uint16_t> hgy_tc;
    // reference calibration over the window, [N][N] (y, x): sqrt(max cal / cal), 0 where cal = 0; empty if off
    std::vector<float> cal;
    // table block of the column-pruned fused kernel (fused_pr.hpp); empty when the geometry is not one it serves
    std::vector<unsigned char> pr;
    // coefficient-only tensor-core contraction (k_coef_tc.cu), empty when G = 0 or beyond its limits:
    // B = the y map [coef_np][2M] as bf16 hi and lo (rows n < G: real part of Y_n, G + n: imaginary part;
    // K = the window rows q of the real, then of the imaginary part of g), stored per chunk of 16 rows q as
    // [hi][lo] planes [coef_np][32] in the canonical K-major layout; then float2 X[G][M] = u_m(x'_i) dx' corr_x[i]
    std::vector<unsigned char> coef_tc;
    int coef_np = 0;
    // scoring contraction (k_coef_tc.cu, box source), the same layout with B = the y map times the y phase over
    // the raw box rows q, and C = Xh[G][M], the x weights carried back through the x inverse transform and the x
    // phase to the box columns p; built for alignment candidates only, empty otherwise or beyond the limits
    std::vector<unsigned char> score_tc;
};

// Rows of the tensor-core B operand (the group count rounded up to 16).
int tc_rows(int groups);
// Round-to-nearest-even bfloat16 bits of a float.
uint16_t bf16_bits(float v);

struct Tables {
    std::vector<float> tw_fwd_n;   // complex [N_x]: exp(-2 pi i k / N_x)
    std::vector<float> tw_inv_m;   // complex [M_x]: exp(+2 pi i k / M_x)
    std::vector<int> radix_n;      // radices of N_x (first pass first)
    std::vector<int> radix_m;      // radices of M_x
    std::vector<float> tw_fwd_ny;  // the y axis' tables (copies of the x ones for square geometries)
    std::vector<float> tw_inv_my;
    std::vector<int> radix_ny;
    std::vector<int> radix_my;
    std::vector<int> mode_m, mode_n;
    // basis transform, transposed: complex [modes][modes_out] holding T[k][l] at [l][k]; empty for HG
    std::vector<float> basis_tt;
    PolTables pol[DH_MAX_POLS];
};

// Round half away from zero, as the window origin and the box centre use.
int round_half_away(double v);
// The guide's reduced field size rule: 16 ceil(2 r / 16).
int ifft_size_rule(double r_bins);
// Factor a length into the radices the kernels implement; empty if impossible.
std::vector<int> radix_plan(int len);

// Validate settings and derive the geometry.  Returns DH_SUCCESS or an error code with a message.
int build_geometry(const Settings& s, Geometry* g, std::string* why);
// Geometry for one alignment candidate (tilt, defocus, waist replaced).
int build_geometry_candidate(const Settings& s, const dh_setting& c, Geometry* g, std::string* why);
// Fill the host tables of a geometry (score: also the scoring contraction's tables, PolTables::score_tc).
void build_tables(const Settings& s, const Geometry& g, Tables* t, bool score = false);
// build_tables of every geometry, the geometries taken in turn by up to `threads` host threads (0: the
// hardware's count, at most 16); tables do not depend on one another, so the result equals the serial loop's.
void build_tables_many(const Settings& s, const std::vector<Geometry>& g, std::vector<Tables>* t, bool score = false,
                       int threads = 0);
// Fill PolTables::coef_tc of polarisation p (u: the FP64 HG functions u_n at the field grid, [G][M]).
void build_coef_tc(const Settings& s, const Geometry& g, int p, const std::vector<double>& u, PolTables* pt);
// Fill PolTables::score_tc of polarisation p (same u).
void build_score_tc(const Settings& s, const Geometry& g, int p, const std::vector<double>& u, PolTables* pt);
// Fill PolTables::pr of polarisation p from its other tables (after they are built).
void build_pr_block(const Geometry& g, int p, PolTables* pt);
// HG -> LG coefficient matrix (FP64, complex interleaved [modes][modes], LG rows by group then l ascending,
// HG columns by group then m ascending): c_LG = T c_HG.
void lg_transform(int groups, std::vector<double>* t);
// HG 1D functions u_0..u_{G-1} at positions x (recurrence, FP64), row-major [G][len].
void hg_table(int groups, const double* x, int len, double waist, double* out);

}  // namespace dh
