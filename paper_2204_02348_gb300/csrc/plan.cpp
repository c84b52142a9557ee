// Host-side geometry and tables.  Compiled with -ffp-contract=off so every FP64 expression rounds exactly
// as written; the window-mask decision (a floating-point comparison that decides which bins are kept) is
// taken here, in FP64, once per plan.
#include "plan.hpp"

#include "fused_pr.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <thread>

namespace dh {

static const double kPi = 3.14159265358979323846;
static const double kDegToRad = kPi / 180.0;

int round_half_away(double v) { return (int)std::copysign(std::floor(std::fabs(v) + 0.5), v); }

int ifft_size_rule(double r_bins) { return 16 * (int)std::ceil(2.0 * r_bins / 16.0); }

std::vector<int> radix_plan(int len) {
    std::vector<int> out;
    if (len < 2) return out;
    int odd = len, two = 0;
    while (odd % 2 == 0) { odd /= 2; ++two; }
    // power-of-two part 2^two: few passes of radix 16 / 8, at most one smaller pass
    static const int pow2_plan[11][3] = {
        {0, 0, 0}, {2, 0, 0}, {4, 0, 0}, {8, 0, 0}, {16, 0, 0}, {8, 4, 0},
        {8, 8, 0}, {16, 8, 0}, {16, 16, 0}, {8, 8, 8}, {16, 8, 8}};
    if (two > 10) return out;
    for (int i = 0; i < 3 && pow2_plan[two][i]; ++i) out.push_back(pow2_plan[two][i]);
    static const int primes[] = {3, 5, 7, 11, 13, 17, 19};
    for (int p : primes)
        while (odd % p == 0) { out.push_back(p); odd /= p; }
    if (odd != 1) out.clear();
    return out;
}

static int axis_geometry(const Settings& s, int p, int ax, const double tilt_deg, AxisGeom* a) {
    const double c = s.centre[p][ax];
    const int rc = round_half_away(c / s.pixel);
    const int n = ax == 0 ? s.n : s.ny;
    a->origin = rc - n / 2;
    a->eps = (double)rc - c / s.pixel;
    a->kappa = tilt_deg * kDegToRad * (double)n * s.pixel / s.wavelength;
    a->k0 = round_half_away(a->kappa);
    return DH_SUCCESS;
}

static int fill(const Settings& s, const double tilt[DH_MAX_POLS][2], const double* defocus,
                const double* waist, Geometry* g, std::string* why) {
    if (s.width <= 0 || s.height <= 0) { *why = "frame size not set"; return DH_ERROR_INVALIDDIMENSION; }
    if (s.pols < 1 || s.pols > DH_MAX_POLS) { *why = "polarisation count must be 1 or 2"; return DH_ERROR_INVALIDPOLARISATION; }
    if (!(s.pixel > 0.0) || !(s.wavelength > 0.0)) { *why = "pixel size and wavelength must be positive"; return DH_ERROR_INVALIDARGUMENT; }
    if (!(s.radius_deg > 0.0)) { *why = "Fourier window radius must be positive"; return DH_ERROR_INVALIDARGUMENT; }
    g->n = s.n;
    g->ny = s.ny;
    g->pols = s.pols;
    g->groups = s.groups;
    g->modes = s.groups * (s.groups + 1) / 2;
    g->basis = s.basis == DH_BASIS_CUSTOM && s.custom.empty() ? DH_BASIS_HG : s.basis;
    g->modes_out = g->modes == 0 ? 0 : g->basis == DH_BASIS_CUSTOM ? s.custom_out : g->modes;
    // the radius in bins along each axis: the angle times that axis' N px / lambda
    const double r = s.radius_deg * kDegToRad * (double)s.n * s.pixel / s.wavelength;
    const double ry = s.radius_deg * kDegToRad * (double)s.ny * s.pixel / s.wavelength;
    g->m = s.m_req > 0 ? s.m_req : ifft_size_rule(r);
    g->my = s.my_req > 0 ? s.my_req : ifft_size_rule(ry);
    for (int ax = 0; ax < 2; ++ax) {
        const int m = ax == 0 ? g->m : g->my, n = ax == 0 ? s.n : s.ny;
        if (m < 16 || m % 16 || m > n || m > DH_MAX_FIELD || radix_plan(m).empty()) {
            char b[192];
            std::snprintf(b, sizeof b,
                          "field size M=%d invalid for window N=%d along axis %d (multiple of 16, <= N, <= %d, odd part 19-smooth)",
                          m, n, ax, DH_MAX_FIELD);
            *why = b;
            return DH_ERROR_INVALIDARGUMENT;
        }
    }
    if (s.cal_on && (s.cal_w != s.width || s.cal_h != s.height)) {
        char b[160];
        std::snprintf(b, sizeof b, "reference calibration is %d x %d, frames are %d x %d", s.cal_w, s.cal_h, s.width,
                      s.height);
        *why = b;
        return DH_ERROR_INVALIDDIMENSION;
    }
    g->dx = (double)s.n * s.pixel / (double)g->m;
    g->dy = (double)s.ny * s.pixel / (double)g->my;
    for (int p = 0; p < s.pols; ++p) {
        PolGeom& pg = g->pol[p];
        for (int ax = 0; ax < 2; ++ax) axis_geometry(s, p, ax, tilt[p][ax], &pg.ax[ax]);
        pg.r = r;
        pg.ry = ry;
        pg.defocus = defocus[p];
        pg.waist = waist[p];
        pg.ax[0].klo = pg.ax[0].k0 - g->m / 2;
        pg.ax[1].klo = pg.ax[1].k0 - g->my / 2;
        const int lim[2] = {s.width, s.height};
        for (int ax = 0; ax < 2; ++ax) {
            const int n = ax == 0 ? s.n : s.ny;
            if (pg.ax[ax].origin < 0 || pg.ax[ax].origin + n > lim[ax]) {
                char b[160];
                std::snprintf(b, sizeof b, "window of polarisation %d leaves the frame along axis %d (origin %d, N %d, frame %d)",
                              p, ax, pg.ax[ax].origin, n, lim[ax]);
                *why = b;
                return DH_ERROR_INVALIDARGUMENT;
            }
        }
        if (!(pg.ax[0].kappa > 0.0 && pg.ax[0].kappa <= s.n / 2.0)) {
            *why = "tilt x must place the window centre inside the half plane 0 < kappa_x <= N/2";
            return DH_ERROR_INVALIDARGUMENT;
        }
        if (s.groups > 0 && !(pg.waist > 0.0)) { *why = "basis waist must be positive"; return DH_ERROR_INVALIDARGUMENT; }
    }
    return DH_SUCCESS;
}

int build_geometry(const Settings& s, Geometry* g, std::string* why) {
    return fill(s, s.tilt_deg, s.defocus, s.waist, g, why);
}

int build_geometry_candidate(const Settings& s, const dh_setting& c, Geometry* g, std::string* why) {
    return fill(s, c.tilt_deg, c.defocus, c.waist, g, why);
}

void hg_table(int groups, const double* x, int len, double waist, double* out) {
    const double s2 = std::sqrt(2.0);
    const double norm = std::sqrt(s2 / waist);
    for (int i = 0; i < len; ++i) {
        const double xi = s2 * x[i] / waist;
        double prev = 0.0, cur = std::pow(kPi, -0.25) * std::exp(-0.5 * xi * xi);
        for (int k = 0; k < groups; ++k) {
            out[(size_t)k * len + i] = norm * cur;
            // psi_{k+1} = sqrt(2/(k+1)) xi psi_k - sqrt(k/(k+1)) psi_{k-1}
            const double next = std::sqrt(2.0 / (k + 1)) * xi * cur - std::sqrt((double)k / (k + 1)) * prev;
            prev = cur;
            cur = next;
        }
    }
}

int tc_rows(int groups) { return groups <= 16 ? 16 : 32; }

uint16_t bf16_bits(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);   // inf / nan unchanged
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

// Offset in elements of (row, k) in a [rows][K] bf16 tensor-core operand stored K-major in 8 x 8 core
// matrices (8 rows x 16 bytes, contiguous; core (row / 8, k / 8) at ((row / 8) (K / 8) + k / 8) * 64).
static size_t umma_offset(int row, int k, int K) {
    return ((size_t)(row >> 3) * (size_t)(K >> 3) + (size_t)(k >> 3)) * 64 + (size_t)(row & 7) * 8 + (size_t)(k & 7);
}

static float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

static void push_c(std::vector<float>& v, double re, double im) {
    v.push_back((float)re);
    v.push_back((float)im);
}

// Beam-centre phase of box bin klo + q along one axis, FP64: (-1)^klo exp(-2 pi i (klo + q) eps / N) / N, divided
// by the pixel response sinc((klo + q) / N) when the fill-factor correction is on.
static void phase_fp64(const Settings& s, const AxisGeom& a, int n, int q, double* re, double* im) {
    const double sgn = (a.klo % 2 == 0) ? 1.0 : -1.0;
    const double ang = -2.0 * kPi * (double)(a.klo + q) * a.eps / n;
    double w = sgn / n;
    if (s.fill_factor) {
        const double u = kPi * (double)(a.klo + q) / n;
        w /= (u == 0.0) ? 1.0 : std::sin(u) / u;
    }
    *re = w * std::cos(ang);
    *im = w * std::sin(ang);
}

// Tilt and defocus correction of field sample i along one axis, FP64:
// (-1)^i exp(-2 pi i (kappa - k0)(i - M/2) / M) exp(-i pi D x'_i^2 / lambda).
static void corr_fp64(const Settings& s, const Geometry& g, const PolGeom& pg, const AxisGeom& a, int ax, int i,
                      double* re, double* im) {
    const int m = ax == 0 ? g.m : g.my;
    const double xp = (double)(i - m / 2) * (ax == 0 ? g.dx : g.dy);
    const double ang = -2.0 * kPi * (a.kappa - a.k0) * (double)(i - m / 2) / m - kPi * pg.defocus * xp * xp / s.wavelength;
    const double sg = (i % 2 == 0) ? 1.0 : -1.0;
    *re = sg * std::cos(ang);
    *im = sg * std::sin(ang);
}

// LG_p^l as a sum over the HG modes of its group N = 2p + |l| (Hermite-Laguerre-Gauss relation, as in
// Beijersbergen et al., Opt. Commun. 96, 123 (1993)): with n = p + max(l, 0), m = p + max(-l, 0),
//   <HG(N-k, k) | LG_p^l> = (-1)^p (-i)^k b(n, m, k),
//   b(n, m, k) = sqrt((N-k)! k! / (2^N n! m!)) sum_j C(n, j) (-1)^j C(m, k-j),
// HG(a, b) = u_a(x) u_b(y) and LG_p^l carrying exp(+i l phi).  The LG coefficient of a field is
// <LG | E> = sum_k conj(<HG_k | LG>) <HG_k | E>, so T holds the conjugates: (-1)^p i^k b(n, m, k).  The binomial
// sums are integers below 2^(N+5) and are summed exactly in 64-bit integers.
void lg_transform(int groups, std::vector<double>* t) {
    const int modes = groups * (groups + 1) / 2;
    t->assign((size_t)2 * modes * modes, 0.0);
    auto binom = [](int a, int b) -> long long {
        if (b < 0 || b > a) return 0;
        long long r = 1;
        for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
        return r;
    };
    auto lfact = [](int a) { return std::lgamma((double)a + 1.0); };
    int base = 0;
    for (int grp = 0; grp < groups; ++grp) {
        int row = base;
        for (int l = -grp; l <= grp; l += 2, ++row) {
            const int p = (grp - std::abs(l)) / 2;
            const int n = p + std::max(l, 0), m = p + std::max(-l, 0);
            for (int k = 0; k <= grp; ++k) {
                long long sum = 0;
                for (int j = 0; j <= std::min(n, k); ++j) {
                    const long long term = binom(n, j) * binom(m, k - j);
                    sum += (j % 2) ? -term : term;
                }
                const double mag = std::exp(0.5 * (lfact(grp - k) + lfact(k) - grp * std::log(2.0) - lfact(n) - lfact(m)));
                const double b = mag * (double)sum * ((p % 2) ? -1.0 : 1.0);
                // i^k b; HG(x order grp - k, y order k) sits at column base + (grp - k)
                const double re = (k % 4 == 0) ? b : (k % 4 == 2) ? -b : 0.0;
                const double im = (k % 4 == 1) ? b : (k % 4 == 3) ? -b : 0.0;
                const size_t at = (size_t)row * modes + base + (grp - k);
                (*t)[2 * at] = re;
                (*t)[2 * at + 1] = im;
            }
        }
        base += grp + 1;
    }
}

void build_tables(const Settings& s, const Geometry& g, Tables* t, bool score) {
    const int n = g.n, m = g.m, ny = g.ny, my = g.my;
    t->tw_fwd_n.clear();
    t->tw_inv_m.clear();
    t->tw_fwd_ny.clear();
    t->tw_inv_my.clear();
    for (int k = 0; k < n; ++k) push_c(t->tw_fwd_n, std::cos(-2.0 * kPi * k / n), std::sin(-2.0 * kPi * k / n));
    for (int k = 0; k < m; ++k) push_c(t->tw_inv_m, std::cos(2.0 * kPi * k / m), std::sin(2.0 * kPi * k / m));
    for (int k = 0; k < ny; ++k) push_c(t->tw_fwd_ny, std::cos(-2.0 * kPi * k / ny), std::sin(-2.0 * kPi * k / ny));
    for (int k = 0; k < my; ++k) push_c(t->tw_inv_my, std::cos(2.0 * kPi * k / my), std::sin(2.0 * kPi * k / my));
    t->radix_n = radix_plan(n);
    // the tuner's radix plan is one of M (square geometries only)
    t->radix_m = s.radix_m.empty() || !g.square() ? radix_plan(m) : s.radix_m;
    t->radix_ny = radix_plan(ny);
    t->radix_my = g.square() ? t->radix_m : radix_plan(my);
    t->mode_m.clear();
    t->mode_n.clear();
    for (int gg = 0; gg < g.groups; ++gg)
        for (int mm = 0; mm <= gg; ++mm) { t->mode_m.push_back(mm); t->mode_n.push_back(gg - mm); }
    t->basis_tt.clear();
    if (g.modes > 0 && g.basis != DH_BASIS_HG) {
        const int mi = g.modes, mo = g.modes_out;
        t->basis_tt.assign((size_t)2 * mi * mo, 0.f);
        if (g.basis == DH_BASIS_LG) {
            std::vector<double> lg;
            lg_transform(g.groups, &lg);
            for (int k = 0; k < mo; ++k)
                for (int l = 0; l < mi; ++l) {
                    t->basis_tt[2 * ((size_t)l * mo + k)] = (float)lg[2 * ((size_t)k * mi + l)];
                    t->basis_tt[2 * ((size_t)l * mo + k) + 1] = (float)lg[2 * ((size_t)k * mi + l) + 1];
                }
        } else {
            // columns beyond the HG mode count are unused; HG modes beyond the matrix's columns contribute 0
            const int used = std::min(mi, s.custom_in);
            for (int k = 0; k < mo; ++k)
                for (int l = 0; l < used; ++l) {
                    t->basis_tt[2 * ((size_t)l * mo + k)] = s.custom[2 * ((size_t)k * s.custom_in + l)];
                    t->basis_tt[2 * ((size_t)l * mo + k) + 1] = s.custom[2 * ((size_t)k * s.custom_in + l) + 1];
                }
        }
    }
    std::vector<double> xp(m), yp(my);
    for (int i = 0; i < m; ++i) xp[i] = (double)(i - m / 2) * g.dx;
    for (int j = 0; j < my; ++j) yp[j] = (double)(j - my / 2) * g.dy;
    for (int p = 0; p < g.pols; ++p) {
        const PolGeom& pg = g.pol[p];
        PolTables& pt = t->pol[p];
        pt.cal.clear();
        if (s.cal_on) {
            // divide the frame by the reference's relative amplitude sqrt(cal / max cal)
            pt.cal.resize((size_t)ny * n);
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < n; ++x) {
                    const double c = s.cal[(size_t)(pg.ax[1].origin + y) * s.cal_w + pg.ax[0].origin + x];
                    pt.cal[(size_t)y * n + x] = c > 0.0 ? (float)std::sqrt(s.cal_max / c) : 0.f;
                }
        }
        std::vector<float>* ph[2] = {&pt.phase_x, &pt.phase_y};
        std::vector<float>* co[2] = {&pt.corr_x, &pt.corr_y};
        for (int ax = 0; ax < 2; ++ax) {
            const AxisGeom& a = pg.ax[ax];
            ph[ax]->clear();
            co[ax]->clear();
            const int ma = ax == 0 ? m : my, na = ax == 0 ? n : ny;
            for (int q = 0; q < ma; ++q) {
                double re, im;
                phase_fp64(s, a, na, q, &re, &im);
                push_c(*ph[ax], re, im);
            }
            for (int i = 0; i < ma; ++i) {
                double re, im;
                corr_fp64(s, g, pg, a, ax, i, &re, &im);
                push_c(*co[ax], re, im);
            }
        }
        // mask rows: the same FP64 expression as the definition, ((ky-kappa_y)/r_y)^2 + ((kx-kappa_x)/r_x)^2 <= 1
        // (per box row q < M_y, the kept box columns p < M_x)
        pt.mask_lo.assign(my, 1);
        pt.mask_hi.assign(my, 0);
        for (int q = 0; q < my; ++q) {
            const double ky = (double)(pg.ax[1].klo + q);
            const double ddy = (ky - pg.ax[1].kappa) / pg.ry;
            int lo = -1, hi = -2;
            for (int pp = 0; pp < m; ++pp) {
                const int kxi = pg.ax[0].klo + pp;
                const double ddx = ((double)kxi - pg.ax[0].kappa) / pg.r;
                const bool keep = (ddy * ddy + ddx * ddx <= 1.0) && kxi >= 0 && kxi <= n / 2;
                if (keep) {
                    if (lo < 0) lo = pp;
                    hi = pp;
                }
            }
            if (lo >= 0) { pt.mask_lo[q] = lo; pt.mask_hi[q] = hi; }
        }
        const double w = g.dx;   // quadrature weight of one axis: c = dx' dy' sum u_m u_n E
        std::vector<double> u((size_t)std::max(g.groups, 1) * m);
        pt.hg_x.clear();
        pt.hg_y.clear();
        pt.hgy_tc.clear();
        pt.pr.clear();
        pt.coef_tc.clear();
        pt.coef_np = 0;
        pt.score_tc.clear();
        if (g.groups > 0 && !g.square()) {
            // a field of M_x x M_y: u_m on the x grid (pitch dx'), u_n on the y grid (pitch dy'); the tensor-core
            // and fused-kernel tables are built for square geometries only
            hg_table(g.groups, xp.data(), m, pg.waist, u.data());
            for (size_t k = 0; k < (size_t)g.groups * m; ++k) pt.hg_x.push_back((float)(u[k] * w));
            std::vector<double> uy((size_t)g.groups * my);
            hg_table(g.groups, yp.data(), my, pg.waist, uy.data());
            for (size_t k = 0; k < (size_t)g.groups * my; ++k) pt.hg_y.push_back((float)(uy[k] * g.dy));
            continue;
        }
        if (!g.square()) continue;
        if (g.groups > 0) {
            hg_table(g.groups, xp.data(), m, pg.waist, u.data());
            for (size_t k = 0; k < (size_t)g.groups * m; ++k) pt.hg_x.push_back((float)(u[k] * w));
            pt.hg_y = pt.hg_x;   // the y grid equals the x grid (square box, same pitch)
            const int np = tc_rows(g.groups);
            pt.hgy_tc.assign((size_t)2 * np * m, 0);
            for (int n = 0; n < g.groups; ++n) {
                for (int j = 0; j < m; ++j) {
                    const double v = u[(size_t)n * m + j] * w;
                    const uint16_t hi = bf16_bits((float)v);
                    const uint16_t lo = bf16_bits((float)(v - (double)bf16_value(hi)));
                    const size_t off = ((size_t)(n / 8) * (m / 8) + j / 8) * 64 + (n % 8) * 8 + (j % 8);
                    pt.hgy_tc[off] = hi;
                    pt.hgy_tc[(size_t)np * m + off] = lo;
                }
            }
        }
        build_pr_block(g, p, &pt);
        build_coef_tc(s, g, p, u, &pt);
        pt.score_tc.clear();
        if (score) build_score_tc(s, g, p, u, &pt);
    }
}

void build_tables_many(const Settings& s, const std::vector<Geometry>& g, std::vector<Tables>* t, bool score,
                       int threads) {
    const int count = (int)g.size();
    t->resize(count);
    if (threads <= 0) threads = std::min(16, (int)std::max(1u, std::thread::hardware_concurrency()));
    threads = std::max(1, std::min(threads, count));
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int k = next++; k < count; k = next++) build_tables(s, g[k], &(*t)[k], score);
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < threads; ++i) pool.emplace_back(work);
    work();
    for (std::thread& th : pool) th.join();
}

// out[k] = sum_j in[j * stride] exp(+2 pi i k j / n) for k < n, in FP64: Cooley-Tukey on the smallest prime
// factor p of n (n = p m: p interleaved length-m transforms combined with twiddles), a direct sum for a prime.
// wr / wi: exp(+2 pi i e / L) for e < L, L a multiple of n (the root of unity of order n is entry L / n).
// Exponents k j mod n are stepped incrementally (one conditional subtraction each), so no division runs in the
// inner loops.
static void dft_plus(const double* re, const double* im, int stride, int n, const double* wr, const double* wi, int L,
                     double* ore, double* oim) {
    int p = 2;
    while (p * p <= n && n % p) ++p;
    if (n % p) p = n;
    const int sc = L / n;
    if (p == n) {
        for (int k = 0; k < n; ++k) {
            double sr = 0.0, si = 0.0;
            int e = 0;                                   // k j mod n
            for (int j = 0; j < n; ++j) {
                const double xr = re[(size_t)j * stride], xi = im[(size_t)j * stride];
                sr += xr * wr[e * sc] - xi * wi[e * sc];
                si += xr * wi[e * sc] + xi * wr[e * sc];
                e += k;
                if (e >= n) e -= n;
            }
            ore[k] = sr;
            oim[k] = si;
        }
        return;
    }
    const int m = n / p;
    std::vector<double> sr((size_t)p * m), si((size_t)p * m);
    for (int r = 0; r < p; ++r)
        dft_plus(re + (size_t)r * stride, im + (size_t)r * stride, stride * p, m, wr, wi, L, &sr[(size_t)r * m], &si[(size_t)r * m]);
    int km = 0;                                          // k mod m
    for (int k = 0; k < n; ++k) {
        double tr = 0.0, ti = 0.0;
        int e = 0;                                       // r k mod n
        for (int r = 0; r < p; ++r) {
            const double xr = sr[(size_t)r * m + km], xi = si[(size_t)r * m + km];
            tr += xr * wr[e * sc] - xi * wi[e * sc];
            ti += xr * wi[e * sc] + xi * wr[e * sc];
            e += k;
            if (e >= n) e -= n;
        }
        ore[k] = tr;
        oim[k] = ti;
        if (++km == m) km = 0;
    }
}

// Bytes of one tensor-core contraction table: the B operand [np][2M] as bfloat16 hi and lo, built from the
// complex K-side map A_n[k] (rows n < G: [Re A_n | -Im A_n], rows G + n: [Im A_n | Re A_n], rows past 2G zero),
// then float2 C[G][M], the second contraction's weights.  A and C are FP64 [G][M] (real and imaginary parts
// apart).  B is stored chunk by chunk, as the kernel streams it: chunk c (K rows 16 c .. 16 c + 15) holds
// [hi plane][lo plane], each [np][32] in the canonical K-major layout with K = 32 (the 16 rows' real-part
// columns, then their imaginary-part columns), so one chunk is 128 np contiguous bytes.
static void pack_tc_table(int m, int G, int np, const std::vector<double>& ar, const std::vector<double>& ai,
                          const std::vector<double>& cr, const std::vector<double>& ci, std::vector<unsigned char>* out) {
    const size_t plane_el = (size_t)np * 32;            // one plane of one chunk, in bf16 elements
    std::vector<uint16_t> b((size_t)(m / 16) * 2 * plane_el, 0);
    auto put = [&](int row, int k, double v) {
        const int kr = k % m, c = kr / 16, kk = (k >= m ? 16 : 0) + kr % 16;
        const uint16_t h = bf16_bits((float)v);
        const size_t off = (size_t)c * 2 * plane_el + (size_t)umma_offset(row, kk, 32);
        b[off] = h;
        b[off + plane_el] = bf16_bits((float)(v - (double)bf16_value(h)));
    };
    for (int n = 0; n < G; ++n)
        for (int q = 0; q < m; ++q) {
            const double re = ar[(size_t)n * m + q], im = ai[(size_t)n * m + q];
            put(n, q, re);
            put(n, m + q, -im);
            put(G + n, q, im);
            put(G + n, m + q, re);
        }
    const size_t bbytes = b.size() * 2;
    out->resize(bbytes + (size_t)G * m * 8);
    std::memcpy(out->data(), b.data(), bbytes);
    float* x = reinterpret_cast<float*>(out->data() + bbytes);
    for (size_t k = 0; k < (size_t)G * m; ++k) {
        x[2 * k] = (float)cr[k];
        x[2 * k + 1] = (float)ci[k];
    }
}

// Limits of the contraction tables: 2G <= 48 output columns, M a multiple of 16 and at most 384.
static bool tc_table_fits(int m, int G) { return G > 0 && 2 * G <= 48 && m <= 384 && m % 16 == 0; }

// The y map and the x weights of the regrouped sums, FP64 [G][M]:
//   Y_n[q] = sum_j u_n(y'_j) dy' corr_y[j] exp(+2 pi i q j / M),   X_m[i] = u_m(x'_i) dx' corr_x[i].
static void coef_maps(const Settings& s, const Geometry& g, int p, const std::vector<double>& u, std::vector<double>* yr,
                      std::vector<double>* yi, std::vector<double>* xr, std::vector<double>* xi) {
    const int m = g.m, G = g.groups;
    const PolGeom& pg = g.pol[p];
    const double w = g.dx;
    yr->assign((size_t)G * m, 0.0);
    yi->assign((size_t)G * m, 0.0);
    xr->assign((size_t)G * m, 0.0);
    xi->assign((size_t)G * m, 0.0);
    std::vector<double> cxr(m), cxi(m), cyr(m), cyi(m);
    for (int i = 0; i < m; ++i) {
        corr_fp64(s, g, pg, pg.ax[0], 0, i, &cxr[i], &cxi[i]);   // square fields only here
        corr_fp64(s, g, pg, pg.ax[1], 1, i, &cyr[i], &cyi[i]);
    }
    std::vector<double> ar(m), ai(m), wr(m), wi(m);
    for (int e = 0; e < m; ++e) {
        wr[e] = std::cos(2.0 * kPi * e / m);
        wi[e] = std::sin(2.0 * kPi * e / m);
    }
    for (int n = 0; n < G; ++n) {
        for (int j = 0; j < m; ++j) {
            const double uc = u[(size_t)n * m + j] * w;
            ar[j] = uc * cyr[j];
            ai[j] = uc * cyi[j];
            (*xr)[(size_t)n * m + j] = uc * cxr[j];
            (*xi)[(size_t)n * m + j] = uc * cxi[j];
        }
        dft_plus(ar.data(), ai.data(), 1, m, wr.data(), wi.data(), m, &(*yr)[(size_t)n * m], &(*yi)[(size_t)n * m]);
    }
}

// Tables of the coefficient-only tensor-core contraction.  With g[q][i] the x-inverse-transformed window
// rows, the y inverse transform, the y correction and the y overlap weights form one complex map Y_n[q], so
// that c_mn = sum_i X_m[i] sum_q Y_n[q] g[q][i] (the same sums as transform-then-overlap, regrouped; FP64 here).
void build_coef_tc(const Settings& s, const Geometry& g, int p, const std::vector<double>& u, PolTables* ptp) {
    PolTables& pt = *ptp;
    pt.coef_tc.clear();
    pt.coef_np = 0;
    if (!tc_table_fits(g.m, g.groups)) return;
    std::vector<double> yr, yi, xr, xi;
    coef_maps(s, g, p, u, &yr, &yi, &xr, &xi);
    const int np = (2 * g.groups + 15) / 16 * 16;
    pack_tc_table(g.m, g.groups, np, yr, yi, xr, xi, &pt.coef_tc);
    pt.coef_np = np;
}

// Tables of the scoring contraction, which reads the raw box bins B[q][p] (before the mask's zeros, the beam-centre
// phases and the x inverse transform).  With g[q][i] = sum_p B[q][p] phx[p] phy[q] exp(+2 pi i p i / M) over the
// kept bins,
//     c_mn = sum_p Xh_m[p] sum_q Yh_n[q] B[q][p],   Yh_n[q] = phy[q] Y_n[q],
//     Xh_m[p] = phx[p] sum_i X_m[i] exp(+2 pi i p i / M),
// the same sums once more regrouped: the x inverse transform moves into the x weights (FP64 here).
void build_score_tc(const Settings& s, const Geometry& g, int p, const std::vector<double>& u, PolTables* ptp) {
    PolTables& pt = *ptp;
    pt.score_tc.clear();
    const int m = g.m, G = g.groups;
    if (!tc_table_fits(m, G)) return;
    std::vector<double> yr, yi, xr, xi;
    coef_maps(s, g, p, u, &yr, &yi, &xr, &xi);
    const PolGeom& pg = g.pol[p];
    std::vector<double> pxr(m), pxi(m), pyr(m), pyi(m);
    for (int q = 0; q < m; ++q) {
        phase_fp64(s, pg.ax[0], g.n, q, &pxr[q], &pxi[q]);
        phase_fp64(s, pg.ax[1], g.n, q, &pyr[q], &pyi[q]);
    }
    std::vector<double> wr(m), wi(m), hr(m), hi(m);
    for (int e = 0; e < m; ++e) {
        wr[e] = std::cos(2.0 * kPi * e / m);
        wi[e] = std::sin(2.0 * kPi * e / m);
    }
    for (int n = 0; n < G; ++n) {
        double* ry = &yr[(size_t)n * m];
        double* iy = &yi[(size_t)n * m];
        for (int q = 0; q < m; ++q) {
            const double a = ry[q], b = iy[q];
            ry[q] = a * pyr[q] - b * pyi[q];
            iy[q] = a * pyi[q] + b * pyr[q];
        }
        dft_plus(&xr[(size_t)n * m], &xi[(size_t)n * m], 1, m, wr.data(), wi.data(), m, hr.data(), hi.data());
        for (int q = 0; q < m; ++q) {
            xr[(size_t)n * m + q] = hr[q] * pxr[q] - hi[q] * pxi[q];
            xi[(size_t)n * m + q] = hr[q] * pxi[q] + hi[q] * pxr[q];
        }
    }
    pack_tc_table(m, G, (2 * G + 15) / 16 * 16, yr, yi, xr, xi, &pt.score_tc);
}

// Table block of the column-pruned fused kernel (layout in fused_pr.hpp), or empty when the geometry is not
// one it serves (N = 128, M = 64, G <= 16, at most kPrMaxK kept columns, each with a contiguous row range).
// Every value derives from the tables above, in FP64: the kept bins are exactly those of the row-wise mask.
void build_pr_block(const Geometry& g, int p, PolTables* ptp) {
    using L = dhk::PrLayout;
    PolTables& pt = *ptp;
    pt.pr.clear();
    const int n = g.n, m = g.m, G = g.groups;
    if (n != dhk::kPrN || m != dhk::kPrM || G > dhk::kPrG) return;
    const PolGeom& pg = g.pol[p];
    const int klx = pg.ax[0].klo, kly = pg.ax[1].klo;
    // columns p of the box with at least one kept bin, and each column's kept rows
    int plo = m, phi = -1;
    for (int q = 0; q < m; ++q)
        if (pt.mask_lo[q] <= pt.mask_hi[q]) { plo = std::min(plo, pt.mask_lo[q]); phi = std::max(phi, pt.mask_hi[q]); }
    if (phi < plo) return;
    const int nk = phi - plo + 1;
    if (nk > dhk::kPrMaxK) return;
    std::vector<int> qlo(nk, m), qhi(nk, -1);
    for (int c = 0; c < nk; ++c) {
        const int pp = plo + c;
        for (int q = 0; q < m; ++q)
            if (pt.mask_lo[q] <= pp && pp <= pt.mask_hi[q]) { qlo[c] = std::min(qlo[c], q); qhi[c] = std::max(qhi[c], q); }
        for (int q = qlo[c]; q <= qhi[c]; ++q)   // the kernel keeps a contiguous row range per column
            if (!(pt.mask_lo[q] <= pp && pp <= pt.mask_hi[q])) return;
        if (qhi[c] < qlo[c]) { qlo[c] = 1; qhi[c] = 0; }
    }
    const int kxlo = klx + plo;
    std::vector<unsigned char> blk(L::BYTES, 0);
    auto i32 = [&](int off) { return reinterpret_cast<int*>(blk.data() + off); };
    auto f32 = [&](int off) { return reinterpret_cast<float*>(blk.data() + off); };
    i32(L::HDR)[0] = nk;
    i32(L::HDR)[1] = kxlo;
    i32(L::HDR)[2] = klx;
    i32(L::HDR)[3] = kly;
    for (int c = 0; c < nk; ++c) {
        i32(L::QLIM)[2 * c] = qlo[c];
        i32(L::QLIM)[2 * c + 1] = qhi[c];
        // the 1/2 of separating the two real rows packed in one complex row (a power of two: exact)
        f32(L::PHX)[2 * c] = 0.5f * pt.phase_x[2 * (plo + c)];
        f32(L::PHX)[2 * c + 1] = 0.5f * pt.phase_x[2 * (plo + c) + 1];
    }
    for (int q = 0; q < 2 * m; ++q) {
        f32(L::PHY)[q] = pt.phase_y[q];
        f32(L::CY)[q] = pt.corr_y[q];
        f32(L::CX)[q] = pt.corr_x[q];
    }
    for (int k = 0; k < n; ++k) {
        f32(L::TWN)[2 * k] = (float)std::cos(-2.0 * kPi * k / n);
        f32(L::TWN)[2 * k + 1] = (float)std::sin(-2.0 * kPi * k / n);
    }
    for (int j = 0; j < m; ++j)
        for (int nn = 0; nn < G; ++nn) f32(L::HGY)[j * 20 + nn] = pt.hg_y[(size_t)nn * m + j];
    // V[mm][c] = phx[c] sum_i u_mm(x'_i) dx' corr_x[i] exp(+2 pi i p_c i / M), p_c = plo + c the box column:
    // the x inverse transform, the x correction and the x contraction of column c in one complex weight
    for (int mm = 0; mm < G; ++mm)
        for (int c = 0; c < nk; ++c) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < m; ++i) {
                const double ang = 2.0 * kPi * (double)((plo + c) * i % m) / m;
                const double u = pt.hg_x[(size_t)mm * m + i];
                const double cr = pt.corr_x[2 * i], ci = pt.corr_x[2 * i + 1];
                const double wr = std::cos(ang), wi = std::sin(ang);
                re += u * (cr * wr - ci * wi);
                im += u * (cr * wi + ci * wr);
            }
            const double pr = 0.5 * pt.phase_x[2 * (plo + c)], pi = 0.5 * pt.phase_x[2 * (plo + c) + 1];
            f32(L::V)[2 * (mm * dhk::kPrMaxK + c)] = (float)(re * pr - im * pi);
            f32(L::V)[2 * (mm * dhk::kPrMaxK + c) + 1] = (float)(re * pi + im * pr);
        }
    pt.pr.swap(blk);
}

}  // namespace dh
