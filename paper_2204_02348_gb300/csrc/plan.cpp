// Host-side geometry and tables.  Compiled with -ffp-contract=off so every FP64 expression rounds exactly
// as written; the window-mask decision (a floating-point comparison that decides which bins are kept) is
// taken here, in FP64, once per plan.
#include "plan.hpp"

#include "fused_pr.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

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
    a->origin = rc - s.n / 2;
    a->eps = (double)rc - c / s.pixel;
    a->kappa = tilt_deg * kDegToRad * (double)s.n * s.pixel / s.wavelength;
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
    g->pols = s.pols;
    g->groups = s.groups;
    g->modes = s.groups * (s.groups + 1) / 2;
    g->basis = s.basis == DH_BASIS_CUSTOM && s.custom.empty() ? DH_BASIS_HG : s.basis;
    g->modes_out = g->modes == 0 ? 0 : g->basis == DH_BASIS_CUSTOM ? s.custom_out : g->modes;
    const double r = s.radius_deg * kDegToRad * (double)s.n * s.pixel / s.wavelength;
    g->m = s.m_req > 0 ? s.m_req : ifft_size_rule(r);
    if (g->m < 16 || g->m % 16 || g->m > s.n || g->m > DH_MAX_FIELD || radix_plan(g->m).empty()) {
        char b[160];
        std::snprintf(b, sizeof b, "field size M=%d invalid for window N=%d (multiple of 16, <= N, <= %d, odd part 19-smooth)",
                      g->m, s.n, DH_MAX_FIELD);
        *why = b;
        return DH_ERROR_INVALIDARGUMENT;
    }
    if (s.cal_on && (s.cal_w != s.width || s.cal_h != s.height)) {
        char b[160];
        std::snprintf(b, sizeof b, "reference calibration is %d x %d, frames are %d x %d", s.cal_w, s.cal_h, s.width,
                      s.height);
        *why = b;
        return DH_ERROR_INVALIDDIMENSION;
    }
    g->dx = (double)s.n * s.pixel / (double)g->m;
    for (int p = 0; p < s.pols; ++p) {
        PolGeom& pg = g->pol[p];
        for (int ax = 0; ax < 2; ++ax) axis_geometry(s, p, ax, tilt[p][ax], &pg.ax[ax]);
        pg.r = r;
        pg.defocus = defocus[p];
        pg.waist = waist[p];
        for (int ax = 0; ax < 2; ++ax) pg.ax[ax].klo = pg.ax[ax].k0 - g->m / 2;
        const int lim[2] = {s.width, s.height};
        for (int ax = 0; ax < 2; ++ax) {
            if (pg.ax[ax].origin < 0 || pg.ax[ax].origin + s.n > lim[ax]) {
                char b[160];
                std::snprintf(b, sizeof b, "window of polarisation %d leaves the frame along axis %d (origin %d, N %d, frame %d)",
                              p, ax, pg.ax[ax].origin, s.n, lim[ax]);
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

void build_tables(const Settings& s, const Geometry& g, Tables* t) {
    const int n = g.n, m = g.m;
    t->tw_fwd_n.clear();
    t->tw_inv_m.clear();
    for (int k = 0; k < n; ++k) push_c(t->tw_fwd_n, std::cos(-2.0 * kPi * k / n), std::sin(-2.0 * kPi * k / n));
    for (int k = 0; k < m; ++k) push_c(t->tw_inv_m, std::cos(2.0 * kPi * k / m), std::sin(2.0 * kPi * k / m));
    t->radix_n = radix_plan(n);
    t->radix_m = s.radix_m.empty() ? radix_plan(m) : s.radix_m;
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
    std::vector<double> xp(m);
    for (int i = 0; i < m; ++i) xp[i] = (double)(i - m / 2) * g.dx;
    for (int p = 0; p < g.pols; ++p) {
        const PolGeom& pg = g.pol[p];
        PolTables& pt = t->pol[p];
        pt.cal.clear();
        if (s.cal_on) {
            // divide the frame by the reference's relative amplitude sqrt(cal / max cal)
            pt.cal.resize((size_t)n * n);
            for (int y = 0; y < n; ++y)
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
            const double sgn = (a.klo % 2 == 0) ? 1.0 : -1.0;
            for (int q = 0; q < m; ++q) {
                const double ang = -2.0 * kPi * (double)(a.klo + q) * a.eps / n;
                double w = sgn / n;
                if (s.fill_factor) {
                    // 100 % fill factor: divide by the pixel response sinc(k / N) of this axis
                    const double u = kPi * (double)(a.klo + q) / n;
                    w /= (u == 0.0) ? 1.0 : std::sin(u) / u;
                }
                push_c(*ph[ax], w * std::cos(ang), w * std::sin(ang));
            }
            for (int i = 0; i < m; ++i) {
                const double ang = -2.0 * kPi * (a.kappa - a.k0) * (double)(i - m / 2) / m
                                   - kPi * pg.defocus * xp[i] * xp[i] / s.wavelength;
                const double sg = (i % 2 == 0) ? 1.0 : -1.0;
                push_c(*co[ax], sg * std::cos(ang), sg * std::sin(ang));
            }
        }
        // mask rows: the same FP64 expression as the definition, ((ky-kappa_y)/r)^2 + ((kx-kappa_x)/r)^2 <= 1
        pt.mask_lo.assign(m, 1);
        pt.mask_hi.assign(m, 0);
        for (int q = 0; q < m; ++q) {
            const double ky = (double)(pg.ax[1].klo + q);
            const double ddy = (ky - pg.ax[1].kappa) / pg.r;
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
    }
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
