"""FP64 CPU oracle for digHolo's off-axis reconstruction path.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` may use it.  It shares no
code with the CUDA path: it is written from the paper's description of the method (the user guide's
"Background" and "digHolo processing pipeline" sections) and computes every step as its plain definition,
in float64 / complex128, with numpy matrix products as the only library primitive:

1. window cut around the beam centre (pipeline step 1, digHoloConfigSetBeamCentre);
2. the window's spectrum F(k) = sum_n I_n exp(-2 pi i k x_n / (N px)) evaluated directly on the bins of the
   selected box (pipeline step 1, the FFT; explicit DFT matrices, no fast transform);
3. the circular Fourier window of radius w_c around the reference tilt (pipeline step 2,
   digHoloConfigSetFourierWindowRadius, digHoloConfigSetTilt);
4. the reduced-size inverse transform with the residual tilt and the defocus removed
   (pipeline step 2, digHoloConfigSetIFFTResolutionMode, digHoloProcessRemoveTilt, digHoloConfigSetDefocus);
5. the Hermite-Gaussian basis by its three-term recurrence and the overlap sums
   (pipeline step 3, digHoloConfigSetBasisGroupCount, digHoloConfigSetBasisWaist); Laguerre-Gaussian
   overlaps by direct sums with LG modes from Laguerre polynomials, and custom bases as a matrix applied to
   the HG overlaps (digHoloConfigSetBasisType*);
6. total captured power per alignment candidate (the quantity the AutoAlign search scores);
7. batch averaging (digHoloSetBatchAvg, "Averaging modes"): the windows of the frames of one averaging
   group, rotated into phase with the group's first frame, averaged, then inverse transformed once;
8. reference-wave calibration (digHoloConfigSetRefCalibrationIntensity): the frame divided pixel by pixel by
   the reference's relative amplitude sqrt(cal / max cal) before the transform;
9. the transfer-matrix metrics of the AutoAlign section (DIGHOLO_METRIC_IL ... SNRMG, digHoloAutoAlignCalcMetrics)
   and the fine-alignment search that maximises the captured power (digHoloAutoAlign's tweak stage).

Conventions the paper leaves open (the same readings are used by the CUDA library):

* x is the fast axis; window pixel n of polarisation p sits at x_n = (o + n) px - c with
  o = round_half_away(c / px) - N/2 and c the beam centre in metres;
* angles map to bins linearly: kappa = theta_rad N px / lambda, r = w_c,rad N px / lambda;
* the box is M x M bins starting at k0 - M/2 with k0 = round_half_away(kappa); a bin is kept when it lies
  inside the circle ((k - kappa)/r)^2 summed over both axes <= 1 and inside the real-to-complex half plane
  0 <= k_x <= N/2; everything else is zero;
* the field is sampled at x'_i = (i - M/2) N px / M relative to the beam centre and equals
      E(x'_i, y'_j) = 1/(Nx Ny) sum_q F(k0 + q) exp(+2 pi i q.x'/(N px))
                       * exp(-2 pi i (kappa - k0).x'/(N px)) * exp(-i pi D |x'|^2 / lambda),
  i.e. the reference's own tilt and defocus phase multiply the inverse transform, which returns
  A_R * S for a band-limited signal;
* M defaults to the paper's size rule M = 16 ceil(2 r / 16) (the FFT [IFFT] table of the Benchmarks
  section);
* u_n(x) = (sqrt(2)/w)^(1/2) psi_n(sqrt(2) x / w) with psi_0 = pi^(-1/4) exp(-xi^2/2),
  psi_{n+1} = sqrt(2/(n+1)) xi psi_n - sqrt(n/(n+1)) psi_{n-1}; modes (m, n) with m + n < G ordered by group
  then m ascending; c_mn = dx' dy' sum_ij u_m(x'_i) u_n(y'_j) E_ji (the basis is real).

Every function below is pinned by ``tests/test_oracle_pins.py`` against values the paper prints, closed
forms, library special cases or brute force.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------------------------------
# Geometry rules (Background: "How do you choose the angle of the Reference Field?")
# ---------------------------------------------------------------------------------------------------


def w_max_rad(wavelength: float, pixel: float) -> float:
    """Largest resolvable angle lambda / (2 px), radians (Background, worked example)."""
    return wavelength / (2.0 * pixel)


def window_radius_fraction() -> float:
    """Largest non-overlapping window radius as a fraction of w_max: sqrt(2) / (3 + sqrt(2)) (Background)."""
    return math.sqrt(2.0) / (3.0 + math.sqrt(2.0))


def wrap_radius_fraction() -> float:
    """Window fraction when the window may wrap along one axis: positive root of 8 w^2 + 2 w - 2 = 0
    (Background; the printed equation is garbled, the printed root (-2 + sqrt(68)) / 16 fixes it)."""
    a, b, c = 8.0, 2.0, -2.0
    return (-b + math.sqrt(b * b - 4.0 * a * c)) / (2.0 * a)


def rule_tilt(radius: float) -> float:
    """Per-axis reference tilt 3 w_c / sqrt(2) that puts the window beside the autocorrelation term."""
    return 3.0 * radius / math.sqrt(2.0)


def ifft_size_rule(r_bins: float) -> int:
    """Reduced inverse-transform size: the window diameter rounded up to a multiple of 16 pixels
    (the FFT [IFFT] size table of the Benchmarks section: 64[32], 128[48], 256[96], 512[176], 1024[336])."""
    return int(16 * math.ceil(2.0 * r_bins / 16.0))


def round_half_away(v: float) -> int:
    """Nearest integer, halves rounded away from zero."""
    return int(math.copysign(math.floor(abs(v) + 0.5), v))


@dataclass
class AxisGeometry:
    n: int            # FFT window length N along this axis
    origin: int       # frame index of window pixel 0
    centre: float     # beam centre, metres
    kappa: float      # reference tilt, bins
    k0: int           # box centre bin
    m: int            # box / field length M
    dx: float         # field sample pitch N px / M, metres

    @property
    def klo(self) -> int:
        return self.k0 - self.m // 2

    def pixel_positions(self, pixel: float) -> np.ndarray:
        """x_n = (o + n) px - c for the window pixels."""
        return (self.origin + np.arange(self.n)) * pixel - self.centre

    def field_positions(self) -> np.ndarray:
        """x'_i = (i - M/2) dx'."""
        return (np.arange(self.m) - self.m // 2) * self.dx


@dataclass
class PolGeometry:
    x: AxisGeometry
    y: AxisGeometry
    r_x: float        # window radius, bins along x
    r_y: float        # window radius, bins along y
    defocus: float    # dioptre
    waist: float      # metres
    groups: int
    pixel: float
    wavelength: float
    fill_factor: bool = False   # divide the window by the 100 %-fill-factor pixel response


def _per_axis(v) -> Tuple[int, int]:
    """A size given once for both axes, or as (x, y)."""
    return (int(v), int(v)) if np.isscalar(v) else (int(v[0]), int(v[1]))


def pol_geometry(setup, p: int, tilt_deg=None, defocus=None, waist=None) -> PolGeometry:
    """Per-polarisation geometry from the acquisition settings (Alignment: beam centre, tilt, defocus;
    Window sizes: FFT window and IFFT resolution mode 1 per axis, Fourier window radius).  Angles become bins
    with that axis' window length: kappa = theta N px / lambda, r = w_c N px / lambda."""
    px, lam = float(setup.pixel), float(setup.wavelength)
    ns = _per_axis(setup.window)
    ms_req = _per_axis(setup.ifft_size)
    tdeg = setup.tilt_deg[p] if tilt_deg is None else tilt_deg
    dfc = float(setup.defocus[p] if defocus is None else defocus)
    wst = float(setup.waist[p] if waist is None else waist)
    r_rad = math.radians(float(setup.radius_deg))
    ag, rs = [], []
    for ax in range(2):
        n = ns[ax]
        c = float(setup.beam_centre[p][ax])
        origin = round_half_away(c / px) - n // 2
        kappa = math.radians(float(tdeg[ax])) * n * px / lam
        r_bins = r_rad * n * px / lam
        m = ms_req[ax] if ms_req[ax] > 0 else ifft_size_rule(r_bins)
        ag.append(AxisGeometry(n=n, origin=origin, centre=c, kappa=kappa, k0=round_half_away(kappa), m=m,
                               dx=n * px / m))
        rs.append(r_bins)
    return PolGeometry(x=ag[0], y=ag[1], r_x=rs[0], r_y=rs[1], defocus=dfc, waist=wst,
                       groups=int(setup.group_count), pixel=px, wavelength=lam,
                       fill_factor=bool(getattr(setup, "fill_factor", False)))


# ---------------------------------------------------------------------------------------------------
# Pipeline step 1: the window and its spectrum on the selected bins
# ---------------------------------------------------------------------------------------------------


def reference_calibration_factor(cal) -> np.ndarray:
    """Per-pixel factor that removes a non-uniform reference amplitude: the measured reference intensity
    (uint16 [H][W], or [L][H][W] per wavelength, of which the single wavelength used here is the first) is
    normalised by its maximum over all pixels and frames, and the frame is multiplied by
    sqrt(max / cal) = 1 / (relative reference amplitude), 0 where cal = 0 (no reference light)."""
    c = np.asarray(cal, dtype=np.float64)
    top = float(c.max())
    first = c[0] if c.ndim == 3 else c
    out = np.zeros_like(first)
    lit = first > 0
    out[lit] = np.sqrt(top / first[lit])
    return out


def calibrated(frame: np.ndarray, setup) -> np.ndarray:
    """The frame as the transform sees it: with a reference calibration, divided by the reference's
    relative amplitude; otherwise unchanged."""
    cal = getattr(setup, "ref_cal", None)
    if cal is None:
        return frame
    return np.asarray(frame, dtype=np.float64) * reference_calibration_factor(cal)


def cut_window(frame: np.ndarray, g: PolGeometry) -> np.ndarray:
    """The N_y x N_x window of polarisation p, as float64 (pipeline step 1; uint16 converts exactly)."""
    oy, ox, ny, nx = g.y.origin, g.x.origin, g.y.n, g.x.n
    if oy < 0 or ox < 0 or oy + ny > frame.shape[0] or ox + nx > frame.shape[1]:
        raise ValueError("window outside the frame")
    return np.asarray(frame[oy:oy + ny, ox:ox + nx], dtype=np.float64)


def dft_rows(ax: AxisGeometry, pixel: float, bins: np.ndarray) -> np.ndarray:
    """exp(-2 pi i k x_n / (N px)) for the given integer bins k (rows) and window pixels n (columns)."""
    xn = ax.pixel_positions(pixel)
    return np.exp(-2j * np.pi * np.outer(bins, xn) / (ax.n * pixel))


def box_bins(ax: AxisGeometry) -> np.ndarray:
    """The M integer bins k0 - M/2 ... k0 + M/2 - 1 of the selected box (unwrapped)."""
    return ax.klo + np.arange(ax.m)


def window_spectrum(window: np.ndarray, g: PolGeometry, bins_x=None, bins_y=None) -> np.ndarray:
    """F(k_y, k_x) = sum_{n_y, n_x} I exp(-2 pi i (k_x x_n + k_y y_n) / (N px)) on the box bins, as the
    separable product A_y I A_x^T of explicit DFT matrices (pipeline step 1, the real-to-complex FFT)."""
    bx = box_bins(g.x) if bins_x is None else np.asarray(bins_x)
    by = box_bins(g.y) if bins_y is None else np.asarray(bins_y)
    ax_m = dft_rows(g.x, g.pixel, bx)
    ay_m = dft_rows(g.y, g.pixel, by)
    return ay_m @ window @ ax_m.T


# ---------------------------------------------------------------------------------------------------
# Pipeline step 2: circular Fourier window, reduced inverse transform, tilt and defocus removal
# ---------------------------------------------------------------------------------------------------


def window_mask(g: PolGeometry) -> np.ndarray:
    """Bins of the box kept by the circular window (radius r around the tilt kappa) and lying in the
    real-to-complex half plane 0 <= k_x <= N/2 (pipeline step 2; digHoloGetFourierPlaneFull's (w/2+1) width)."""
    kx = box_bins(g.x).astype(np.float64)
    ky = box_bins(g.y).astype(np.float64)
    dx = (kx - g.x.kappa) / g.r_x
    dy = (ky - g.y.kappa) / g.r_y
    inside = (dy[:, None] ** 2 + dx[None, :] ** 2) <= 1.0
    half = (kx >= 0) & (kx <= g.x.n // 2)
    return inside & half[None, :]


def pixel_response(ax: AxisGeometry, bins: np.ndarray) -> np.ndarray:
    """Spectral response sinc(k / N) = sin(pi k / N) / (pi k / N) of a pixel that integrates over its full
    width (digHoloConfigSetFillFactorCorrectionEnabled: a 100 % fill factor)."""
    return np.sinc(np.asarray(bins, dtype=np.float64) / ax.n)


def reconstruct_field(f_box: np.ndarray, mask: np.ndarray, g: PolGeometry) -> np.ndarray:
    """E(x'_i, y'_j) by the explicit inverse sum over the kept bins, times the reference's residual
    tilt and defocus phase (pipeline step 2 and digHoloProcessRemoveTilt).  With fill-factor correction the
    kept bins are first divided by the pixel response of both axes (done during the inverse transform in the
    guide)."""
    px, lam = g.pixel, g.wavelength
    if g.fill_factor:
        f_box = f_box / np.outer(pixel_response(g.y, box_bins(g.y)), pixel_response(g.x, box_bins(g.x)))
    out = []
    for ax in (g.x, g.y):
        q = np.arange(ax.m) - ax.m // 2                     # k - k0
        xp = ax.field_positions()
        inv = np.exp(2j * np.pi * np.outer(xp, q) / (ax.n * px))          # [i][q]
        tilt = np.exp(-2j * np.pi * (ax.kappa - ax.k0) * xp / (ax.n * px))
        focus = np.exp(-1j * np.pi * g.defocus * xp ** 2 / lam)
        out.append((inv, tilt * focus))
    (bx, cx), (by, cy) = out
    e = by @ (f_box * mask) @ bx.T / (g.x.n * g.y.n)
    return e * cy[:, None] * cx[None, :]


# ---------------------------------------------------------------------------------------------------
# Pipeline step 3: Hermite-Gaussian modal decomposition
# ---------------------------------------------------------------------------------------------------


def hg_1d(n_max: int, x: np.ndarray, waist: float) -> np.ndarray:
    """u_0 .. u_{n_max-1} at positions x by the three-term recurrence (Modal decomposition:
    Hermite-Gaussian modes of the given waist, stored separably in x and y)."""
    x = np.asarray(x, dtype=np.float64)
    xi = math.sqrt(2.0) * x / waist
    psi = np.zeros((max(n_max, 1),) + x.shape)
    psi[0] = math.pi ** -0.25 * np.exp(-xi ** 2 / 2.0)
    if n_max > 1:
        psi[1] = math.sqrt(2.0) * xi * psi[0]
    for n in range(1, n_max - 1):
        psi[n + 1] = math.sqrt(2.0 / (n + 1)) * xi * psi[n] - math.sqrt(n / (n + 1.0)) * psi[n - 1]
    return math.sqrt(math.sqrt(2.0) / waist) * psi[:n_max]


def mode_list(groups: int) -> List[Tuple[int, int]]:
    """HG(m, n) with m + n < groups, by group g = m + n then m ascending (digHoloConfigSetBasisGroupCount)."""
    return [(m, g - m) for g in range(groups) for m in range(g + 1)]


def overlap(e: np.ndarray, g: PolGeometry) -> np.ndarray:
    """c_mn = dx' dy' sum_{j,i} u_m(x'_i) u_n(y'_j) E(x'_i, y'_j) for every mode (pipeline step 3)."""
    if g.groups <= 0:
        return np.zeros(0, dtype=np.complex128)
    ux = hg_1d(g.groups, g.x.field_positions(), g.waist)    # [G][Mx]
    uy = hg_1d(g.groups, g.y.field_positions(), g.waist)    # [G][My]
    full = uy @ e @ ux.T * (g.x.dx * g.y.dx)                  # [n][m]
    return np.array([full[n, m] for (m, n) in mode_list(g.groups)])


def lg_mode_list(groups: int) -> List[Tuple[int, int]]:
    """Laguerre-Gaussian (p, l) with mode group N = 2p + |l| < groups, ordered by group, then l ascending
    (-N, -N+2, ..., N); the same count per group as the HG basis (digHoloConfigSetBasisTypeLG)."""
    out = []
    for n_grp in range(groups):
        for l in range(-n_grp, n_grp + 1, 2):
            out.append(((n_grp - abs(l)) // 2, l))
    return out


def lg_2d(p: int, l: int, x: np.ndarray, y: np.ndarray, waist: float) -> np.ndarray:
    """LG_p^l(x, y) = sqrt(2 p! / (pi (p+|l|)!)) / w (sqrt(2) r / w)^|l| L_p^|l|(2 r^2 / w^2) exp(-r^2/w^2)
    exp(i l phi), L the generalised Laguerre polynomial (scipy.special.eval_genlaguerre), L2-normalised;
    returned as [len(y)][len(x)]."""
    from scipy.special import eval_genlaguerre
    X, Y = np.meshgrid(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    r2 = X * X + Y * Y
    c = math.sqrt(2.0 * math.factorial(p) / (math.pi * math.factorial(p + abs(l)))) / waist
    radial = (2.0 * r2 / waist ** 2) ** (abs(l) / 2.0) * eval_genlaguerre(p, abs(l), 2.0 * r2 / waist ** 2)
    return c * radial * np.exp(-r2 / waist ** 2) * np.exp(1j * l * np.arctan2(Y, X))


def overlap_lg(e: np.ndarray, g: PolGeometry) -> np.ndarray:
    """c_pl = dx' dy' sum_ij conj(LG_p^l(x'_i, y'_j)) E(x'_i, y'_j) by direct sums over the field grid."""
    xp, yp = output_axes(g)
    return np.array([np.sum(np.conj(lg_2d(p, l, xp, yp, g.waist)) * e) * g.x.dx * g.y.dx
                     for (p, l) in lg_mode_list(g.groups)])


def basis_coefficients(e: np.ndarray, g: PolGeometry, basis: str = "hg", transform=None) -> np.ndarray:
    """Coefficients in the chosen basis: HG overlaps, LG overlaps, or a custom matrix applied to the HG
    overlaps (digHoloConfigSetBasisTypeCustom: transform is [modes_out][modes_in], columns beyond the HG mode
    count are unused)."""
    if basis == "hg":
        return overlap(e, g)
    if basis == "lg":
        return overlap_lg(e, g)
    c = overlap(e, g)
    t = np.asarray(transform, dtype=np.complex128)
    k = min(t.shape[1], c.shape[0])
    return t[:, :k] @ c[:k]


# ---------------------------------------------------------------------------------------------------
# Whole path
# ---------------------------------------------------------------------------------------------------


def process_window(frame: np.ndarray, g: PolGeometry):
    """Steps 1-3 for one polarisation of one frame: returns (F_box, mask, field, coefficients)."""
    win = cut_window(frame, g)
    f_box = window_spectrum(win, g)
    mask = window_mask(g)
    e = reconstruct_field(f_box, mask, g)
    return f_box, mask, e, overlap(e, g)


def process_batch(frames: np.ndarray, setup) -> Tuple[np.ndarray, np.ndarray]:
    """digHoloProcessBatch: fields [B][P][M_y][M_x] and coefficients [B][P][modes] (pol-blocked, as
    digHoloBasisGetCoefs lays them out), in the setup's basis (attribute basis: "hg" default, "lg", or
    "custom" with attribute basis_transform)."""
    geos = [pol_geometry(setup, p) for p in range(setup.pol_count)]
    mx, my = geos[0].x.m, geos[0].y.m
    basis = getattr(setup, "basis", "hg")
    transform = getattr(setup, "basis_transform", None)
    modes = np.asarray(transform).shape[0] if basis == "custom" else len(mode_list(geos[0].groups))
    B = frames.shape[0]
    fields = np.empty((B, setup.pol_count, my, mx), dtype=np.complex128)
    coefs = np.empty((B, setup.pol_count, modes), dtype=np.complex128)
    for b in range(B):
        frame = calibrated(frames[b], setup)
        for p, g in enumerate(geos):
            _, _, e, c = process_window(frame, g)
            fields[b, p] = e
            coefs[b, p] = c if basis == "hg" else basis_coefficients(e, g, basis, transform)
    return fields, coefs


# ---------------------------------------------------------------------------------------------------
# Batch averaging (digHoloSetBatchAvg, digHoloConfigSetBatchAvgCount, "Averaging modes")
# ---------------------------------------------------------------------------------------------------


def avg_member_index(group: int, member: int, batch: int, avg_count: int, avg_mode: int) -> int:
    """Frame index of member j of averaging group g: sequential blocks [A A A B B B] (mode 0, and mode 2,
    which equals mode 0 with a single wavelength) at g avg_count + j, interlaced [A B A B] (mode 1) at
    j batch + g."""
    if avg_mode == 1:
        return member * batch + group
    return group * avg_count + member


def align_phases(windows) -> np.ndarray:
    """Unit phasors a_j that bring the windows of one group in phase with its first member: with
    <W_0, W_j> = sum over polarisations and bins of conj(W_0) W_j, a_j = conj(<W_0, W_j>) / |<W_0, W_j>|
    (1 when the inner product vanishes), so that arg <W_0, a_j W_j> = 0.  windows: [A][P][...]."""
    out = np.ones(len(windows), dtype=np.complex128)
    for j in range(len(windows)):
        d = sum(np.vdot(windows[0][p], windows[j][p]) for p in range(len(windows[0])))
        if d != 0:
            out[j] = np.conj(d) / abs(d)
    return out


def process_batch_avg(frames: np.ndarray, setup, avg_count: int, avg_mode: int = 0):
    """Averaged reconstruction of batch = len(frames) / avg_count fields: per group, every member's kept
    window (after the fill-factor correction when enabled, i.e. the spectrum that is inverse transformed)
    is phase-aligned with the first member's by align_phases, the aligned windows are averaged, and the
    average is inverse transformed and decomposed once.  Returns fields [batch][P][M_y][M_x] and coefficients
    [batch][P][modes] in the setup's basis."""
    geos = [pol_geometry(setup, p) for p in range(setup.pol_count)]
    A = max(int(avg_count), 1)
    B = frames.shape[0] // A
    mx, my = geos[0].x.m, geos[0].y.m
    basis = getattr(setup, "basis", "hg")
    transform = getattr(setup, "basis_transform", None)
    modes = np.asarray(transform).shape[0] if basis == "custom" else len(mode_list(geos[0].groups))
    fields = np.empty((B, setup.pol_count, my, mx), dtype=np.complex128)
    coefs = np.empty((B, setup.pol_count, modes), dtype=np.complex128)
    masks = [window_mask(g) for g in geos]
    corr = []
    for g in geos:
        if g.fill_factor:
            corr.append(1.0 / np.outer(pixel_response(g.y, box_bins(g.y)), pixel_response(g.x, box_bins(g.x))))
        else:
            corr.append(np.ones((my, mx)))
    for b in range(B):
        boxes = []
        for j in range(A):
            fr = calibrated(frames[avg_member_index(b, j, B, A, avg_mode)], setup)
            boxes.append([window_spectrum(cut_window(fr, g), g) * masks[p] for p, g in enumerate(geos)])
        a = align_phases([[boxes[j][p] * corr[p] for p in range(len(geos))] for j in range(A)])
        for p, g in enumerate(geos):
            avg = sum(a[j] * boxes[j][p] for j in range(A)) / A
            e = reconstruct_field(avg, masks[p], g)
            fields[b, p] = e
            coefs[b, p] = overlap(e, g) if basis == "hg" else basis_coefficients(e, g, basis, transform)
    return fields, coefs


def score_settings(frames: np.ndarray, setup, tilt_deg: np.ndarray, defocus: np.ndarray,
                   waist: np.ndarray) -> np.ndarray:
    """Total captured power P[b][s] = sum_p sum_modes |c_{b,p,s}|^2 for every alignment candidate s,
    each candidate re-running window selection, inverse transform, correction and overlap with its own
    tilt, defocus and waist (the inner loop of the AutoAlign search)."""
    B, S = frames.shape[0], tilt_deg.shape[0]
    power = np.zeros((B, S))
    for b in range(B):
        frame = calibrated(frames[b], setup)
        for s in range(S):
            tot = 0.0
            for p in range(setup.pol_count):
                g = pol_geometry(setup, p, tilt_deg=tilt_deg[s, p], defocus=defocus[s, p], waist=waist[s, p])
                win = cut_window(frame, g)
                e = reconstruct_field(window_spectrum(win, g), window_mask(g), g)
                c = overlap(e, g)
                tot += float(np.sum(np.abs(c) ** 2))
            power[b, s] = tot
    return power


# ---------------------------------------------------------------------------------------------------
# Transfer-matrix metrics and the fine-alignment search (AutoAlign section)
# ---------------------------------------------------------------------------------------------------

METRICS = ("IL", "MDL", "DIAG", "SNRAVG", "DIAGBEST", "DIAGWORST", "SNRBEST", "SNRWORST", "SNRMG")


def _db(v: float) -> float:
    """10 log10(v) with the IEEE limits: -inf for 0, +inf for +inf."""
    with np.errstate(divide="ignore"):
        return float(10.0 * np.log10(v))


def _ratio(num: float, den: float) -> float:
    return math.inf if den == 0.0 else num / den


def transfer_metrics(coefs: np.ndarray, groups=None, mul_conj_trans: bool = False) -> dict:
    """The AutoAlign metrics of a batch of coefficient vectors (the transfer matrix A: row b = batch element b,
    column k = coefficient k of all polarisations, [B][P][modes] flattened to [B][P modes]), all in dB:

    IL        mean of the eigenvalues of the Gram matrix of A (its squared singular values; the smaller of
              A A^H and A^H A)                                             (insertion loss)
    MDL       largest over smallest of those eigenvalues                   (mode dependent loss; eigenvalues
              below 1e-12 of the largest count as zero, giving +inf)
    DIAG      total power on the diagonal, sum_i |X_ii|^2
    SNRAVG    diagonal power over off-diagonal power
    DIAGBEST / DIAGWORST   largest / smallest diagonal element power
    SNRBEST / SNRWORST     largest / smallest row ratio |X_ii|^2 / sum_{j != i} |X_ij|^2
    SNRMG     as SNRAVG, with every coupling inside one mode group of one polarisation counted as signal;
              NaN-free only for group-ordered bases: groups = G, modes per polarisation G (G + 1) / 2, row i and
              column i describing the same mode (pol-blocked)

    X is A, or A A^H with mul_conj_trans (digHoloConfigSetAutoAlignBasisMulConjTrans).  The diagonal has
    min(rows, columns) elements; rows without one count in the totals only.  SNRMG is None (not calculated)
    without a group structure."""
    c = np.asarray(coefs, dtype=np.complex128)
    B = c.shape[0]
    P = c.shape[1]
    modes = c.shape[2]
    A = c.reshape(B, P * modes)
    gram = A @ A.conj().T if B <= P * modes else A.conj().T @ A
    # eigenvalues of a Gram matrix are >= 0; rounding can leave the zero ones of a rank-deficient matrix at a
    # relative size near the FP64 epsilon, which counts as zero (MDL infinite)
    lam = np.linalg.eigvalsh(gram)
    lam = np.where(lam <= 1e-12 * max(float(lam.max()), 0.0), 0.0, lam)
    out = {"IL": _db(float(lam.sum()) / lam.size), "MDL": _db(_ratio(float(lam.max()), float(lam.min())))}
    X = A @ A.conj().T if mul_conj_trans else A
    pw = np.abs(X) ** 2
    r, k = pw.shape
    nd = min(r, k)
    d = np.array([pw[i, i] for i in range(nd)])
    t = pw.sum(axis=1)
    out["DIAG"] = _db(float(d.sum()))
    out["SNRAVG"] = _db(_ratio(float(d.sum()), float(t.sum() - d.sum())))
    out["DIAGBEST"] = _db(float(d.max()))
    out["DIAGWORST"] = _db(float(d.min()))
    snr = [_ratio(float(d[i]), float(t[i] - d[i])) for i in range(nd)]
    out["SNRBEST"] = _db(max(snr))
    out["SNRWORST"] = _db(min(snr))
    if groups is not None and modes == groups * (groups + 1) // 2:
        grp = np.array([g for g in range(groups) for _ in range(g + 1)])
        def key(i):
            return (i // modes, grp[i % modes])
        sig = sum(pw[i, j] for i in range(r) for j in range(k) if key(i) == key(j))
        out["SNRMG"] = _db(_ratio(float(sig), float(t.sum() - sig)))
    else:
        out["SNRMG"] = None
    return out


def search_candidates(tilt: np.ndarray, defocus: np.ndarray, waist: np.ndarray, steps: np.ndarray):
    """The compass stencil of the fine-alignment search around the current settings: the centre, then for each
    polarisation p and parameter (tilt x, tilt y, defocus, waist) the settings with that parameter moved by
    -step and +step (waist steps are relative: w (1 -/+ step)).  Returns (tilt [S][P][2], defocus [S][P],
    waist [S][P]) with S = 1 + 8 P."""
    P = tilt.shape[0]
    T, D, W = [tilt.copy()], [defocus.copy()], [waist.copy()]
    for p in range(P):
        for par in range(4):
            for sgn in (-1.0, 1.0):
                t, dd, w = tilt.copy(), defocus.copy(), waist.copy()
                if par < 2:
                    t[p, par] += sgn * steps[0]
                elif par == 2:
                    dd[p] += sgn * steps[1]
                else:
                    w[p] *= 1.0 + sgn * steps[2]
                T.append(t)
                D.append(dd)
                W.append(w)
    return np.array(T), np.array(D), np.array(W)


def auto_align_tweak(frames: np.ndarray, setup, steps=(0.02, 0.1, 0.05), min_steps=(2e-4, 1e-3, 5e-4),
                     max_iter: int = 40):
    """Fine-alignment search (the tweak stage of digHoloAutoAlign, goal: captured power, i.e. insertion loss):
    a compass search that scores the stencil of search_candidates with score_settings, moves to the stencil
    point of largest total power sum_b P[b][s] when it beats the centre, and otherwise halves every step;
    it stops when all steps are below min_steps or after max_iter scorings.  Ties go to the lowest stencil index.
    steps / min_steps: (tilt degrees, defocus dioptre, relative waist).  Returns (tilt [P][2], defocus [P],
    waist [P], total power, scorings)."""
    P = setup.pol_count
    tilt = np.array(setup.tilt_deg, dtype=np.float64).reshape(P, 2)
    defocus = np.array(setup.defocus, dtype=np.float64).reshape(P)
    waist = np.array(setup.waist, dtype=np.float64).reshape(P)
    st = np.array(steps, dtype=np.float64)
    lo = np.array(min_steps, dtype=np.float64)
    best = None
    it = 0
    while it < max_iter and np.any(st >= lo):
        T, D, W = search_candidates(tilt, defocus, waist, st)
        power = score_settings(frames, setup, T, D, W).sum(axis=0)
        it += 1
        k = int(np.argmax(power))
        best = float(power[0])
        if power[k] > power[0]:
            tilt, defocus, waist, best = T[k], D[k], W[k], float(power[k])
        else:
            st = st / 2.0
    return tilt, defocus, waist, best, it


def output_axes(g: PolGeometry) -> Tuple[np.ndarray, np.ndarray]:
    """x and y axes of the reconstructed field, metres from the beam centre (digHoloGetFields)."""
    return g.x.field_positions(), g.y.field_positions()


def validate(g: PolGeometry) -> None:
    """Reject geometries whose circle centre leaves the real-to-complex half plane or whose box is
    larger than the window (the library returns an invalid-argument code for these)."""
    if not (0.0 < g.x.kappa <= g.x.n / 2.0):
        raise ValueError("tilt x outside the half plane")
    if g.x.m > g.x.n or g.y.m > g.y.n or g.x.m % 16 or g.y.m % 16:
        raise ValueError("bad field size")
    if g.r_x <= 0.0:
        raise ValueError("window radius must be positive")


def geometries(setup) -> Sequence[PolGeometry]:
    return [pol_geometry(setup, p) for p in range(setup.pol_count)]
