"""Seeded forward model: camera frames |S + A_R R|^2 of Hermite-Gaussian signals (frame simulator).

Conventions (shared *as conventions*, not as code, with the oracle and the CUDA library):

* frames are row-major ``[B][H][W]`` with x the fast axis; pixel (i, j) has its centre at (i*px, j*px);
* polarisation p occupies the p-th vertical strip of the frame (``W/P`` pixels wide), as in the paper's
  two-polarisation layout ("digHolo processing pipeline", step 1: the two components sit on opposite
  halves of the frame width);
* angles map to spatial frequency linearly, f = theta_rad / lambda (the paper's w_max = lambda/(2 px));
* the reference of polarisation p is R = exp(-2 pi i (f_x X + f_y Y)) * exp(-i pi D (X^2 + Y^2) / lambda)
  with X, Y measured from that polarisation's beam centre and D in dioptre, so S R* carries the signal
  to +f in Fourier space;
* the signal is S = sum_{m+n<G} c_mn u_m(X) u_n(Y), modes ordered by group g = m+n, then m ascending;
  u_n is the L2-normalised 1D Hermite-Gaussian of waist w, evaluated here from its closed form with
  physicists' Hermite polynomials (numpy.polynomial.hermite), a different route from the oracle's
  three-term recurrence.

Seeds: every generator takes an integer seed; frame b of a batch draws from
``numpy.random.default_rng([seed, b])`` so any subset of frames can be regenerated independently.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Tuple

import numpy as np

PIXEL = 20e-6
WAVELENGTH = 1565e-9
BASE_SEED = 2204_02348


def w_max_deg(wavelength: float = WAVELENGTH, pixel: float = PIXEL) -> float:
    """Maximum resolvable angle lambda/(2 px) in degrees (Background section, worked example)."""
    return wavelength / (2.0 * pixel) * 180.0 / math.pi


def defocus_from_waves(waves: float, window: int, pixel: float = PIXEL, wavelength: float = WAVELENGTH) -> float:
    """Dioptre D whose quadratic phase pi D rho^2 / lambda equals 2 pi * waves at rho = window*px/2."""
    rho = window * pixel / 2.0
    return 2.0 * waves * wavelength / rho ** 2


@dataclass
class Setup:
    """One acquisition geometry plus the reconstruction settings that match it."""

    name: str
    frame_w: int
    frame_h: int
    pol_count: int
    window: int                                  # FFT window N (square), pixels
    beam_centre: List[Tuple[float, float]]       # metres, per polarisation
    tilt_deg: List[Tuple[float, float]]          # reference tilt (x, y), degrees, per polarisation
    defocus: List[float]                         # reference defocus, dioptre, per polarisation
    radius_deg: float                            # Fourier window radius, degrees
    ifft_size: int                               # reconstructed field size M (0: the paper's rule)
    group_count: int                             # HG groups G used for the decomposition
    waist: List[float]                           # HG basis waist, metres, per polarisation
    signal_groups: int                           # HG groups present in the synthetic signal
    dtype: str = "u16"                           # "u16" (12-bit camera) or "f32"
    noise: str = "poisson"                       # "poisson" (u16) or "gauss" (f32, sigma = 1e-3 peak)
    coefs: str = "gauss"                         # "gauss" (unit power) or "haar" (unitary columns)
    peak_counts: float = 4000.0
    pixel: float = PIXEL
    wavelength: float = WAVELENGTH
    fill_factor: bool = False                    # reconstruct with the pixel-response (fill-factor) correction
    basis: str = "hg"                            # coefficient basis: "hg", "lg" or "custom"
    basis_transform: object = None               # custom basis: complex matrix [modes_out][modes_in]
    ref_amplitude: object = None                 # simulator: relative reference amplitude on the camera [H][W]
    ref_cal: object = None                       # reconstruction: measured reference intensity, uint16 [H][W]
    extra: dict = field(default_factory=dict)

    @property
    def modes(self) -> int:
        return self.group_count * (self.group_count + 1) // 2

    @property
    def signal_modes(self) -> int:
        return self.signal_groups * (self.signal_groups + 1) // 2


def _centres(frame_w: int, frame_h: int, pols: int, pixel: float) -> List[Tuple[float, float]]:
    """Window centres at the middle of each polarisation strip."""
    strip = frame_w // pols
    return [((p * strip + strip // 2) * pixel, (frame_h // 2) * pixel) for p in range(pols)]


def setup_plain() -> Setup:
    """1 frame, 128x128 float32 |S+R|^2, one polarisation, 15 modes, 32x32 field (plain-method case)."""
    wm = w_max_deg()
    return Setup(
        name="plain_128_f32",
        frame_w=128, frame_h=128, pol_count=1, window=128,
        beam_centre=_centres(128, 128, 1, PIXEL),
        tilt_deg=[(1.0, 1.0)], defocus=[0.0],
        radius_deg=0.32 * wm, ifft_size=32, group_count=5, waist=[150e-6],
        signal_groups=5, dtype="f32", noise="gauss", coefs="gauss",
    )


def setup_batching(seed: int = BASE_SEED + 1) -> Setup:
    """320x256 uint16 frames, two 128x128 windows, 45 modes, 64x64 fields (batching case).

    Tilts are 1.5 deg + U(-0.05, 0.05) deg per polarisation and axis; defocus U(0, 0.05) waves.
    """
    rng = np.random.default_rng([seed, 10**6])
    wm = w_max_deg()
    tilts = [tuple(1.5 + rng.uniform(-0.05, 0.05, 2)) for _ in range(2)]
    dfs = [defocus_from_waves(rng.uniform(0.0, 0.05), 128) for _ in range(2)]
    return Setup(
        name="batching_320x256_u16",
        frame_w=320, frame_h=256, pol_count=2, window=128,
        beam_centre=_centres(320, 256, 2, PIXEL),
        tilt_deg=tilts, defocus=dfs,
        radius_deg=0.32 * wm, ifft_size=64, group_count=9, waist=[200e-6, 200e-6],
        signal_groups=9, dtype="u16", noise="poisson", coefs="gauss",
    )


def _rule_tilt(radius_deg: float) -> float:
    """Per-axis reference tilt 3 w_c / sqrt(2) that places the window next to the autocorrelation term."""
    return 3.0 * radius_deg / math.sqrt(2.0)


def setup_precision(seed: int = BASE_SEED + 2) -> Setup:
    """640x512 uint16 frames, two 256x256 windows, 120 modes (Haar-unitary coefficient columns)."""
    rng = np.random.default_rng([seed, 10**6])
    wm = w_max_deg()
    rad = 0.32 * wm
    t0 = _rule_tilt(rad)
    tilts = [tuple(t0 + rng.uniform(-0.05, 0.05, 2)) for _ in range(2)]
    return Setup(
        name="precision_640x512_u16",
        frame_w=640, frame_h=512, pol_count=2, window=256,
        beam_centre=_centres(640, 512, 2, PIXEL),
        tilt_deg=tilts, defocus=[0.0, 0.0],
        radius_deg=rad, ifft_size=0, group_count=15, waist=[300e-6, 300e-6],
        signal_groups=15, dtype="u16", noise="poisson", coefs="haar",
    )


def setup_large_batch(seed: int = BASE_SEED + 4) -> Setup:
    """1280x1024 uint16 frames, two 512x512 windows, 210 modes, paper-rule field size (176)."""
    rng = np.random.default_rng([seed, 10**6])
    wm = w_max_deg()
    rad = 0.32 * wm
    t0 = _rule_tilt(rad)
    tilts = [tuple(t0 + rng.uniform(-0.02, 0.02, 2)) for _ in range(2)]
    return Setup(
        name="large_1280x1024_u16",
        frame_w=1280, frame_h=1024, pol_count=2, window=512,
        beam_centre=_centres(1280, 1024, 2, PIXEL),
        tilt_deg=tilts, defocus=[0.0, 0.0],
        radius_deg=rad, ifft_size=0, group_count=20, waist=[400e-6, 400e-6],
        signal_groups=20, dtype="u16", noise="poisson", coefs="gauss",
    )


SERVING_KINDS = ("256x256_1pol", "512x512_2pol", "1024x1024_1pol")


def serving_geometry(kind: str, rng: np.random.Generator) -> Setup:
    """One serving request geometry: radius U(0.15, 0.32) w_max, G in {6..16}, tilt by the 3 w_c/sqrt(2) rule.

    The basis waist is 0.8 (N px / 2) / sqrt(2 G + 1), so the highest group stays inside the window.
    """
    wm = w_max_deg()
    rad = float(rng.uniform(0.15, 0.32)) * wm
    g = int(rng.integers(6, 17))
    if kind == "256x256_1pol":
        fw, fh, pols, n = 256, 256, 1, 256
    elif kind == "512x512_2pol":
        fw, fh, pols, n = 512, 512, 2, 256
    elif kind == "1024x1024_1pol":
        fw, fh, pols, n = 1024, 1024, 1, 1024
    else:
        raise ValueError(kind)
    w = 0.8 * (n * PIXEL / 2.0) / math.sqrt(2 * g + 1)
    t = _rule_tilt(rad)
    return Setup(
        name=f"serve_{kind}",
        frame_w=fw, frame_h=fh, pol_count=pols, window=n,
        beam_centre=_centres(fw, fh, pols, PIXEL),
        tilt_deg=[(t, t)] * pols, defocus=[0.0] * pols,
        radius_deg=rad, ifft_size=0, group_count=g, waist=[w] * pols,
        signal_groups=g, dtype="u16", noise="poisson", coefs="gauss",
    )


WORKLOADS = {
    "plain": setup_plain,
    "batching": setup_batching,
    "precision": setup_precision,
    "large_batch": setup_large_batch,
}


def mode_indices(groups: int) -> List[Tuple[int, int]]:
    """(m, n) pairs with m + n < groups, ordered by group g = m + n, then m ascending."""
    return [(m, g - m) for g in range(groups) for m in range(g + 1)]


def hg_closed_form(n_max: int, x: np.ndarray, w: float) -> np.ndarray:
    """u_n(x), n = 0..n_max-1: (2/pi)^(1/4) / sqrt(2^n n! w) H_n(sqrt(2) x / w) exp(-x^2/w^2).

    Physicists' Hermite polynomials come from numpy.polynomial.hermite.hermval; the normalisation is
    evaluated in log space so it stays finite for n up to a few tens.
    """
    x = np.asarray(x, dtype=np.float64)
    xi = math.sqrt(2.0) * x / w
    out = np.empty((n_max,) + x.shape, dtype=np.float64)
    gauss = np.exp(-(x / w) ** 2)
    for n in range(n_max):
        coef = np.zeros(n + 1)
        coef[n] = 1.0
        hn = np.polynomial.hermite.hermval(xi, coef)
        lognorm = 0.25 * math.log(2.0 / math.pi) - 0.5 * (n * math.log(2.0) + math.lgamma(n + 1) + math.log(w))
        out[n] = math.exp(lognorm) * hn * gauss
    return out


def random_unit_coefs(rng: np.random.Generator, modes: int) -> np.ndarray:
    """Complex-Gaussian coefficient vector normalised to unit total power."""
    c = rng.standard_normal(modes) + 1j * rng.standard_normal(modes)
    return c / np.linalg.norm(c)


def haar_unitary(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-random n x n unitary: QR of a complex Gaussian matrix with the phases of diag(R) removed."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def _signal_coefs(setup: Setup, b: int, p: int, rng: np.random.Generator, seed: int) -> np.ndarray:
    k = setup.signal_modes
    if setup.coefs == "haar":
        # one unitary per polarisation, its columns used by consecutive frames (cycled)
        u = _haar_cache(seed, p, k)
        return u[:, b % k]
    return random_unit_coefs(rng, k)


_HAAR = {}


def _haar_cache(seed: int, p: int, k: int) -> np.ndarray:
    key = (seed, p, k)
    if key not in _HAAR:
        _HAAR[key] = haar_unitary(np.random.default_rng([seed, 2 * 10**6, p]), k)
    return _HAAR[key]


def _pol_tables(setup: Setup):
    """Per-polarisation reference wave R and HG tables on the frame grid (independent of the frame)."""
    H, W, P = setup.frame_h, setup.frame_w, setup.pol_count
    strip = W // P
    px, lam = setup.pixel, setup.wavelength
    ys = np.arange(H) * px
    pol_tabs = []
    for p in range(P):
        cx, cy = setup.beam_centre[p]
        xs = (np.arange(p * strip, (p + 1) * strip)) * px
        X = xs - cx
        Y = ys - cy
        tx, ty = (math.radians(t) for t in setup.tilt_deg[p])
        D = setup.defocus[p]
        rx = np.exp(-2j * math.pi * (tx / lam) * X) * np.exp(-1j * math.pi * D * X ** 2 / lam)
        ry = np.exp(-2j * math.pi * (ty / lam) * Y) * np.exp(-1j * math.pi * D * Y ** 2 / lam)
        ux = hg_closed_form(setup.signal_groups, X, setup.waist[p])   # [G][strip]
        uy = hg_closed_form(setup.signal_groups, Y, setup.waist[p])   # [G][H]
        pol_tabs.append((ry[:, None] * rx[None, :], ux, uy))
    return pol_tabs


def _render(setup: Setup, pol_tabs, coefs_p, rng: np.random.Generator, ref_phase: float = 0.0):
    """One camera frame |S + A_R R exp(i ref_phase)|^2 with the setup's noise; returns (frame, field_scale[P])."""
    H, W, P = setup.frame_h, setup.frame_w, setup.pol_count
    strip = W // P
    modes = mode_indices(setup.signal_groups)
    mi = np.array([m for m, _ in modes])
    ni = np.array([n for _, n in modes])
    inten = np.empty((H, W), dtype=np.float64)
    amps = []
    rot = complex(math.cos(ref_phase), math.sin(ref_phase))
    amp = None if setup.ref_amplitude is None else np.asarray(setup.ref_amplitude, dtype=np.float64)
    for p in range(P):
        R, ux, uy = pol_tabs[p]
        if amp is not None:
            R = R * amp[:, p * strip:(p + 1) * strip]
        C = np.zeros((setup.signal_groups, setup.signal_groups), dtype=np.complex128)
        C[ni, mi] = coefs_p[p]                          # C[n][m]
        S = uy.T @ C @ ux                               # [H][strip]
        a_r = float(np.abs(S).max())
        amps.append(a_r)
        inten[:, p * strip:(p + 1) * strip] = np.abs(S + a_r * rot * R) ** 2
    peak = inten.max()
    if setup.dtype == "u16":
        scale = setup.peak_counts / peak
        counts = rng.poisson(inten * scale)
        frame = np.clip(counts, 0, 4095).astype(np.uint16)
    else:
        scale = 1.0 / peak
        frame = (inten * scale + rng.normal(0.0, 1e-3, size=inten.shape)).astype(np.float32)
    return frame, np.array(amps) * scale


def reference_profile(setup: Setup, sigma_fraction: float = 0.45, floor: int = 600, peak: int = 4000):
    """A non-uniform reference beam for calibration tests: a measured reference intensity cal (uint16 [H][W],
    a Gaussian of width sigma_fraction x frame size centred on the frame, from `floor` to `peak` counts) and
    the relative amplitude sqrt(cal / max cal) that the simulator gives the reference (so the measured
    calibration describes the simulated beam exactly)."""
    H, W = setup.frame_h, setup.frame_w
    y = (np.arange(H) - (H - 1) / 2.0) / (sigma_fraction * H)
    x = (np.arange(W) - (W - 1) / 2.0) / (sigma_fraction * W)
    g = np.exp(-0.5 * (y[:, None] ** 2 + x[None, :] ** 2))
    cal = np.rint(floor + (peak - floor) * g).astype(np.uint16)
    amp = np.sqrt(cal.astype(np.float64) / float(cal.max()))
    return cal, amp


def make_frames(setup: Setup, count: int, seed: int = BASE_SEED, first: int = 0):
    """Generate frames ``first .. first+count-1`` of the seeded stream for ``setup``.

    Returns a dict with
      frames      : [count][H][W] uint16 (12-bit, Poisson) or float32 (Gaussian noise, peak 1),
      coefs_true  : [count][P][signal_modes] complex128 signal coefficients,
      field_scale : [count][P] float64, the factor A_R * (intensity scale) that multiplies S in the
                    linear cross term, so an ideal reconstruction returns field_scale * S.
    """
    H, W, P = setup.frame_h, setup.frame_w, setup.pol_count
    out_dtype = np.uint16 if setup.dtype == "u16" else np.float32
    frames = np.empty((count, H, W), dtype=out_dtype)
    coefs = np.empty((count, P, setup.signal_modes), dtype=np.complex128)
    fscale = np.empty((count, P), dtype=np.float64)
    pol_tabs = _pol_tables(setup)
    for i in range(count):
        b = first + i
        rng = np.random.default_rng([seed, b])
        for p in range(P):
            coefs[i, p] = _signal_coefs(setup, b, p, rng, seed)
        frames[i], fscale[i] = _render(setup, pol_tabs, coefs[i], rng)
    return {"frames": frames, "coefs_true": coefs, "field_scale": fscale}


def make_avg_frames(setup: Setup, batch: int, avg_count: int, avg_mode: int, seed: int = BASE_SEED,
                    drift: float = math.pi):
    """Frames for averaged processing: ``batch`` distinct fields, each measured ``avg_count`` times with
    independent noise and a reference phase drawn uniformly from [-drift, drift] per measurement (the drift
    that phase-aligned averaging removes).  Arranged as the averaging modes lay them out: sequential blocks
    (mode 0, and mode 2 with a single wavelength) [A A A B B B], or interlaced (mode 1) [A B A B A B].

    Returns a dict with frames [batch * avg_count][H][W], coefs_true [batch][P][signal_modes],
    ref_phase [batch][avg_count] and field_scale [batch][avg_count][P].
    """
    H, W, P = setup.frame_h, setup.frame_w, setup.pol_count
    out_dtype = np.uint16 if setup.dtype == "u16" else np.float32
    frames = np.empty((batch * avg_count, H, W), dtype=out_dtype)
    coefs = np.empty((batch, P, setup.signal_modes), dtype=np.complex128)
    phase = np.empty((batch, avg_count), dtype=np.float64)
    fscale = np.empty((batch, avg_count, P), dtype=np.float64)
    pol_tabs = _pol_tables(setup)
    for g in range(batch):
        rng = np.random.default_rng([seed, g, 3])
        for p in range(P):
            coefs[g, p] = _signal_coefs(setup, g, p, rng, seed)
        for j in range(avg_count):
            phase[g, j] = float(rng.uniform(-drift, drift))
            at = g * avg_count + j if avg_mode != 1 else j * batch + g
            frames[at], fscale[g, j] = _render(setup, pol_tabs, coefs[g], rng, phase[g, j])
    return {"frames": frames, "coefs_true": coefs, "ref_phase": phase, "field_scale": fscale}


def candidate_settings(setup: Setup, count: int = 64, seed: int = BASE_SEED + 5):
    """Seeded alignment candidates around the setup's own values (tilt +-0.02 deg, defocus U(0, 0.05) waves,
    waist x U(0.9, 1.1)); returns arrays tilt[count][P][2] (deg), defocus[count][P] (dioptre),
    waist[count][P] (metres)."""
    rng = np.random.default_rng([seed, 3 * 10**6])
    P = setup.pol_count
    tilt = np.empty((count, P, 2))
    dfc = np.empty((count, P))
    wst = np.empty((count, P))
    for s in range(count):
        for p in range(P):
            tilt[s, p] = np.array(setup.tilt_deg[p]) + rng.uniform(-0.02, 0.02, 2)
            dfc[s, p] = defocus_from_waves(rng.uniform(0.0, 0.05), setup.window, setup.pixel, setup.wavelength)
            wst[s, p] = setup.waist[p] * rng.uniform(0.9, 1.1)
    return {"tilt_deg": tilt, "defocus": dfc, "waist": wst}


def with_(setup: Setup, **kw) -> Setup:
    """Copy of ``setup`` with fields replaced (convenience for tests)."""
    return replace(setup, **kw)
