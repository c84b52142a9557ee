"""Pins for the FP64 oracle: each check ties it to something other than itself.

* values the paper prints (worked example of the window-radius rule, the FFT [IFFT] size table);
* library special cases (numpy.fft.fft2 when the beam centre sits on a pixel, numpy's Hermite polynomials);
* closed forms (exact recovery of a band-limited signal carried by a tilted, defocused reference; HG
  orthonormality; single-mode overlaps);
* invariants (Parseval);
* planted mistakes, showing that the pins above fail when the oracle is wrong.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import digholo_oracle as orc
from synth import holograms as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_example.json")
PX, LAM = 20e-6, 1565e-9


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- printed values


def test_worked_example_window_rule():
    gd = _golden()
    tol = gd["printed_precision_rel"]
    wmax = math.degrees(orc.w_max_rad(gd["wavelength_m"], gd["pixel_m"]))
    assert wmax == pytest.approx(gd["w_max_deg_printed"], rel=tol)
    frac = orc.window_radius_fraction()
    assert frac == pytest.approx(gd["window_fraction_printed"], rel=tol)
    wc = frac * wmax
    assert wc <= gd["window_radius_deg_printed_upper_bound"] * (1 + tol)
    assert wc == pytest.approx(gd["window_radius_deg_printed_upper_bound"], rel=tol)
    t = orc.rule_tilt(wc)
    for v in gd["tilt_deg_printed"]:
        assert t == pytest.approx(v, rel=tol)
    assert orc.wrap_radius_fraction() == pytest.approx(gd["wrap_fraction_printed"], rel=tol)
    # the wrap root solves 8 w^2 + 2 w - 2 = 0
    w = orc.wrap_radius_fraction()
    assert 8 * w * w + 2 * w - 2 == pytest.approx(0.0, abs=1e-12)


def test_ifft_size_table():
    gd = _golden()
    for n, m in gd["fft_ifft_sizes_printed"]:
        r_bins = orc.window_radius_fraction() * n / 2.0   # w_c N px / lambda with w_c = frac * lambda/(2 px)
        assert orc.ifft_size_rule(r_bins) == m


def test_mode_count_and_order():
    for g, k in [(5, 15), (9, 45), (15, 120), (20, 210), (0, 0), (1, 1)]:
        assert len(orc.mode_list(g)) == k
    assert orc.mode_list(3) == [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]


def test_round_half_away():
    assert [orc.round_half_away(v) for v in (2.5, -2.5, 2.49, -0.5, 0.5, 3.0)] == [3, -3, 2, -1, 1, 3]


# ----------------------------------------------------------------------------- spectrum


def _geom(n=16, m=16, centre=(8.0, 8.0), kappa=(5.0, 4.0), r=3.0, defocus=0.0, waist=100e-6, groups=3):
    ax = []
    for a in range(2):
        c = centre[a] * PX
        o = orc.round_half_away(c / PX) - n // 2
        ax.append(orc.AxisGeometry(n=n, origin=o, centre=c, kappa=kappa[a], k0=orc.round_half_away(kappa[a]),
                                   m=m, dx=n * PX / m))
    return orc.PolGeometry(x=ax[0], y=ax[1], r_x=r, r_y=r, defocus=defocus, waist=waist, groups=groups,
                           pixel=PX, wavelength=LAM)


def test_spectrum_equals_numpy_fft_for_pixel_centred_window():
    rng = np.random.default_rng(1)
    n = 16
    g = _geom(n=n, centre=(10.0, 9.0))
    frame = rng.standard_normal((24, 24))
    win = orc.cut_window(frame, g)
    bins = np.arange(-n // 2, n // 2 + 5)          # more than one period, unwrapped
    f = orc.window_spectrum(win, g, bins_x=bins, bins_y=bins)
    d = np.fft.fft2(win)                             # d[ky][kx]
    sign = (-1.0) ** (bins[:, None] + bins[None, :])
    ref = sign * d[np.ix_(bins % n, bins % n)]
    assert np.max(np.abs(f - ref)) < 1e-12 * np.max(np.abs(ref))


def test_spectrum_parseval_subpixel_centre():
    rng = np.random.default_rng(2)
    n = 32
    g = _geom(n=n, centre=(16.37, 15.81))
    frame = rng.uniform(0, 4095, size=(40, 40))
    win = orc.cut_window(frame, g)
    bins = np.arange(3, 3 + n)                       # any n consecutive bins form a full period
    f = orc.window_spectrum(win, g, bins_x=bins, bins_y=bins)
    assert np.sum(np.abs(f) ** 2) / n ** 2 == pytest.approx(np.sum(win ** 2), rel=1e-12)


# ----------------------------------------------------------------------------- closed-form recovery


def _trig_case(n=64, m=32, centre=(40.37, 39.81), kappa=(12.3, 10.7), r=9.0, dioptre=1.7, a_r=2.5, seed=3):
    """Linear hologram A_R^2 + 2 Re(A_R S R*) of a signal S chosen so that S R* has integer frequencies:
    S = P(x, y) exp(-2 pi i (kappa - k0).x/(N px)) exp(-i pi D |x|^2 / lambda), P a trigonometric
    polynomial whose bins k0 + q lie inside the circle.  The exact reconstruction is A_R S on the grid."""
    rng = np.random.default_rng(seed)
    g = _geom(n=n, m=m, centre=centre, kappa=kappa, r=r, defocus=dioptre)
    k0 = np.array([g.x.k0, g.y.k0])
    kap = np.array(kappa)
    qs = []
    for qx in range(-4, 5):
        for qy in range(-4, 5):
            if ((k0[0] + qx - kap[0]) ** 2 + (k0[1] + qy - kap[1]) ** 2) <= (0.9 * r) ** 2 and rng.uniform() < 0.6:
                qs.append((qx, qy))
    amps = rng.standard_normal(len(qs)) + 1j * rng.standard_normal(len(qs))

    def signal(X, Y):
        p = np.zeros(np.broadcast(X, Y).shape, dtype=np.complex128)
        for (qx, qy), a in zip(qs, amps):
            p += a * np.exp(2j * np.pi * (qx * X + qy * Y) / (n * PX))
        res = np.exp(-2j * np.pi * ((kap[0] - k0[0]) * X + (kap[1] - k0[1]) * Y) / (n * PX))
        foc = np.exp(-1j * np.pi * dioptre * (X ** 2 + Y ** 2) / LAM)
        return p * res * foc

    H = W = 80
    X = np.arange(W)[None, :] * PX - g.x.centre
    Y = np.arange(H)[:, None] * PX - g.y.centre
    R = np.exp(-2j * np.pi * (kap[0] * X + kap[1] * Y) / (n * PX)) * np.exp(-1j * np.pi * dioptre * (X ** 2 + Y ** 2) / LAM)
    S = signal(X, Y)
    frame = a_r ** 2 + 2.0 * np.real(a_r * S * np.conj(R))
    xp, yp = orc.output_axes(g)
    expected = a_r * signal(xp[None, :], yp[:, None])
    return g, frame, expected


@pytest.mark.parametrize("case", [
    dict(),
    dict(n=32, m=16, centre=(20.5, 19.49), kappa=(6.6, 9.2), r=4.5, dioptre=-3.0),
    dict(n=64, m=48, centre=(37.0, 41.0), kappa=(14.0, -9.0), r=8.0, dioptre=0.0),
])
def test_exact_recovery_band_limited(case):
    g, frame, expected = _trig_case(**case)
    _, mask, e, _ = orc.process_window(frame, g)
    err = np.linalg.norm(e - expected) / np.linalg.norm(expected)
    assert err < 1e-10, err


def test_hermite_recurrence_matches_library_polynomials():
    x = np.linspace(-2e-3, 2e-3, 401)
    for w in (150e-6, 400e-6):
        u = orc.hg_1d(21, x, w)
        ref = syn.hg_closed_form(21, x, w)
        assert np.max(np.abs(u - ref)) < 1e-11 * np.max(np.abs(ref))
    # u_0 has unit norm and the 1/e^2 intensity radius w
    w = 200e-6
    u0 = orc.hg_1d(1, np.array([0.0, w]), w)[0]
    assert u0[1] / u0[0] == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert u0[0] == pytest.approx((2.0 / (math.pi * w * w)) ** 0.25, rel=1e-14)


def test_hg_orthonormal_on_fine_grid():
    w = 300e-6
    dx = w / 16
    x = (np.arange(512) - 256) * dx
    u = orc.hg_1d(20, x, w)
    gram = u @ u.T * dx
    assert np.max(np.abs(gram - np.eye(20))) < 1e-10


def test_overlap_single_asymmetric_mode():
    # fine output grid so the discrete Gram matrix is the identity to rounding
    n, m = 256, 256
    g = _geom(n=n, m=m, centre=(128.0, 128.0), kappa=(60.0, 60.0), r=10.0, waist=8 * n * PX / m, groups=6)
    xp, yp = orc.output_axes(g)
    ux = orc.hg_1d(6, xp, g.waist)
    uy = orc.hg_1d(6, yp, g.waist)
    modes = orc.mode_list(6)
    for (mm, nn) in [(3, 1), (0, 2), (4, 1)]:
        e = (1.5 - 0.5j) * uy[nn][:, None] * ux[mm][None, :]
        c = orc.overlap(e, g)
        target = np.zeros(len(modes), dtype=complex)
        target[modes.index((mm, nn))] = 1.5 - 0.5j
        assert np.max(np.abs(c - target)) < 1e-10


def test_end_to_end_hg_recovery_linear_hologram():
    """A linear hologram of a known HG superposition on an on-bin tilt returns A_R * c_true."""
    setup = syn.Setup(name="pin", frame_w=160, frame_h=160, pol_count=1, window=128,
                      beam_centre=[(80.3 * PX, 79.6 * PX)], tilt_deg=[(0.0, 0.0)], defocus=[0.9],
                      radius_deg=0.32 * math.degrees(LAM / (2 * PX)), ifft_size=64, group_count=5,
                      waist=[200e-6], signal_groups=5)
    # tilt so that kappa is an integer number of bins (40, 37)
    setup.tilt_deg = [(math.degrees(40 * LAM / (128 * PX)), math.degrees(37 * LAM / (128 * PX)))]
    rng = np.random.default_rng(7)
    c_true = syn.random_unit_coefs(rng, 15)
    g = orc.pol_geometry(setup, 0)
    H = W = 160
    X = np.arange(W) * PX - g.x.centre
    Y = np.arange(H) * PX - g.y.centre
    ux = syn.hg_closed_form(5, X, 200e-6)
    uy = syn.hg_closed_form(5, Y, 200e-6)
    S = sum(c * uy[n][:, None] * ux[m][None, :] for c, (m, n) in zip(c_true, orc.mode_list(5)))
    fx, fy = (math.radians(t) / LAM for t in setup.tilt_deg[0])
    R = np.exp(-2j * np.pi * (fx * X[None, :] + fy * Y[:, None])) * \
        np.exp(-1j * np.pi * 0.9 * (X[None, :] ** 2 + Y[:, None] ** 2) / LAM)
    a_r = float(np.abs(S).max())
    frame = a_r ** 2 + 2 * np.real(a_r * S * np.conj(R))
    _, _, _, c = orc.process_window(frame, g)
    assert np.linalg.norm(c - a_r * c_true) / a_r < 1e-6


def test_score_is_total_power_of_per_candidate_runs():
    setup = syn.setup_plain()
    setup = syn.with_(setup, group_count=3)
    data = syn.make_frames(setup, 2, seed=11)
    cand = syn.candidate_settings(setup, 3, seed=12)
    p = orc.score_settings(data["frames"], setup, cand["tilt_deg"], cand["defocus"], cand["waist"])
    for b in range(2):
        for s in range(3):
            su = syn.with_(setup, tilt_deg=[tuple(cand["tilt_deg"][s, 0])], defocus=[cand["defocus"][s, 0]],
                           waist=[cand["waist"][s, 0]])
            _, coefs = orc.process_batch(data["frames"][b:b + 1], su)
            assert p[b, s] == pytest.approx(float(np.sum(np.abs(coefs) ** 2)), rel=1e-12)


def test_synthetic_frames_recover_close_to_truth():
    """On the plain 128x128 case the oracle's coefficients approach field_scale * c_true; the |S|^2
    leakage and noise are physics, so this bound is loose (reported, not a parity bound)."""
    setup = syn.setup_plain()
    data = syn.make_frames(setup, 1, seed=5)
    _, coefs = orc.process_batch(data["frames"], setup)
    ref = data["field_scale"][0, 0] * data["coefs_true"][0, 0]
    assert np.linalg.norm(coefs[0, 0] - ref) / np.linalg.norm(ref) < 0.2


# ----------------------------------------------------------------------------- planted mistakes


def test_planted_defocus_sign_fails_exact_recovery(monkeypatch):
    g, frame, expected = _trig_case()
    orig = orc.reconstruct_field

    def mutant(f_box, mask, geo):
        geo2 = orc.PolGeometry(**{**geo.__dict__, "defocus": -geo.defocus})
        return orig(f_box, mask, geo2)

    monkeypatch.setattr(orc, "reconstruct_field", mutant)
    _, _, e, _ = orc.process_window(frame, g)
    assert np.linalg.norm(e - expected) / np.linalg.norm(expected) > 1e-3


def test_planted_transposed_field_fails_mode_pin(monkeypatch):
    n = m = 256
    g = _geom(n=n, m=m, centre=(128.0, 128.0), kappa=(60.0, 60.0), r=10.0, waist=8 * n * PX / m, groups=6)
    xp, yp = orc.output_axes(g)
    e = orc.hg_1d(6, yp, g.waist)[1][:, None] * orc.hg_1d(6, xp, g.waist)[3][None, :]
    orig = orc.overlap
    monkeypatch.setattr(orc, "overlap", lambda f, geo: orig(f.T, geo))
    c = orc.overlap(e, g)
    assert abs(c[orc.mode_list(6).index((3, 1))]) < 0.5


def test_planted_spectrum_sign_fails_fft_pin(monkeypatch):
    rng = np.random.default_rng(1)
    n = 16
    g = _geom(n=n, centre=(10.0, 9.0))
    win = orc.cut_window(rng.standard_normal((24, 24)), g)
    bins = np.arange(-n // 2, n // 2)
    orig = orc.dft_rows
    monkeypatch.setattr(orc, "dft_rows", lambda ax, px, b: np.conj(orig(ax, px, b)))
    f = orc.window_spectrum(win, g, bins_x=bins, bins_y=bins)
    ref = ((-1.0) ** (bins[:, None] + bins[None, :])) * np.fft.fft2(win)[np.ix_(bins % n, bins % n)]
    assert np.max(np.abs(f - ref)) > 1e-3 * np.max(np.abs(ref))


def _box_integrated_case(n=64, m=32, centre=(40.37, 39.81), kappa=(12.3, 10.7), r=9.0, dioptre=0.0, a_r=2.0, seed=8):
    """Linear hologram of a trigonometric-polynomial cross term recorded by pixels that integrate over their
    whole width: every component exp(2 pi i k.x / (N px)) is multiplied by sinc(k_x/N) sinc(k_y/N)."""
    rng = np.random.default_rng(seed)
    g = _geom(n=n, m=m, centre=centre, kappa=kappa, r=r, defocus=dioptre)
    k0 = np.array([g.x.k0, g.y.k0])
    kap = np.array(kappa)
    qs = [(qx, qy) for qx in range(-3, 4) for qy in range(-3, 4)
          if ((k0[0] + qx - kap[0]) ** 2 + (k0[1] + qy - kap[1]) ** 2) <= (0.9 * r) ** 2]
    amps = rng.standard_normal(len(qs)) + 1j * rng.standard_normal(len(qs))
    X = np.arange(80)[None, :] * PX - g.x.centre
    Y = np.arange(80)[:, None] * PX - g.y.centre
    cross = np.zeros((80, 80), dtype=complex)
    for (qx, qy), a in zip(qs, amps):
        kx, ky = k0[0] + qx, k0[1] + qy
        cross += a * np.sinc(kx / n) * np.sinc(ky / n) * np.exp(2j * np.pi * (kx * X + ky * Y) / (n * PX))
    frame = a_r ** 2 + 2.0 * np.real(a_r * cross)
    xp, yp = orc.output_axes(g)
    res = np.exp(-2j * np.pi * ((kap[0] - k0[0]) * xp[None, :] + (kap[1] - k0[1]) * yp[:, None]) / (n * PX))
    p = sum(a * np.exp(2j * np.pi * (qx * xp[None, :] + qy * yp[:, None]) / (n * PX)) for (qx, qy), a in zip(qs, amps))
    return g, frame, a_r * p * res


def test_fill_factor_correction_recovers_box_integrated_signal():
    g, frame, expected = _box_integrated_case()
    g.fill_factor = True
    _, _, e, _ = orc.process_window(frame, g)
    assert np.linalg.norm(e - expected) / np.linalg.norm(expected) < 1e-10
    g.fill_factor = False
    _, _, e2, _ = orc.process_window(frame, g)
    assert np.linalg.norm(e2 - expected) / np.linalg.norm(expected) > 1e-3


# ----------------------------------------------------------------------------- LG and custom bases


def test_lg_modes_orthonormal_and_textbook_low_orders():
    w = 1.0
    x = (np.arange(320) - 160) * (w / 16)
    modes = orc.lg_mode_list(5)
    assert len(modes) == 15 and modes[:6] == [(0, 0), (0, -1), (0, 1), (0, -2), (1, 0), (0, 2)]
    L = np.array([orc.lg_2d(p, l, x, x, w).ravel() for (p, l) in modes])
    gram = np.conj(L) @ L.T * (w / 16) ** 2
    assert np.max(np.abs(gram - np.eye(len(modes)))) < 1e-10
    u = orc.hg_1d(3, x, w)
    hg = lambda m, n: u[n][:, None] * u[m][None, :]
    assert np.max(np.abs(orc.lg_2d(0, 0, x, x, w) - hg(0, 0))) < 1e-12
    # LG_0^{+-1} = (HG_10 +- i HG_01) / sqrt(2): exp(+- i phi) r exp(-r^2/w^2) is proportional to x +- i y
    for l in (1, -1):
        ref = (hg(1, 0) + 1j * l * hg(0, 1)) / math.sqrt(2.0)
        assert np.max(np.abs(orc.lg_2d(0, l, x, x, w) - ref)) < 1e-12


def test_lg_overlap_recovers_single_mode_on_fine_grid():
    n = m = 256
    g = _geom(n=n, m=m, centre=(128.0, 128.0), kappa=(60.0, 60.0), r=10.0, waist=8 * n * PX / m, groups=5)
    xp, yp = orc.output_axes(g)
    modes = orc.lg_mode_list(5)
    for (p, l) in [(1, 2), (0, -3), (2, 0)]:
        e = (0.5 + 2j) * orc.lg_2d(p, l, xp, yp, g.waist)
        c = orc.overlap_lg(e, g)
        target = np.zeros(len(modes), dtype=complex)
        target[modes.index((p, l))] = 0.5 + 2j
        assert np.max(np.abs(c - target)) < 1e-10


def test_custom_basis_is_the_matrix_applied_to_hg_overlaps():
    rng = np.random.default_rng(12)
    g = _geom(n=64, m=32, centre=(32.0, 32.0), kappa=(14.0, 12.0), r=8.0, waist=200e-6, groups=4)
    e = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    t = rng.standard_normal((5, 12)) + 1j * rng.standard_normal((5, 12))   # more inputs than the 10 HG modes
    c = orc.basis_coefficients(e, g, "custom", t)
    assert c.shape == (5,)
    assert np.allclose(c, t[:, :10] @ orc.overlap(e, g), rtol=1e-13, atol=0)
    assert np.allclose(orc.basis_coefficients(e, g, "custom", np.eye(10)), orc.overlap(e, g), rtol=1e-14, atol=0)


# ----------------------------------------------------------------------------- batch averaging


def test_avg_member_layouts():
    # sequential [A A A B B B]: group 1 of 2, 3 per group -> frames 3, 4, 5; interlaced [A B A B A B] -> 1, 3, 5
    assert [orc.avg_member_index(1, j, 2, 3, 0) for j in range(3)] == [3, 4, 5]
    assert [orc.avg_member_index(1, j, 2, 3, 2) for j in range(3)] == [3, 4, 5]
    assert [orc.avg_member_index(1, j, 2, 3, 1) for j in range(3)] == [1, 3, 5]


def test_align_phases_hand_example_and_pure_rotation():
    # W_0 = [1, 0], W_1 = [i, 1]: <W_0, W_1> = i, so W_1 is rotated by -i -> [1, -i]; average [1, -i/2]
    w = [[np.array([1.0 + 0j, 0.0])], [np.array([1j, 1.0 + 0j])]]
    a = orc.align_phases(w)
    assert np.allclose(a, [1.0, -1j], atol=1e-15)
    assert np.allclose((a[0] * w[0][0] + a[1] * w[1][0]) / 2, [1.0, -0.5j], atol=1e-15)
    # copies of one window rotated by arbitrary phases average back to the first copy exactly
    rng = np.random.default_rng(31)
    base = [rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)) for _ in range(2)]
    th = np.array([0.0, 2.5, -1.2, 3.1])
    group = [[np.exp(1j * t) * base[p] for p in range(2)] for t in th]
    a = orc.align_phases(group)
    assert np.allclose(a, np.exp(-1j * th), atol=1e-14)
    # a zero window (no light) keeps phasor 1
    assert orc.align_phases([[np.ones(3)], [np.zeros(3)]])[1] == 1.0


def test_avg_count_one_is_plain_processing_and_modes_agree():
    s = syn.setup_batching()
    d = syn.make_frames(s, 3, seed=40)
    f1, c1 = orc.process_batch(d["frames"], s)
    fa, ca = orc.process_batch_avg(d["frames"], s, 1, 0)
    assert np.allclose(fa, f1, rtol=0, atol=1e-12 * np.abs(f1).max())
    assert np.allclose(ca, c1, rtol=0, atol=1e-12 * np.abs(c1).max())
    # the same frames laid out interlaced give the same averages as the sequential layout
    dd = syn.make_avg_frames(s, 2, 3, 0, seed=41)
    seq = dd["frames"]
    inter = np.stack([seq[g * 3 + j] for j in range(3) for g in range(2)])
    fs, _ = orc.process_batch_avg(seq, s, 3, 0)
    fi, _ = orc.process_batch_avg(inter, s, 3, 1)
    assert np.array_equal(fs, fi)


def test_avg_of_identical_frames_and_drift_removal():
    s = syn.setup_batching()
    d = syn.make_frames(s, 1, seed=42)
    f1, _ = orc.process_batch(d["frames"], s)
    fa, _ = orc.process_batch_avg(np.repeat(d["frames"], 4, axis=0), s, 4, 0)
    assert np.allclose(fa, f1, rtol=0, atol=1e-12 * np.abs(f1).max())
    # one field measured 6 times with reference drift: the aligned average stays close to the true field
    # (times the first member's phase), closer than a single noisy measurement, while the plain mean of the
    # drifting fields loses most of its amplitude
    dd = syn.make_avg_frames(s, 1, 6, 0, seed=43)
    fa, _ = orc.process_batch_avg(dd["frames"], s, 6, 0)
    singles, _ = orc.process_batch(dd["frames"], s)
    g0 = orc.pol_geometry(s, 0)
    xp, yp = orc.output_axes(g0)
    true = np.zeros((len(yp), len(xp)), dtype=complex)
    u_x = syn.hg_closed_form(s.signal_groups, xp, s.waist[0])
    u_y = syn.hg_closed_form(s.signal_groups, yp, s.waist[0])
    for k, (m, n) in enumerate(syn.mode_indices(s.signal_groups)):
        true += dd["coefs_true"][0, 0, k] * np.outer(u_y[n], u_x[m])
    def err(e):   # relative error after the best global phase
        z = np.vdot(true, e)
        return np.linalg.norm(e * np.conj(z) / abs(z) / np.linalg.norm(e) - true / np.linalg.norm(true))
    assert err(fa[0, 0]) < min(err(singles[j, 0]) for j in range(6))
    plain_mean = singles[:, 0].mean(axis=0)
    assert np.linalg.norm(plain_mean) < 0.8 * np.linalg.norm(fa[0, 0])


# ----------------------------------------------------------------------------- reference calibration


def test_reference_calibration_factor_values():
    cal = np.array([[4000, 1000], [0, 250]], dtype=np.uint16)
    f = orc.reference_calibration_factor(cal)
    assert np.array_equal(f, np.array([[1.0, 2.0], [0.0, 4.0]]))           # sqrt(4000 / cal), 0 for dark pixels
    # with several wavelength frames the maximum is taken over all of them; the first frame is used
    cal3 = np.stack([cal, np.full((2, 2), 16000, dtype=np.uint16)])
    assert np.array_equal(orc.reference_calibration_factor(cal3), np.array([[2.0, 4.0], [0.0, 8.0]]))


def test_reference_calibration_removes_a_nonuniform_reference_exactly_on_the_cross_term():
    # linear hologram 2 Re(S a R*) with a non-uniform reference amplitude a = sqrt(cal / max cal): after the
    # calibration it is exactly the uniform-reference hologram 2 Re(S R*), so the reconstructions agree to
    # rounding, pixel for pixel (a transposed or wrongly scaled factor fails)
    s = syn.setup_batching()
    cal, amp = syn.reference_profile(s, sigma_fraction=0.3)
    assert amp.shape == (s.frame_h, s.frame_w) and amp.min() < 0.5
    rng = np.random.default_rng(50)
    H, W = s.frame_h, s.frame_w
    cross = rng.standard_normal((H, W))            # any pattern: the identity is pixelwise
    f_uniform, c_uniform = orc.process_batch(cross[None], s)
    sc = syn.with_(s, ref_cal=cal)
    f_cal, c_cal = orc.process_batch((cross * amp)[None], sc)
    assert np.allclose(f_cal, f_uniform, rtol=0, atol=1e-12 * np.abs(f_uniform).max())
    assert np.allclose(c_cal, c_uniform, rtol=0, atol=1e-12 * np.abs(c_uniform).max())


def test_reference_calibration_improves_recovery_on_simulated_frames():
    # a reference beam narrower than the frame, so its amplitude falls steeply across both polarisation
    # windows (beams at W/4 and 3W/4): uncalibrated, the field carries that envelope
    s0 = syn.setup_batching()
    cal, amp = syn.reference_profile(s0, sigma_fraction=0.15, floor=200)
    s = syn.with_(s0, ref_amplitude=amp)
    d = syn.make_frames(s, 1, seed=51)
    g = orc.pol_geometry(s, 0)
    xp, yp = orc.output_axes(g)
    true = np.zeros((len(yp), len(xp)), dtype=complex)
    u_x = syn.hg_closed_form(s.signal_groups, xp, s.waist[0])
    u_y = syn.hg_closed_form(s.signal_groups, yp, s.waist[0])
    for k, (m, n) in enumerate(syn.mode_indices(s.signal_groups)):
        true += d["coefs_true"][0, 0, k] * np.outer(u_y[n], u_x[m])

    def err(e):
        z = np.vdot(true, e)
        return np.linalg.norm(e * np.conj(z) / abs(z) / np.linalg.norm(e) - true / np.linalg.norm(true))

    f_plain, _ = orc.process_batch(d["frames"], s)
    f_cal, _ = orc.process_batch(d["frames"], syn.with_(s, ref_cal=cal))
    assert err(f_cal[0, 0]) < 0.5 * err(f_plain[0, 0])


# ----------------------------------------------------------------------------- transfer-matrix metrics


def _m(A, groups=None, mct=False):
    A = np.asarray(A, dtype=np.complex128)
    return orc.transfer_metrics(A[:, None, :], groups=groups, mul_conj_trans=mct)


def test_metrics_identity_and_unitary():
    m = _m(np.eye(6), groups=3)
    assert m["IL"] == 0.0 and m["MDL"] == 0.0 and m["DIAGBEST"] == 0.0 and m["DIAGWORST"] == 0.0
    assert m["DIAG"] == pytest.approx(10 * math.log10(6), abs=1e-12)
    assert m["SNRAVG"] == math.inf and m["SNRBEST"] == math.inf and m["SNRWORST"] == math.inf
    assert m["SNRMG"] == math.inf
    u = syn.haar_unitary(np.random.default_rng(60), 10)
    mu = _m(u, groups=4)
    assert abs(mu["IL"]) < 1e-12 and abs(mu["MDL"]) < 1e-12
    mc = _m(u, groups=4, mct=True)                     # U U^H = I
    assert mc["SNRAVG"] > 250 and mc["DIAG"] == pytest.approx(10.0, abs=1e-12)


def test_metrics_closed_forms_3x3():
    # singular values^2 {1, 1/2, 1/4}: IL = 10 log10(1.75 / 3), MDL = 10 log10 4
    d = _m(np.diag([1.0, math.sqrt(0.5), 0.5]))
    assert d["IL"] == pytest.approx(10 * math.log10(1.75 / 3), abs=1e-12)
    assert d["MDL"] == pytest.approx(10 * math.log10(4.0), abs=1e-12)
    # powers [[1, .25, 0], [0, 4, .04], [.01, 0, 1]]; groups: mode 0 alone, modes 1-2 together (G = 2)
    A = np.array([[1, 0.5, 0], [0, 2, 0.2j], [-0.1, 0, 1j]])
    m = _m(A, groups=2)
    assert m["DIAG"] == pytest.approx(10 * math.log10(6.0), abs=1e-12)
    assert m["SNRAVG"] == pytest.approx(10 * math.log10(6.0 / 0.3), abs=1e-10)
    assert m["DIAGBEST"] == pytest.approx(10 * math.log10(4.0), abs=1e-12)
    assert m["DIAGWORST"] == pytest.approx(0.0, abs=1e-12)
    assert m["SNRBEST"] == pytest.approx(20.0, abs=1e-10)
    assert m["SNRWORST"] == pytest.approx(10 * math.log10(4.0), abs=1e-10)
    assert m["SNRMG"] == pytest.approx(10 * math.log10(6.04 / 0.26), abs=1e-10)
    sv = np.linalg.svd(A, compute_uv=False) ** 2    # an independent routine for the eigenvalues
    assert m["IL"] == pytest.approx(10 * math.log10(sv.mean()), abs=1e-12)
    assert m["MDL"] == pytest.approx(10 * math.log10(sv.max() / sv.min()), abs=1e-10)
    assert _m(A)["SNRMG"] is None                     # no group structure given


def test_metrics_rectangular_and_two_polarisations():
    rng = np.random.default_rng(61)
    c = rng.standard_normal((4, 2, 3)) + 1j * rng.standard_normal((4, 2, 3))     # 4 rows, 6 columns
    m = orc.transfer_metrics(c, groups=2)
    A = c.reshape(4, 6)
    sv = np.linalg.svd(A, compute_uv=False) ** 2
    assert m["IL"] == pytest.approx(10 * math.log10(sv.mean()), abs=1e-10)
    pw = np.abs(A) ** 2
    d = np.diag(pw)
    assert m["DIAG"] == pytest.approx(10 * math.log10(d.sum()), abs=1e-12)
    # SNRMG signal: same polarisation block (column // 3 == row // 3) and same group
    grp = [0, 1, 1]
    sig = sum(pw[i, j] for i in range(4) for j in range(6) if i // 3 == j // 3 and grp[i % 3] == grp[j % 3])
    assert m["SNRMG"] == pytest.approx(10 * math.log10(sig / (pw.sum() - sig)), abs=1e-10)
    c8 = rng.standard_normal((8, 2, 3)) + 1j * rng.standard_normal((8, 2, 3))     # 8 rows > 6 columns
    mt = orc.transfer_metrics(c8, groups=2)
    sv8 = np.linalg.svd(c8.reshape(8, 6), compute_uv=False) ** 2
    assert mt["IL"] == pytest.approx(10 * math.log10(sv8.mean()), abs=1e-10)
    assert mt["MDL"] == pytest.approx(10 * math.log10(sv8.max() / sv8.min()), abs=1e-9)
    # a rank-deficient matrix has an infinite MDL
    assert orc.transfer_metrics(np.concatenate([c, c], axis=0), groups=2)["MDL"] == math.inf


# ----------------------------------------------------------------------------- fine-alignment search


def test_search_stencil():
    t = np.array([[1.0, 2.0], [3.0, 4.0]])
    T, D, W = orc.search_candidates(t, np.array([0.1, 0.2]), np.array([1e-4, 2e-4]), np.array([0.5, 0.25, 0.1]))
    assert T.shape == (17, 2, 2) and D.shape == (17, 2) and W.shape == (17, 2)
    assert np.array_equal(T[0], t)
    assert T[1][0, 0] == 0.5 and T[2][0, 0] == 1.5 and T[3][0, 1] == 1.5 and T[4][0, 1] == 2.5
    assert D[5][0] == pytest.approx(-0.15) and D[6][0] == pytest.approx(0.35)
    assert W[7][0] == pytest.approx(0.9e-4) and W[8][0] == pytest.approx(1.1e-4)
    assert T[9][1, 0] == 2.5 and W[16][1] == pytest.approx(2.2e-4)


def test_search_recovers_the_true_alignment():
    s = syn.setup_plain()
    d = syn.make_frames(s, 1, seed=62)
    off = syn.with_(s, tilt_deg=[(s.tilt_deg[0][0] + 0.03, s.tilt_deg[0][1] - 0.02)],
                    waist=[s.waist[0] * 1.06])
    t, dfc, w, power, its = orc.auto_align_tweak(d["frames"], off, max_iter=60)
    assert abs(t[0, 0] - s.tilt_deg[0][0]) < 4e-3 and abs(t[0, 1] - s.tilt_deg[0][1]) < 4e-3
    assert abs(w[0] / s.waist[0] - 1.0) < 0.01
    p_true = orc.score_settings(d["frames"], s, np.array([s.tilt_deg]), np.array([s.defocus]),
                                np.array([s.waist])).sum()
    p_start = orc.score_settings(d["frames"], off, np.array([off.tilt_deg]), np.array([off.defocus]),
                                 np.array([off.waist])).sum()
    assert power >= p_true * (1 - 1e-3) and power > p_start


# ----------------------------------------------------------------------------- non-square windows and fields


def _rect_geom(n=(32, 16), m=(16, 32), centre=(20.0, 9.0), kappa=(9.3, 4.6), r=(6.0, 3.0), defocus=0.0):
    ax = []
    for a in range(2):
        c = centre[a] * PX
        o = orc.round_half_away(c / PX) - n[a] // 2
        ax.append(orc.AxisGeometry(n=n[a], origin=o, centre=c, kappa=kappa[a], k0=orc.round_half_away(kappa[a]),
                                   m=m[a], dx=n[a] * PX / m[a]))
    return orc.PolGeometry(x=ax[0], y=ax[1], r_x=r[0], r_y=r[1], defocus=defocus, waist=100e-6, groups=3,
                           pixel=PX, wavelength=LAM)


def test_rectangular_window_spectrum_equals_numpy_fft():
    # an N_y x N_x window (rows along y): the separable DFT on unwrapped bins equals numpy's fft2 with each
    # axis' own period
    rng = np.random.default_rng(11)
    g = _rect_geom(n=(32, 16), centre=(20.0, 9.0))
    frame = rng.standard_normal((24, 48))
    win = orc.cut_window(frame, g)
    assert win.shape == (16, 32)
    bx, by = np.arange(-16, 21), np.arange(-8, 11)
    f = orc.window_spectrum(win, g, bins_x=bx, bins_y=by)
    d = np.fft.fft2(win)                             # d[ky][kx]
    ref = ((-1.0) ** (by[:, None] + bx[None, :])) * d[np.ix_(by % 16, bx % 32)]
    assert np.max(np.abs(f - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,m,kappa,r", [((64, 32), (32, 16), (14.3, 6.7), (9.0, 4.5)),
                                         ((32, 64), (16, 48), (7.2, 14.6), (4.0, 8.0))])
def test_rectangular_exact_recovery(n, m, kappa, r):
    """Linear hologram of a signal whose S R* has integer frequencies inside the elliptic window (the circle in
    angle is an ellipse in bins when N_x != N_y): the reconstruction is A_R S on the M_y x M_x grid."""
    rng = np.random.default_rng(12)
    dioptre, a_r = 1.3, 2.0
    g = _rect_geom(n=n, m=m, centre=(40.4, 38.7), kappa=kappa, r=r, defocus=dioptre)
    k0 = np.array([g.x.k0, g.y.k0])
    kap = np.array(kappa)
    qs = [(qx, qy) for qx in range(-4, 5) for qy in range(-4, 5)
          if ((k0[0] + qx - kap[0]) / r[0]) ** 2 + ((k0[1] + qy - kap[1]) / r[1]) ** 2 <= 0.8 and rng.uniform() < 0.7]
    assert len(qs) >= 4
    amps = rng.standard_normal(len(qs)) + 1j * rng.standard_normal(len(qs))

    def signal(X, Y):
        p = np.zeros(np.broadcast(X, Y).shape, dtype=np.complex128)
        for (qx, qy), a in zip(qs, amps):
            p += a * np.exp(2j * np.pi * (qx * X / (n[0] * PX) + qy * Y / (n[1] * PX)))
        res = np.exp(-2j * np.pi * ((kap[0] - k0[0]) * X / (n[0] * PX) + (kap[1] - k0[1]) * Y / (n[1] * PX)))
        return p * res * np.exp(-1j * np.pi * dioptre * (X ** 2 + Y ** 2) / LAM)

    X = np.arange(80)[None, :] * PX - g.x.centre
    Y = np.arange(80)[:, None] * PX - g.y.centre
    R = np.exp(-2j * np.pi * (kap[0] * X / (n[0] * PX) + kap[1] * Y / (n[1] * PX))) * \
        np.exp(-1j * np.pi * dioptre * (X ** 2 + Y ** 2) / LAM)
    frame = a_r ** 2 + 2.0 * np.real(a_r * signal(X, Y) * np.conj(R))
    _, _, e, _ = orc.process_window(frame, g)
    assert e.shape == (m[1], m[0])
    xp, yp = orc.output_axes(g)
    expected = a_r * signal(xp[None, :], yp[:, None])
    err = np.linalg.norm(e - expected) / np.linalg.norm(expected)
    assert err < 1e-10, err


def test_rectangular_geometry_per_axis_bins():
    # per axis, angles become bins with that axis' window: kappa = theta N px / lambda, r = w_c N px / lambda,
    # and the field-size rule 16 ceil(2 r / 16) uses that axis' radius
    s = syn.with_(syn.setup_batching(), window=(128, 64), ifft_size=0)
    g = orc.pol_geometry(s, 0)
    th = [math.radians(t) for t in s.tilt_deg[0]]
    assert g.x.kappa == pytest.approx(th[0] * 128 * PX / LAM, rel=1e-15)
    assert g.y.kappa == pytest.approx(th[1] * 64 * PX / LAM, rel=1e-15)
    rx = math.radians(s.radius_deg) * 128 * PX / LAM
    assert g.r_x == pytest.approx(rx, rel=1e-15) and g.r_y == pytest.approx(rx / 2, rel=1e-15)
    assert (g.x.m, g.y.m) == (16 * math.ceil(2 * rx / 16), 16 * math.ceil(rx / 16))
    assert (g.x.n, g.y.n) == (128, 64)
    assert g.x.dx == pytest.approx(128 * PX / g.x.m) and g.y.dx == pytest.approx(64 * PX / g.y.m)
