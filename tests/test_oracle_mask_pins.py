"""Pins for the oracle's circular Fourier window (pipeline step 2, digHoloConfigSetFourierWindowRadius, and the
real-to-complex half plane of digHoloGetFourierPlaneFull).

The window keeps a bin k of the box when ((k_x - kappa_x)/r)^2 + ((k_y - kappa_y)/r)^2 <= 1 and
0 <= k_x <= N/2.  These pins fix every part of that rule from outside the oracle:

* hand-written bin lattices for tiny geometries (the expected masks below are typed in, row by row, from
  the squared distances worked out by hand; nothing here calls the mask to make them): bins exactly on the
  circle are kept (the test is "<=", not "<"), bins just inside and just outside the radius, and circles
  that cross k_x = N/2 and k_x = 0;
* exact recovery of a band-limited signal whose off-axis term sits beside the Nyquist column: components of
  S R* just outside the radius must be absent from the field, components just inside must be present, and the
  conjugate twin's aliases (bins N - k_x > N/2 inside the circle) must be rejected by the half plane.  Each of
  these breaks the recovery by many orders of magnitude when the rule is changed.
"""
import numpy as np
import pytest

from oracle import digholo_oracle as orc

PX, LAM = 20e-6, 1565e-9


def _geom(n, m, kappa, r, centre=None, defocus=0.0):
    centre = (n / 2.0, n / 2.0) if centre is None else centre
    ax = []
    for a in range(2):
        c = centre[a] * PX
        o = orc.round_half_away(c / PX) - n // 2
        ax.append(orc.AxisGeometry(n=n, origin=o, centre=c, kappa=kappa[a], k0=orc.round_half_away(kappa[a]),
                                   m=m, dx=n * PX / m))
    return orc.PolGeometry(x=ax[0], y=ax[1], r_x=r, r_y=r, defocus=defocus, waist=100e-6, groups=3,
                           pixel=PX, wavelength=LAM)


def _lattice(rows):
    return np.array([[ch == "#" for ch in row] for row in rows], dtype=bool)


# ----------------------------------------------------------------------------- hand-written lattices


def test_mask_lattice_exact_circle_crossing_nyquist():
    """N = 16, kappa = (7, 3), r = 2, M = 8: box k_x = 3..10, k_y = -1..6.  Every quantity is exact in binary
    floating point, so the bins at distance exactly r, (5, 3), (7, 1) and (7, 5), lie on the circle and are
    kept; (9, 3) is on the circle too but beyond k_x = N/2 = 8 and is dropped, as are (9, 2) and (9, 4)
    (distance^2 = 5 > 4 anyway) and everything at k_x = 9, 10."""
    g = _geom(16, 8, (7.0, 3.0), 2.0)
    assert list(orc.box_bins(g.x)) == list(range(3, 11))
    assert list(orc.box_bins(g.y)) == list(range(-1, 7))
    expected = _lattice([
        # k_x: 3456789A
        "........",   # k_y = -1
        "........",   # k_y = 0
        "....#...",   # k_y = 1: (7,1) on the circle
        "...###..",   # k_y = 2: d^2 = 2, 1, 2
        "..####..",   # k_y = 3: (5,3) on the circle, (9,3) on it but past N/2
        "...###..",   # k_y = 4
        "....#...",   # k_y = 5: (7,5) on the circle
        "........",   # k_y = 6
    ])
    assert np.array_equal(orc.window_mask(g), expected)


def test_mask_lattice_offbin_centre_crossing_nyquist():
    """N = 16, kappa = (7.6, 3.3), r = 2.5, M = 8: k0 = (8, 3), box k_x = 4..11, k_y = -1..6.
    Squared x offsets (k_x - 7.6)^2 for k_x = 5..11: 6.76, 2.56, 0.36, 0.16, 1.96, 5.76, 11.56; squared y
    offsets (k_y - 3.3)^2 for k_y = 0..6: 10.89, 5.29, 1.69, 0.09, 0.49, 2.89, 7.29; kept when the sum is
    <= 6.25 and k_x <= 8.  Row k_y = 1 keeps only k_x = 7, 8 (5.29 + 0.36 = 5.65; 5.29 + 2.56 > 6.25), row
    k_y = 6 keeps nothing (7.29 > 6.25); k_x = 9, 10 lie inside the circle on rows 2..5 but past N/2."""
    g = _geom(16, 8, (7.6, 3.3), 2.5)
    assert (g.x.k0, g.y.k0) == (8, 3)
    expected = _lattice([
        # k_x: 456789AB
        "........",   # k_y = -1
        "........",   # k_y = 0
        "...##...",   # k_y = 1
        "..###...",   # k_y = 2
        "..###...",   # k_y = 3
        "..###...",   # k_y = 4
        "..###...",   # k_y = 5
        "........",   # k_y = 6
    ])
    assert np.array_equal(orc.window_mask(g), expected)


def test_mask_lattice_circle_crossing_zero():
    """N = 16, kappa = (1, 5), r = 2, M = 8: box k_x = -3..4, k_y = 1..8.  The circle reaches k_x = -1, which
    lies outside the half plane (dropped although (-1, 5) is on the circle); (3, 5), (1, 3) and (1, 7) are on
    the circle and kept; k_x = 0 (the lower edge of the half plane) is kept."""
    g = _geom(16, 8, (1.0, 5.0), 2.0)
    assert list(orc.box_bins(g.x)) == list(range(-3, 5))
    assert list(orc.box_bins(g.y)) == list(range(1, 9))
    expected = _lattice([
        # k_x: ---01234  (-3 .. 4)
        "........",   # k_y = 1
        "........",   # k_y = 2
        "....#...",   # k_y = 3: (1,3) on the circle
        "...###..",   # k_y = 4: k_x = -1 has d^2 = 5
        "...####.",   # k_y = 5: (-1,5) on the circle but k_x < 0; (3,5) on the circle
        "...###..",   # k_y = 6
        "....#...",   # k_y = 7: (1,7) on the circle
        "........",   # k_y = 8
    ])
    assert np.array_equal(orc.window_mask(g), expected)


def test_mask_lattice_anisotropic_box_edges():
    """A radius larger than the box: every bin of the box inside the half plane is kept (the box clips the
    circle, as in the plain workload's M = 32 < 2r), and the half-plane column k_x = N/2 is the last one."""
    g = _geom(32, 8, (14.0, 6.0), 10.0)
    kx = orc.box_bins(g.x)
    assert list(kx) == list(range(10, 18))
    expected = np.zeros((8, 8), dtype=bool)
    expected[:, :7] = True              # k_x = 10..16 kept, k_x = 17 > 16 dropped
    assert np.array_equal(orc.window_mask(g), expected)


# ----------------------------------------------------------------------------- exact recovery beside Nyquist


def _nyquist_case(n=64, m=16, kappa=(29.6, 0.7), r=5.0, centre=(40.37, 39.81), dioptre=0.8, a_r=1.7, seed=11):
    """Linear hologram A_R^2 + 2 Re(A_R S R*) with S R* a sum of integer-frequency components (times the
    reference's residual tilt and defocus), split by their distance d from kappa:

    * 'in':    d <= 0.99 r, at least one with d in [0.96 r, 0.99 r], all with k_x <= N/2 - 1;
    * 'out':   d in [1.01 r, 1.10 r], inside the box, k_x <= N/2 - 1.

    The circle reaches past N/2 and kappa_y is near 0, so the conjugate twin of every component at (k_x, k_y),
    aliased to (N - k_x, -k_y) with N - k_x > N/2, falls inside the box and partly inside the circle.  The
    exact field is A_R times the 'in' components only."""
    rng = np.random.default_rng(seed)
    g = _geom(n, m, kappa, r, centre=centre, defocus=dioptre)
    k0 = np.array([g.x.k0, g.y.k0])
    kap = np.array(kappa)
    inside, outside = [], []
    for qx in range(-m // 2, m // 2):
        for qy in range(-m // 2, m // 2):
            kx, ky = k0[0] + qx, k0[1] + qy
            if kx > n // 2 - 1 or kx < 1:
                continue
            d = np.hypot(kx - kap[0], ky - kap[1]) / r
            if d <= 0.99:
                inside.append((qx, qy, d))
            elif 1.01 <= d <= 1.10:
                outside.append((qx, qy, d))
    edge = [q for q in inside if q[2] >= 0.96]
    rest = [q for q in inside if q[2] < 0.96]
    pick = edge + [rest[i] for i in rng.choice(len(rest), size=min(10, len(rest)), replace=False)]
    amps_in = rng.standard_normal(len(pick)) + 1j * rng.standard_normal(len(pick))
    amps_out = rng.standard_normal(len(outside)) + 1j * rng.standard_normal(len(outside))

    def term(comps, amps, X, Y):
        p = np.zeros(np.broadcast(X, Y).shape, dtype=np.complex128)
        for (qx, qy, _), a in zip(comps, amps):
            p += a * np.exp(2j * np.pi * (qx * X + qy * Y) / (n * PX))
        res = np.exp(-2j * np.pi * ((kap[0] - k0[0]) * X + (kap[1] - k0[1]) * Y) / (n * PX))
        foc = np.exp(-1j * np.pi * dioptre * (X ** 2 + Y ** 2) / LAM)
        return p * res * foc

    H = W = 96
    X = np.arange(W)[None, :] * PX - g.x.centre
    Y = np.arange(H)[:, None] * PX - g.y.centre
    R = np.exp(-2j * np.pi * (kap[0] * X + kap[1] * Y) / (n * PX)) * np.exp(-1j * np.pi * dioptre * (X ** 2 + Y ** 2) / LAM)
    S = term(pick, amps_in, X, Y) + term(outside, amps_out, X, Y)
    frame = a_r ** 2 + 2.0 * np.real(a_r * S * np.conj(R))
    xp, yp = orc.output_axes(g)
    expected_in = a_r * term(pick, amps_in, xp[None, :], yp[:, None])
    expected_out = a_r * term(outside, amps_out, xp[None, :], yp[:, None])
    return g, frame, expected_in, expected_out, len(edge), len(outside)


@pytest.mark.parametrize("case", [
    dict(),
    dict(kappa=(30.2, -0.4), r=4.3, centre=(31.5, 47.2), dioptre=-1.2, seed=12),
    dict(n=32, m=16, kappa=(13.7, 0.2), r=3.6, centre=(20.1, 19.9), dioptre=0.0, seed=13),
])
def test_recovery_rejects_outside_circle_and_past_nyquist(case):
    g, frame, exp_in, exp_out, n_edge, n_out = _nyquist_case(**case)
    assert n_edge >= 1 and n_out >= 4
    # the circle crosses the Nyquist column, so the twin's aliases fall inside it
    assert g.x.kappa + g.r_x > g.x.n // 2 + 1
    _, _, e, _ = orc.process_window(frame, g)
    scale = np.linalg.norm(exp_in)
    assert np.linalg.norm(e - exp_in) / scale < 1e-10
    # the rejected components carry comparable power: dropping the window rule would be seen
    assert np.linalg.norm(exp_out) / scale > 0.3
