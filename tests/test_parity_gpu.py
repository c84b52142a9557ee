"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded frames.

Bars (per frame and polarisation): field relative L2 <= 1e-5 and coefficient relative L2 <= 1e-5 on the
FP32 path; the masked Fourier window <= 2e-6.  Outputs are NaN-poisoned before each call.
"""
import math

import numpy as np
import pytest

from gpu_util import (COEF_TOL, FIELD_TOL, SPLIT_COEF_TOL, WINDOW_TOL, oracle_window, rel_l2, run_library)
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(setup, frames, out, field_tol=FIELD_TOL, coef_tol=COEF_TOL):
    f_ref, c_ref = orc.process_batch(frames, setup)
    if out["fields"] is not None:
        ef = rel_l2(out["fields"], f_ref)
        assert np.all(np.isfinite(out["fields"]))
        assert ef.max() <= field_tol, ef
    if out["coefs"] is not None:
        ec = rel_l2(out["coefs"], c_ref)
        assert np.all(np.isfinite(out["coefs"]))
        assert ec.max() <= coef_tol, ec
    return f_ref, c_ref


def test_plain_128_f32():
    s = syn.setup_plain()
    d = syn.make_frames(s, 1)
    out = run_library(s, d["frames"], window=True)        # generic multi-kernel path
    _check(s, d["frames"], out)
    w_ref = oracle_window(d["frames"][0], orc.pol_geometry(s, 0))
    assert rel_l2(out["window"][:, :1], w_ref[None, None])[0, 0] <= WINDOW_TOL
    _check(s, d["frames"], run_library(s, d["frames"]))   # fused single-kernel path


def test_plain_with_paper_size_rule():
    s = syn.with_(syn.setup_plain(), ifft_size=0)     # 48 x 48 field, radix 16 x 3
    d = syn.make_frames(s, 2, seed=9)
    out = run_library(s, d["frames"])
    assert out["m"] == 48
    _check(s, d["frames"], out)


def test_batching_320x256_u16_two_pols():
    s = syn.setup_batching()
    d = syn.make_frames(s, 5)
    _check(s, d["frames"], run_library(s, d["frames"]))   # fused single-kernel path
    out = run_library(s, d["frames"], window=True)        # generic multi-kernel path
    _check(s, d["frames"], out)
    for p in range(2):
        w_ref = oracle_window(d["frames"][3], orc.pol_geometry(s, p))
        assert rel_l2(out["window"][3:4, p:p + 1], w_ref[None, None])[0, 0] <= WINDOW_TOL


def test_precision_640x512_fp32_overlap():
    s = syn.setup_precision()
    d = syn.make_frames(s, 2)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)


def test_large_window_512_m176_g20():
    s = syn.setup_large_batch()
    d = syn.make_frames(s, 1)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)


@pytest.mark.parametrize("kind", list(syn.SERVING_KINDS))
def test_serving_geometries(kind):
    rng = np.random.default_rng(list(syn.SERVING_KINDS).index(kind) + 100)
    s = syn.serving_geometry(kind, rng)
    d = syn.make_frames(s, 1, seed=21)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)


def test_largest_window_and_field_1024_m336():
    s = syn.serving_geometry("1024x1024_1pol", np.random.default_rng(0))
    wm = syn.w_max_deg()
    s = syn.with_(s, radius_deg=0.32 * wm, tilt_deg=[(3 * 0.32 * wm / math.sqrt(2),) * 2], group_count=16)
    d = syn.make_frames(s, 1, seed=22)
    out = run_library(s, d["frames"])
    assert out["m"] == 336
    _check(s, d["frames"], out)


def test_box_wraps_in_y_and_crosses_nyquist():
    base = syn.setup_plain()
    for ty in (-1.0, 1.9, 2.2):
        s = syn.with_(base, tilt_deg=[(1.0, ty)], ifft_size=48)
        d = syn.make_frames(s, 1, seed=int(ty * 10) + 50)
        out = run_library(s, d["frames"])
        _check(s, d["frames"], out)


def test_subpixel_beam_centre_and_defocus():
    base = syn.setup_batching()
    s = syn.with_(base, beam_centre=[(80.37 * 20e-6, 127.62 * 20e-6), (239.51 * 20e-6, 128.49 * 20e-6)],
                  defocus=[0.8, -1.3])
    d = syn.make_frames(s, 2, seed=31)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)


def test_odd_window_origin_unaligned_pixel_pairs():
    """Odd window origins (and an odd frame width) force the scalar pixel loads of the fused path."""
    base = syn.setup_batching()
    s = syn.with_(base, beam_centre=[(81.2 * 20e-6, 128.0 * 20e-6), (240.0 * 20e-6, 129.3 * 20e-6)])
    d = syn.make_frames(s, 2, seed=32)
    _check(s, d["frames"], run_library(s, d["frames"]))
    s2 = syn.with_(syn.setup_plain(), frame_w=131, beam_centre=[(64.6 * 20e-6, 64.0 * 20e-6)])
    d2 = syn.make_frames(s2, 2, seed=33)
    _check(s2, d2["frames"], run_library(s2, d2["frames"]))


def test_fused_and_generic_paths_agree():
    s = syn.setup_batching()
    d = syn.make_frames(s, 7, seed=34)
    a = run_library(s, d["frames"])
    b = run_library(s, d["frames"], window=True)
    assert rel_l2(a["fields"], b["fields"]).max() <= FIELD_TOL
    assert rel_l2(a["coefs"], b["coefs"]).max() <= COEF_TOL


def test_tiny_radius_mostly_empty_rows():
    s = syn.with_(syn.setup_plain(), radius_deg=0.05, ifft_size=32)
    d = syn.make_frames(s, 1, seed=41)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)


def test_small_window_64():
    s = syn.with_(syn.setup_plain(), frame_w=64, frame_h=64, window=64, beam_centre=[(32 * 20e-6, 32 * 20e-6)],
                  ifft_size=32, group_count=3, waist=[80e-6], signal_groups=3)
    d = syn.make_frames(s, 3, seed=42)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)


def test_no_basis_and_partial_outputs():
    s = syn.with_(syn.setup_batching(), group_count=0)
    d = syn.make_frames(s, 2, seed=43)
    out = run_library(s, d["frames"])
    assert out["coefs"] is None and out["modes"] == 0
    _check(s, d["frames"], out)
    s2 = syn.setup_batching()
    o1 = run_library(s2, d["frames"], fields=False)
    o2 = run_library(s2, d["frames"], coefs=False)
    assert o1["fields"] is None and o2["coefs"] is None
    _check(s2, d["frames"], o1)
    _check(s2, d["frames"], o2)


def test_batch_below_one_processes_one_frame():
    s = syn.setup_plain()
    d = syn.make_frames(s, 1, seed=44)
    out = run_library(s, d["frames"], batch=0)
    _check(s, d["frames"], out)


def test_deterministic_bitwise():
    s = syn.setup_batching()
    d = syn.make_frames(s, 3, seed=45)
    a = run_library(s, d["frames"])
    b = run_library(s, d["frames"])
    assert np.array_equal(a["fields"].view(np.uint32), b["fields"].view(np.uint32))
    assert np.array_equal(a["coefs"].view(np.uint32), b["coefs"].view(np.uint32))


def test_full_size_batching_sampled():
    """The bench's workload (1000 frames of 320x256, one call); sampled frames checked against the oracle."""
    s = syn.setup_batching()
    d = syn.make_frames(s, 1000)
    out = run_library(s, d["frames"])
    idx = [0, 1, 499, 998, 999]
    f_ref, c_ref = orc.process_batch(d["frames"][idx], s)
    assert rel_l2(out["fields"][idx], f_ref).max() <= FIELD_TOL
    assert rel_l2(out["coefs"][idx], c_ref).max() <= COEF_TOL
    assert np.all(np.isfinite(out["fields"])) and np.all(np.isfinite(out["coefs"]))


def test_score_settings_matches_oracle():
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.with_(syn.setup_batching(), group_count=5)
    d = syn.make_frames(s, 3, seed=46)
    cand = syn.candidate_settings(s, 4, seed=47)
    ref = orc.score_settings(d["frames"], s, cand["tilt_deg"], cand["defocus"], cand["waist"])
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        fr = torch.from_numpy(d["frames"]).cuda()
        pw = torch.full((3, 4), float("nan"), dtype=torch.float32, device="cuda")
        sets = [dh.make_setting(cand["tilt_deg"][k], cand["defocus"][k], cand["waist"][k]) for k in range(4)]
        dh.dh_score_settings(h, fr, dh.DH_DTYPE_U16, 3, sets, pw)
        torch.cuda.synchronize()
        got = pw.cpu().numpy()
    finally:
        dh.dh_destroy(h)
    assert np.all(np.abs(got - ref) / ref <= 2 * COEF_TOL), (got, ref)


# --------------------------------------------------------------------------------- split-BF16 tensor-core overlap

SPLIT = 1   # DH_PRECISION_SPLIT_BF16


@pytest.mark.parametrize("name,frames", [("precision", 2), ("large_batch", 1), ("plain", 2)])
def test_split_bf16_overlap(name, frames):
    s = syn.WORKLOADS[name]()
    d = syn.make_frames(s, frames, seed=60)
    out = run_library(s, d["frames"], precision=SPLIT)
    _check(s, d["frames"], out, coef_tol=SPLIT_COEF_TOL)
    plain = run_library(s, d["frames"])
    # the split overlap agrees with the FP32 overlap within the split bar, and its fields are the FP32 fields
    assert rel_l2(out["coefs"], plain["coefs"]).max() <= SPLIT_COEF_TOL
    assert rel_l2(out["fields"], plain["fields"]).max() <= FIELD_TOL


@pytest.mark.parametrize("base,kw", [("batching", {}), ("plain", {"ifft_size": 64, "group_count": 16, "signal_groups": 9}),
                                     ("batching", {"group_count": 16, "signal_groups": 9})])
def test_split_bf16_fused_path(base, kw):
    # 128 x 128 windows with 64 x 64 fields run the fused kernel's tensor-core variant (uint16 frames of the
    # batching geometry, float32 frames of the plain one, G up to 16); the window output forces the generic
    # path, whose split-BF16 overlap is the other kernel
    s = syn.with_(syn.WORKLOADS[base](), **kw)
    d = syn.make_frames(s, 5, seed=63)
    out = run_library(s, d["frames"], precision=SPLIT)
    _check(s, d["frames"], out, coef_tol=SPLIT_COEF_TOL)
    gen = run_library(s, d["frames"], precision=SPLIT, window=True)
    fp32 = run_library(s, d["frames"])
    assert rel_l2(out["coefs"], gen["coefs"]).max() <= SPLIT_COEF_TOL
    assert rel_l2(out["coefs"], fp32["coefs"]).max() <= SPLIT_COEF_TOL
    # the fields do not depend on the overlap's precision
    assert rel_l2(out["fields"], fp32["fields"]).max() <= FIELD_TOL
    again = run_library(s, d["frames"], precision=SPLIT)
    assert np.array_equal(out["coefs"].view(np.uint32), again["coefs"].view(np.uint32))


def test_split_bf16_serving_geometry_and_determinism():
    s = syn.serving_geometry("512x512_2pol", np.random.default_rng(61))
    d = syn.make_frames(s, 3, seed=62)
    a = run_library(s, d["frames"], precision=SPLIT)
    b = run_library(s, d["frames"], precision=SPLIT)
    _check(s, d["frames"], a, coef_tol=SPLIT_COEF_TOL)
    assert np.array_equal(a["coefs"].view(np.uint32), b["coefs"].view(np.uint32))


def _score(setup, frames, cand, precision=0):
    import torch
    import paper_2204_02348_gb300 as dh
    B, S = frames.shape[0], cand["tilt_deg"].shape[0]
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        dh.dh_set_precision(h, precision)
        fr = torch.from_numpy(frames).cuda()
        pw = torch.full((B, S), float("nan"), dtype=torch.float32, device="cuda")
        sets = [dh.make_setting(cand["tilt_deg"][k], cand["defocus"][k], cand["waist"][k]) for k in range(S)]
        dt = dh.DH_DTYPE_U16 if frames.dtype == np.uint16 else dh.DH_DTYPE_F32
        dh.dh_score_settings(h, fr, dt, B, sets, pw)
        torch.cuda.synchronize()
        return pw.cpu().numpy()
    finally:
        dh.dh_destroy(h)


@pytest.mark.parametrize("precision,tol", [(0, 2 * COEF_TOL), (1, 2 * SPLIT_COEF_TOL)])
def test_score_large_geometry_superset(precision, tol):
    s = syn.setup_large_batch()
    d = syn.make_frames(s, 2, seed=70)
    cand = syn.candidate_settings(s, 6, seed=71)
    ref = orc.score_settings(d["frames"], s, cand["tilt_deg"], cand["defocus"], cand["waist"])
    got = _score(s, d["frames"], cand, precision)
    assert np.all(np.abs(got - ref) / ref <= tol), (got, ref)


def test_score_candidates_outside_one_superset_fall_back():
    s = syn.with_(syn.setup_plain(), ifft_size=64, group_count=4)
    d = syn.make_frames(s, 2, seed=72)
    tilt = np.array([[[1.0, 1.0]], [[1.0, -1.5]], [[1.2, 0.8]]])
    cand = {"tilt_deg": tilt, "defocus": np.array([[0.0], [0.5], [-0.3]]), "waist": np.array([[150e-6], [140e-6], [160e-6]])}
    ref = orc.score_settings(d["frames"], s, cand["tilt_deg"], cand["defocus"], cand["waist"])
    got = _score(s, d["frames"], cand)
    assert np.all(np.abs(got - ref) / ref <= 2 * COEF_TOL), (got, ref)


def test_fill_factor_correction_parity():
    s = syn.with_(syn.setup_batching(), fill_factor=True)
    d = syn.make_frames(s, 3, seed=80)
    _check(s, d["frames"], run_library(s, d["frames"]))                # fused path
    _check(s, d["frames"], run_library(s, d["frames"], window=True))   # generic path
    s2 = syn.with_(syn.setup_precision(), fill_factor=True)
    d2 = syn.make_frames(s2, 1, seed=81)
    _check(s2, d2["frames"], run_library(s2, d2["frames"]))


# ----------------------------------------------------------------------------- LG and custom bases


@pytest.mark.parametrize("name,frames", [("batching", 3), ("precision", 1), ("large_batch", 1)])
def test_lg_basis_against_direct_lg_overlaps(name, frames):
    # the oracle overlaps the field with LG modes evaluated from Laguerre polynomials; the library applies
    # its closed-form HG -> LG matrix to the HG coefficients
    s = syn.with_(syn.WORKLOADS[name](), basis="lg")
    d = syn.make_frames(s, frames, seed=120)
    out = run_library(s, d["frames"])
    assert out["modes"] == len(orc.lg_mode_list(s.group_count))
    _check(s, d["frames"], out)
    _check(s, d["frames"], run_library(s, d["frames"], window=True))          # generic path
    _check(s, d["frames"], run_library(s, d["frames"], precision=1), coef_tol=SPLIT_COEF_TOL)


def test_lg_total_power_equals_hg_total_power():
    s = syn.setup_batching()
    d = syn.make_frames(s, 4, seed=121)
    hg = run_library(s, d["frames"])["coefs"]
    lg = run_library(syn.with_(s, basis="lg"), d["frames"])["coefs"]
    p_hg = np.sum(np.abs(hg.astype(np.complex128)) ** 2, axis=-1)
    p_lg = np.sum(np.abs(lg.astype(np.complex128)) ** 2, axis=-1)
    assert np.max(np.abs(p_lg - p_hg) / p_hg) <= 1e-5


@pytest.mark.parametrize("modes_in_extra", [7, -4])
def test_custom_basis_more_and_fewer_inputs_than_hg_modes(modes_in_extra):
    rng = np.random.default_rng(122)
    s = syn.setup_batching()
    modes_hg = s.group_count * (s.group_count + 1) // 2
    t = (rng.standard_normal((23, modes_hg + modes_in_extra))
         + 1j * rng.standard_normal((23, modes_hg + modes_in_extra))) / math.sqrt(modes_hg)
    sc = syn.with_(s, basis="custom", basis_transform=t)
    d = syn.make_frames(sc, 3, seed=123)
    out = run_library(sc, d["frames"])
    assert out["modes"] == 23
    _check(sc, d["frames"], out)
    _check(sc, d["frames"], run_library(sc, d["frames"], window=True))


# ----------------------------------------------------------------------------- reference calibration


def _calibrated(setup, sigma=0.15):
    cal, amp = syn.reference_profile(setup, sigma_fraction=sigma, floor=200)
    return syn.with_(setup, ref_amplitude=amp, ref_cal=cal)


def test_reference_calibration_parity():
    s = _calibrated(syn.setup_batching())
    d = syn.make_frames(s, 3, seed=150)
    _check(s, d["frames"], run_library(s, d["frames"]))
    _check(s, d["frames"], run_library(s, d["frames"], window=True))
    s2 = _calibrated(syn.setup_precision(), sigma=0.2)
    d2 = syn.make_frames(s2, 1, seed=151)
    _check(s2, d2["frames"], run_library(s2, d2["frames"]))
    _check(s2, d2["frames"], run_library(s2, d2["frames"], precision=1), coef_tol=SPLIT_COEF_TOL)


def test_reference_calibration_scoring():
    s = _calibrated(syn.setup_batching())
    d = syn.make_frames(s, 2, seed=152)
    cand = syn.candidate_settings(s, 5, seed=153)
    ref = orc.score_settings(d["frames"], s, cand["tilt_deg"], cand["defocus"], cand["waist"])
    got = _score(s, d["frames"], cand)
    assert np.all(np.abs(got - ref) / ref <= 2 * COEF_TOL), (got, ref)


# ----------------------------------------------------------------------------- every fused-kernel instantiation


@pytest.mark.parametrize("m,dtype", [(32, "u16"), (48, "u16"), (64, "u16"), (32, "f32"), (48, "f32"), (64, "f32")])
def test_fused_instantiations_against_oracle(m, dtype):
    # the fused kernel is compiled per field size and pixel type (uint16: two blocks per SM of 256 or 512
    # threads; float32: one 512-thread block); G = 16 is its largest group count
    s = syn.with_(syn.setup_batching(), ifft_size=m, dtype=dtype, group_count=16, signal_groups=9)
    d = syn.make_frames(s, 5, seed=170 + m)
    assert d["frames"].dtype == (np.uint16 if dtype == "u16" else np.float32)
    out = run_library(s, d["frames"])
    _check(s, d["frames"], out)
    # the same frames through the generic path (window output forces it) agree as well
    _check(s, d["frames"], run_library(s, d["frames"], window=True))


# ----------------------------------------------------------------------------- full-size configurations, sampled


def _tiled(setup, count, distinct, seed):
    """count frames cycling over `distinct` seeded frames (the work per frame is the same; generating every
    frame of the large configurations would dominate the test)."""
    d = syn.make_frames(setup, distinct, seed=seed)
    idx = np.arange(count) % distinct
    return d["frames"], np.ascontiguousarray(d["frames"][idx])


@pytest.mark.parametrize("precision,coef_tol", [(0, COEF_TOL), (1, SPLIT_COEF_TOL)])
def test_full_size_precision_sampled(precision, coef_tol):
    """The precision configuration at full size (1024 frames of 640x512, two 256x256 windows, 120 modes) in
    one call, as the bench runs it; sampled frames against the oracle."""
    s = syn.setup_precision()
    distinct, frames = _tiled(s, 1024, 16, seed=180)
    out = run_library(s, frames, precision=precision)
    assert np.all(np.isfinite(out["fields"])) and np.all(np.isfinite(out["coefs"]))
    idx = [0, 17, 511, 1023]
    f_ref, c_ref = orc.process_batch(distinct[[i % 16 for i in idx]], s)
    assert rel_l2(out["fields"][idx], f_ref).max() <= FIELD_TOL
    assert rel_l2(out["coefs"][idx], c_ref).max() <= coef_tol


def test_full_size_large_scoring_sampled():
    """The large scoring configuration at full size (2000 frames of 1280x1024, two 512x512 windows, 210 modes,
    64 candidates, split-BF16) in one call; sampled (frame, candidate) powers against the oracle."""
    s = syn.setup_large_batch()
    distinct, frames = _tiled(s, 2000, 8, seed=181)
    cand = syn.candidate_settings(s, 64)
    got = _score(s, frames, cand, precision=1)
    assert got.shape == (2000, 64) and np.all(np.isfinite(got))
    for b, k in [(0, 0), (1001, 37), (1999, 63)]:
        ref = orc.score_settings(distinct[b % 8][None], s, cand["tilt_deg"][k:k + 1], cand["defocus"][k:k + 1],
                                 cand["waist"][k:k + 1])[0, 0]
        assert abs(got[b, k] - ref) / ref <= 2 * SPLIT_COEF_TOL, (b, k, got[b, k], ref)


# ----------------------------------------------------------------------------- odd-prime inverse radices
@pytest.mark.parametrize("kind,m", [("256x256_1pol", 80), ("256x256_1pol", 112), ("256x256_1pol", 176),
                                    ("256x256_1pol", 208), ("1024x1024_1pol", 272), ("1024x1024_1pol", 304)])
def test_odd_prime_field_sizes(kind, m):
    # M = 16 x {5, 7, 11, 13, 17, 19}: every odd-prime butterfly of the inverse transforms (runtime radix plans,
    # and the compile-time plan at 176), FP32; the split-BF16 overlap where its kernel takes the size (M <= 192)
    s = syn.with_(syn.serving_geometry(kind, np.random.default_rng(400 + m)), ifft_size=m)
    d = syn.make_frames(s, 2, seed=401 + m)
    out = run_library(s, d["frames"])
    assert out["m"] == m
    _check(s, d["frames"], out)
    if m <= 192:
        _check(s, d["frames"], run_library(s, d["frames"], precision=1, fields=False), coef_tol=SPLIT_COEF_TOL)


# ----------------------------------------------------------------------------- fused split-BF16 with the optional stages
@pytest.mark.parametrize("stage", ["lg", "fill_factor", "calibration"])
def test_split_bf16_fused_optional_stages(stage):
    # the tensor-core variant of the fused kernel under the LG output basis (k_basis after it), the fill-factor
    # correction (in its phase tables) and the reference calibration (applied as the window is read)
    base = syn.setup_batching()
    if stage == "lg":
        s = syn.with_(base, basis="lg")
    elif stage == "fill_factor":
        s = syn.with_(base, fill_factor=True)
    else:
        s = _calibrated(base)
    d = syn.make_frames(s, 3, seed=160)
    out = run_library(s, d["frames"], precision=SPLIT)
    _check(s, d["frames"], out, coef_tol=SPLIT_COEF_TOL)


def test_split_bf16_fused_host_pipeline():
    # the host-buffer entry point runs the same fused tensor-core kernel per chunk: bit-identical results
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.setup_batching()
    fr = syn.make_frames(s, 40, seed=161)["frames"]
    dev = run_library(s, fr, precision=SPLIT)
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        dh.dh_set_precision(h, SPLIT)
        hin = torch.from_numpy(fr).pin_memory()
        f = torch.empty(dev["fields"].shape, dtype=torch.complex64).pin_memory()
        c = torch.empty(dev["coefs"].shape, dtype=torch.complex64).pin_memory()
        dh.dh_process_batch_host(h, hin, dh.DH_DTYPE_U16, fr.shape[0], f, c)
    finally:
        dh.dh_destroy(h)
    assert np.array_equal(f.numpy().view(np.uint32), dev["fields"].view(np.uint32))
    assert np.array_equal(c.numpy().view(np.uint32), dev["coefs"].view(np.uint32))
