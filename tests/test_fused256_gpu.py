"""The 256 x 256 fused kernel (k_fused256: 96 x 96 fields, uint16 frames, FP32 overlap or its split-BF16
tensor-core variant, up to 16 HG groups) against the oracle: window positions (odd origins, frame edges, sub-pixel centres), box positions (wrapping
below bin 0, crossing Nyquist), the optional stages, partial outputs, batch sizes around the persistent grid,
and the rules that send other frames to the generic path."""
import math

import numpy as np
import pytest

from gpu_util import COEF_TOL, FIELD_TOL, SPLIT_COEF_TOL, rel_l2, run_library
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu

PX = syn.PIXEL


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dh():
    import paper_2204_02348_gb300 as dh
    return dh


def _check(setup, frames, out, idx=None, coef_tol=COEF_TOL):
    sel = frames if idx is None else frames[idx]
    f_ref, c_ref = orc.process_batch(sel, setup)
    if out["fields"] is not None:
        f = out["fields"] if idx is None else out["fields"][idx]
        assert np.all(np.isfinite(f))
        ef = rel_l2(f, f_ref)
        assert ef.max() <= FIELD_TOL, ef
    if out["coefs"] is not None:
        c = out["coefs"] if idx is None else out["coefs"][idx]
        assert np.all(np.isfinite(c))
        ec = rel_l2(c, c_ref)
        assert ec.max() <= coef_tol, ec


def test_precision_geometry_selects_the_fused_kernel():
    dh = _dh()
    s = syn.setup_precision()
    d = syn.make_frames(s, 3, seed=400)
    out = run_library(s, d["frames"])
    assert out["variant"] == dh.DH_VARIANT_FUSED and out["m"] == 96 and out["modes"] == 120
    _check(s, d["frames"], out)


@pytest.mark.parametrize("centres", [
    # odd window origins: staging offsets 3 and 6 within the 16-byte boxes
    [(163.4, 255.6), (477.7, 256.4)],
    # the frame's edges: origin (0, 0), and (384, 256) whose second box runs 8 columns past the frame
    [(128.0, 128.0), (512.0, 384.0)],
    # sub-pixel centres either side of the half
    [(200.51, 300.49), (420.49, 211.51)],
])
def test_window_positions(centres):
    s = syn.with_(syn.setup_precision(), beam_centre=[(x * PX, y * PX) for x, y in centres])
    d = syn.make_frames(s, 2, seed=401)
    _check(s, d["frames"], run_library(s, d["frames"]))


@pytest.mark.parametrize("tilt", [0.35, 1.2, 2.15])
def test_box_positions(tilt):
    """Small tilts put the 96-bin box across bin 0 (first box bin negative), large ones across Nyquist."""
    base = syn.setup_precision()
    s = syn.with_(base, tilt_deg=[(tilt, tilt + 0.13), (tilt + 0.07, tilt - 0.05)])
    d = syn.make_frames(s, 2, seed=402)
    _check(s, d["frames"], run_library(s, d["frames"]))


def test_defocus_and_fill_factor():
    s = syn.with_(syn.setup_precision(), defocus=[0.7, -1.1], fill_factor=True)
    d = syn.make_frames(s, 2, seed=403)
    _check(s, d["frames"], run_library(s, d["frames"]))


def test_reference_calibration():
    cal, amp = syn.reference_profile(syn.setup_precision(), sigma_fraction=0.2, floor=200)
    s = syn.with_(syn.setup_precision(), ref_amplitude=amp, ref_cal=cal)
    d = syn.make_frames(s, 2, seed=404)
    _check(s, d["frames"], run_library(s, d["frames"]))


@pytest.mark.parametrize("groups", [0, 1, 16])
def test_group_counts(groups):
    s = syn.with_(syn.setup_precision(), group_count=groups, signal_groups=max(groups, 1))
    d = syn.make_frames(s, 2, seed=405 + groups)
    out = run_library(s, d["frames"])
    if groups == 0:
        assert out["coefs"] is None and out["modes"] == 0
    _check(s, d["frames"], out)


def test_one_polarisation_and_lg_basis():
    base = syn.setup_precision()
    s = syn.with_(base, pol_count=1, beam_centre=[(300.2 * PX, 260.7 * PX)], tilt_deg=base.tilt_deg[:1],
                  defocus=[0.3], waist=base.waist[:1])
    d = syn.make_frames(s, 3, seed=410)
    _check(s, d["frames"], run_library(s, d["frames"]))
    s2 = syn.with_(base, basis="lg")
    d2 = syn.make_frames(s2, 2, seed=411)
    _check(s2, d2["frames"], run_library(s2, d2["frames"]))


def test_partial_outputs():
    s = syn.setup_precision()
    d = syn.make_frames(s, 2, seed=412)
    o1 = run_library(s, d["frames"], fields=False)
    o2 = run_library(s, d["frames"], coefs=False)
    assert o1["fields"] is None and o2["coefs"] is None
    _check(s, d["frames"], o1)
    _check(s, d["frames"], o2)


@pytest.mark.parametrize("count", [1, 77, 230])
def test_batches_around_the_persistent_grid(count):
    """One frame; fewer frames than blocks per polarisation; several windows per block (ragged last wave).
    Sampled frames against the oracle, every frame finite."""
    s = syn.setup_precision()
    distinct = syn.make_frames(s, 5, seed=413)["frames"]
    frames = np.ascontiguousarray(distinct[np.arange(count) % 5])
    out = run_library(s, frames)
    assert np.all(np.isfinite(out["fields"])) and np.all(np.isfinite(out["coefs"]))
    idx = sorted({0, count // 2, count - 1})
    f_ref, c_ref = orc.process_batch(distinct[[i % 5 for i in idx]], s)
    assert rel_l2(out["fields"][idx], f_ref).max() <= FIELD_TOL
    assert rel_l2(out["coefs"][idx], c_ref).max() <= COEF_TOL
    # equal frames give equal outputs wherever they sit in the batch
    for i in range(5, count, 37):
        assert np.array_equal(out["fields"][i], out["fields"][i % 5])
        assert np.array_equal(out["coefs"][i], out["coefs"][i % 5])


def test_float_frames_and_held_variant_run_the_generic_path():
    dh = _dh()
    s = syn.with_(syn.setup_precision(), dtype="f32", noise="gauss")
    d = syn.make_frames(s, 2, seed=414)
    assert d["frames"].dtype == np.float32
    _check(s, d["frames"], run_library(s, d["frames"]))
    s16 = syn.setup_precision()
    d16 = syn.make_frames(s16, 2, seed=415)
    fused = run_library(s16, d16["frames"])
    generic = run_library(s16, d16["frames"], variant=dh.DH_VARIANT_GENERIC)
    assert generic["variant"] == dh.DH_VARIANT_GENERIC
    _check(s16, d16["frames"], generic)
    assert rel_l2(fused["fields"], generic["fields"]).max() <= FIELD_TOL
    assert rel_l2(fused["coefs"], generic["coefs"]).max() <= COEF_TOL
    # every other variant request resolves to the fused kernel at this size
    for v in (dh.DH_VARIANT_FUSED_PRUNED, dh.DH_VARIANT_FUSED_GROUPS):
        assert run_library(s16, d16["frames"][:1], variant=v)["variant"] == dh.DH_VARIANT_FUSED


def test_deterministic_bitwise():
    s = syn.setup_precision()
    d = syn.make_frames(s, 4, seed=416)
    a = run_library(s, d["frames"])
    b = run_library(s, d["frames"])
    assert np.array_equal(a["fields"], b["fields"]) and np.array_equal(a["coefs"], b["coefs"])


# ----------------------------------------------------------------------------- split-BF16 (tensor-core y contraction)
SPLIT = 1


def test_split_bf16_selects_the_fused_kernel():
    dh = _dh()
    s = syn.setup_precision()
    d = syn.make_frames(s, 3, seed=420)
    out = run_library(s, d["frames"], precision=SPLIT)
    assert out["variant"] == dh.DH_VARIANT_FUSED
    _check(s, d["frames"], out, coef_tol=SPLIT_COEF_TOL)
    # the fields are the FP32 path's (only the overlap differs)
    fp32 = run_library(s, d["frames"])
    assert np.array_equal(out["fields"], fp32["fields"])
    assert rel_l2(out["coefs"], fp32["coefs"]).max() <= SPLIT_COEF_TOL


@pytest.mark.parametrize("groups", [0, 1, 16])
def test_split_bf16_group_counts(groups):
    s = syn.with_(syn.setup_precision(), group_count=groups, signal_groups=max(groups, 1))
    d = syn.make_frames(s, 2, seed=421 + groups)
    out = run_library(s, d["frames"], precision=SPLIT)
    _check(s, d["frames"], out, coef_tol=SPLIT_COEF_TOL)


def test_split_bf16_options_and_one_polarisation():
    base = syn.setup_precision()
    cal, amp = syn.reference_profile(base, sigma_fraction=0.2, floor=200)
    s = syn.with_(base, defocus=[0.7, -1.1], fill_factor=True, ref_amplitude=amp, ref_cal=cal,
                  beam_centre=[(163.4 * PX, 255.6 * PX), (477.7 * PX, 256.4 * PX)])
    d = syn.make_frames(s, 2, seed=425)
    _check(s, d["frames"], run_library(s, d["frames"], precision=SPLIT), coef_tol=SPLIT_COEF_TOL)
    s1 = syn.with_(base, pol_count=1, beam_centre=[(300.2 * PX, 260.7 * PX)], tilt_deg=base.tilt_deg[:1],
                   defocus=[0.3], waist=base.waist[:1], basis="lg")
    d1 = syn.make_frames(s1, 3, seed=426)
    _check(s1, d1["frames"], run_library(s1, d1["frames"], precision=SPLIT), coef_tol=SPLIT_COEF_TOL)


@pytest.mark.parametrize("count", [1, 230])
def test_split_bf16_batches_and_determinism(count):
    s = syn.setup_precision()
    distinct = syn.make_frames(s, 5, seed=427)["frames"]
    frames = np.ascontiguousarray(distinct[np.arange(count) % 5])
    a = run_library(s, frames, precision=SPLIT)
    b = run_library(s, frames, precision=SPLIT, coefs=True, fields=False)
    assert np.all(np.isfinite(a["coefs"])) and np.array_equal(a["coefs"], b["coefs"])
    idx = sorted({0, count // 2, count - 1})
    f_ref, c_ref = orc.process_batch(distinct[[i % 5 for i in idx]], s)
    assert rel_l2(a["fields"][idx], f_ref).max() <= FIELD_TOL
    assert rel_l2(a["coefs"][idx], c_ref).max() <= SPLIT_COEF_TOL
    for i in range(5, count, 37):
        assert np.array_equal(a["coefs"][i], a["coefs"][i % 5])
