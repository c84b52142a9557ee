"""Every kernel variant against the FP64 oracle: the fused kernel that transforms every column (DH_VARIANT_FUSED,
the default for 128 x 128 windows), the group-transform fused kernel (DH_VARIANT_FUSED_GROUPS) and the
column-pruned fused kernel (DH_VARIANT_FUSED_PRUNED), both for 64 x 64 fields with the FP32 overlap, and the
three-kernel generic path (DH_VARIANT_GENERIC), on the geometries and options that reach each one's special
cases.  Bars as the other parity tests: field and coefficient relative L2 <= 1e-5 per
(frame, polarisation).
"""
import numpy as np
import pytest

from gpu_util import COEF_TOL, FIELD_TOL, rel_l2, run_library
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu

PRUNED, FUSED, GENERIC, GROUPS = 2, 1, 3, 4
PX = 20e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(setup, frames, out):
    f_ref, c_ref = orc.process_batch(frames, setup)
    if out["fields"] is not None:
        assert np.all(np.isfinite(out["fields"]))
        ef = rel_l2(out["fields"], f_ref)
        assert ef.max() <= FIELD_TOL, ef
    if out["coefs"] is not None:
        assert np.all(np.isfinite(out["coefs"]))
        ec = rel_l2(out["coefs"], c_ref)
        assert ec.max() <= COEF_TOL, ec


def _cases():
    b = syn.setup_batching()
    return {
        "batching": b,
        "f32_frames": syn.with_(b, dtype="f32"),
        "odd_origin": syn.with_(b, beam_centre=[(81.2 * PX, 128.0 * PX), (240.0 * PX, 129.3 * PX)]),
        "subpixel_defocus": syn.with_(b, beam_centre=[(80.37 * PX, 127.62 * PX), (239.51 * PX, 128.49 * PX)],
                                      defocus=[0.8, -1.3]),
        "g16": syn.with_(b, group_count=16, signal_groups=9),
        "fill_factor": syn.with_(b, fill_factor=True),
        # tilts that put the box across the y wrap and the circle onto the Nyquist column
        "wrap_nyquist": syn.with_(b, tilt_deg=[(1.7, -0.35), (1.6, 2.05)]),
        "one_pol": syn.with_(b, pol_count=1, frame_w=160, beam_centre=[(80.0 * PX, 128.0 * PX)],
                             tilt_deg=[(1.5, 1.5)], defocus=[0.3], waist=[200e-6]),
    }


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("variant", [GROUPS, PRUNED, FUSED, GENERIC])
def test_variant_against_oracle(name, variant):
    s = _cases()[name]
    d = syn.make_frames(s, 4, seed=300 + variant)
    out = run_library(s, d["frames"], variant=variant)
    assert out["variant"] == variant
    _check(s, d["frames"], out)


@pytest.mark.parametrize("variant", [GROUPS, PRUNED])
def test_reference_calibration_and_lg_basis(variant):
    s0 = syn.setup_batching()
    cal, amp = syn.reference_profile(s0, sigma_fraction=0.2, floor=300)
    s = syn.with_(s0, ref_amplitude=amp, ref_cal=cal)
    d = syn.make_frames(s, 3, seed=311)
    out = run_library(s, d["frames"], variant=variant)
    assert out["variant"] == variant
    _check(s, d["frames"], out)
    s_lg = syn.with_(s0, basis="lg")
    d2 = syn.make_frames(s_lg, 3, seed=312)
    out = run_library(s_lg, d2["frames"], variant=variant)
    _check(s_lg, d2["frames"], out)


@pytest.mark.parametrize("variant", [GROUPS, PRUNED])
def test_partial_outputs_and_no_basis(variant):
    s = syn.setup_batching()
    d = syn.make_frames(s, 3, seed=313)
    _check(s, d["frames"], run_library(s, d["frames"], variant=variant, coefs=False))
    _check(s, d["frames"], run_library(s, d["frames"], variant=variant, fields=False))
    s0 = syn.with_(s, group_count=0)
    out = run_library(s0, d["frames"], variant=variant)
    assert out["modes"] == 0 and out["coefs"] is None
    _check(s0, d["frames"], out)


def test_variants_agree_and_are_deterministic():
    s = syn.setup_batching()
    d = syn.make_frames(s, 9, seed=314)
    a = run_library(s, d["frames"], variant=PRUNED)
    a2 = run_library(s, d["frames"], variant=PRUNED)
    g = run_library(s, d["frames"], variant=GROUPS)
    g2 = run_library(s, d["frames"], variant=GROUPS)
    b = run_library(s, d["frames"], variant=FUSED)
    c = run_library(s, d["frames"], variant=GENERIC)
    assert np.array_equal(a["fields"], a2["fields"]) and np.array_equal(a["coefs"], a2["coefs"])
    assert np.array_equal(g["fields"], g2["fields"]) and np.array_equal(g["coefs"], g2["coefs"])
    for o in (g, b, c):
        assert rel_l2(a["fields"], o["fields"]).max() <= FIELD_TOL
        assert rel_l2(a["coefs"], o["coefs"]).max() <= COEF_TOL


def test_pruned_and_groups_fall_back_where_they_do_not_apply():
    # 32 x 32 fields: the fused kernel; a circle of 57 bins across inside the half plane (more than 48 kept
    # columns): the fused kernel for the pruned variant, the group variant itself (it has no column limit)
    b = syn.setup_batching()
    for s in (syn.with_(b, ifft_size=32), syn.with_(b, radius_deg=0.45 * syn.w_max_deg(), ifft_size=64,
                                                     tilt_deg=[(1.1, 1.1), (1.1, 1.1)])):
        d = syn.make_frames(s, 2, seed=315)
        out = run_library(s, d["frames"], variant=PRUNED)
        assert out["variant"] == FUSED
        _check(s, d["frames"], out)
        out = run_library(s, d["frames"], variant=GROUPS)
        assert out["variant"] == (FUSED if s.ifft_size == 32 else GROUPS)
        _check(s, d["frames"], out)
    # split-BF16 overlap at 64 x 64: the fused kernel's tensor-core variant, not the pruned or the group one
    d = syn.make_frames(b, 2, seed=316)
    assert run_library(b, d["frames"], variant=PRUNED, precision=1)["variant"] == FUSED
    assert run_library(b, d["frames"], variant=GROUPS, precision=1)["variant"] == FUSED
    assert run_library(b, d["frames"], precision=1)["variant"] == FUSED


@pytest.mark.parametrize("variant", [GROUPS, PRUNED])
def test_full_size_batching_sampled(variant):
    """The 1000-frame batching step through the kernel's persistent grid; sampled frames against the oracle,
    every frame finite."""
    s = syn.setup_batching()
    distinct = syn.make_frames(s, 8, seed=317)["frames"]
    frames = np.ascontiguousarray(distinct[np.arange(1000) % 8])
    out = run_library(s, frames, variant=variant)
    assert out["variant"] == variant
    assert np.all(np.isfinite(out["fields"])) and np.all(np.isfinite(out["coefs"]))
    idx = [0, 5, 499, 998, 999]
    f_ref, c_ref = orc.process_batch(frames[idx], s)
    assert rel_l2(out["fields"][idx], f_ref).max() <= FIELD_TOL
    assert rel_l2(out["coefs"][idx], c_ref).max() <= COEF_TOL
    # frames with the same content give bit-identical results wherever they sit in the batch
    assert np.array_equal(out["fields"][3], out["fields"][11]) and np.array_equal(out["coefs"][3], out["coefs"][995])
