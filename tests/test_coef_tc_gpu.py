"""The coefficient-only split-BF16 contraction (k_coef_tc): with no field requested, the y inverse transform, the
y correction and the y overlap run as one tensor-core contraction of the x-inverse-transformed rows.  Its
coefficients against the FP64 oracle (the split-BF16 bar, 1e-4 relative L2 per frame and polarisation) and
against the FP32 path, on field sizes of one, two and three 128-row tiles; the library's profiler shows the
kernel ran."""
import math

import numpy as np
import pytest

from gpu_util import COEF_TOL, SPLIT_COEF_TOL, rel_l2
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _coefs(setup, frames, precision):
    import torch
    import paper_2204_02348_gb300 as dh
    dev = torch.device("cuda", 0)
    fr = torch.from_numpy(np.ascontiguousarray(frames)).to(dev)
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        dh.dh_set_precision(h, precision)
        # the generic path, whose last kernel the coefficient-only contraction replaces (the fused kernels would
        # take the 256 x 256 geometries with 96 x 96 fields)
        dh.dh_set_variant(h, dh.DH_VARIANT_GENERIC)
        _, modes, _ = dh.dh_get_output_dims(h)
        B = frames.shape[0]
        c = torch.full((B, setup.pol_count, modes), complex(math.nan, math.nan), dtype=torch.complex64, device=dev)
        dh.dh_set_profiling(h, True)
        dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, B, None, c)
        torch.cuda.synchronize()
        prof = dh.dh_get_profile(h)
        return c.cpu().numpy(), set(prof)
    finally:
        dh.dh_destroy(h)


def _cases():
    rng = np.random.default_rng(501)
    pre = syn.setup_precision()
    out = {
        "precision_m96": pre,
        "precision_g24": syn.with_(pre, group_count=24, signal_groups=15),
        "large_m176": syn.setup_large_batch(),
        "serving_256": syn.serving_geometry("256x256_1pol", rng),
        "serving_512_2pol": syn.serving_geometry("512x512_2pol", rng),
        "serving_1024": syn.serving_geometry("1024x1024_1pol", rng),
    }
    # three 128-row tiles, the last one ragged (288 = 2 x 128 + 32)
    out["serving_1024_m288"] = syn.with_(out["serving_1024"], ifft_size=288)
    return out


@pytest.mark.parametrize("name", list(_cases()))
def test_coefficient_only_split_against_oracle_and_fp32(name):
    s = _cases()[name]
    frames = syn.make_frames(s, 3, seed=502)["frames"]
    c_split, kernels = _coefs(s, frames, 1)
    assert "k_coef_tc" in kernels, kernels
    c_fp32, kernels32 = _coefs(s, frames, 0)
    assert "k_coef_tc" not in kernels32
    _, c_ref = orc.process_batch(frames, s)
    assert np.all(np.isfinite(c_split))
    assert rel_l2(c_split, c_ref).max() <= SPLIT_COEF_TOL
    assert rel_l2(c_fp32, c_ref).max() <= COEF_TOL
    assert rel_l2(c_split, c_fp32).max() <= SPLIT_COEF_TOL


def test_coefficient_only_split_many_frames_sampled_and_deterministic():
    """700 precision frames: more than one scratch chunk and more windows than the grid holds at once; sampled
    frames against the oracle, repeated frames bit-identical, two runs bit-identical."""
    s = syn.setup_precision()
    distinct = syn.make_frames(s, 7, seed=503)["frames"]
    frames = np.ascontiguousarray(distinct[np.arange(700) % 7])
    c1, kernels = _coefs(s, frames, 1)
    c2, _ = _coefs(s, frames, 1)
    assert "k_coef_tc" in kernels
    assert np.array_equal(c1, c2)
    assert np.array_equal(c1[3], c1[3 + 7 * 90])
    idx = [0, 1, 350, 699]
    _, c_ref = orc.process_batch(frames[idx], s)
    assert rel_l2(c1[idx], c_ref).max() <= SPLIT_COEF_TOL


def _score(setup, frames, cand, precision):
    import torch
    import paper_2204_02348_gb300 as dh
    B, S = frames.shape[0], cand["tilt_deg"].shape[0]
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        dh.dh_set_precision(h, precision)
        fr = torch.from_numpy(np.ascontiguousarray(frames)).cuda()
        pw = torch.full((B, S), float("nan"), dtype=torch.float32, device="cuda")
        sets = [dh.make_setting(cand["tilt_deg"][k], cand["defocus"][k], cand["waist"][k]) for k in range(S)]
        dh.dh_set_profiling(h, True)
        dh.dh_score_settings(h, fr, dh.DH_DTYPE_U16, B, sets, pw)
        torch.cuda.synchronize()
        return pw.cpu().numpy(), set(dh.dh_get_profile(h))
    finally:
        dh.dh_destroy(h)


@pytest.mark.parametrize("name", ["precision_m96", "large_m176", "serving_512_2pol", "serving_1024_m288"])
def test_split_scoring_reads_the_box_bins(name):
    """Split-BF16 candidate scoring runs the box-source contraction (no x-inverse kernel): every candidate's
    power against the FP64 oracle and against FP32 scoring, on one-, two- and three-tile field sizes."""
    s = _cases()[name]
    frames = syn.make_frames(s, 2, seed=504)["frames"]
    cand = syn.candidate_settings(s, 5, seed=505)
    ref = orc.score_settings(frames, s, cand["tilt_deg"], cand["defocus"], cand["waist"])
    got, kernels = _score(s, frames, cand, 1)
    assert "k_score_tc" in kernels and "k_xinv_sel" not in kernels, kernels
    fp32, kernels32 = _score(s, frames, cand, 0)
    assert "k_score_tc" not in kernels32
    assert np.all(np.isfinite(got))
    # |c|^2 summed: its relative error is at most about twice the coefficients' relative L2 error
    assert np.all(np.abs(got - ref) / ref <= 2 * SPLIT_COEF_TOL), (got, ref)
    assert np.all(np.abs(got - fp32) / fp32 <= 2 * SPLIT_COEF_TOL)
    again, _ = _score(s, frames, cand, 1)
    assert np.array_equal(got.view(np.uint32), again.view(np.uint32))
