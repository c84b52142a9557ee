"""GPU parity of batch averaging (dh_process_batch_avg) against the oracle's phase-aligned averaging.

Frames: distinct fields each measured avg_count times with independent noise and a reference phase drifting
uniformly over [-pi, pi] per measurement, in the sequential and interlaced layouts.  Bars as for plain
processing: field and coefficient relative L2 <= 1e-5 per output window on the FP32 path.
"""
import math

import numpy as np
import pytest

from gpu_util import COEF_TOL, FIELD_TOL, SPLIT_COEF_TOL, rel_l2
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run_avg(setup, frames, batch, avg, mode, precision=0):
    import torch
    import paper_2204_02348_gb300 as dh
    fr = torch.from_numpy(np.ascontiguousarray(frames)).cuda()
    dt = dh.DH_DTYPE_U16 if frames.dtype == np.uint16 else dh.DH_DTYPE_F32
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        dh.dh_set_precision(h, precision)
        m, modes, _ = dh.dh_get_output_dims(h)
        nan = complex(math.nan, math.nan)
        f = torch.full((batch, setup.pol_count, m, m), nan, dtype=torch.complex64, device="cuda")
        c = torch.full((batch, setup.pol_count, modes), nan, dtype=torch.complex64, device="cuda") if modes else None
        dh.dh_process_batch_avg(h, fr, dt, batch, avg, mode, f, c)
        torch.cuda.synchronize()
        return f.cpu().numpy(), (None if c is None else c.cpu().numpy())
    finally:
        dh.dh_destroy(h)


def _check(fields, coefs, f_ref, c_ref, coef_tol=COEF_TOL):
    assert np.all(np.isfinite(fields))
    assert rel_l2(fields, f_ref).max() <= FIELD_TOL
    if c_ref is not None:
        assert np.all(np.isfinite(coefs))
        assert rel_l2(coefs, c_ref).max() <= coef_tol


@pytest.mark.parametrize("mode", [0, 1])
def test_avg_batching_two_pols(mode):
    s = syn.setup_batching()
    d = syn.make_avg_frames(s, 3, 4, mode, seed=130)
    f, c = _run_avg(s, d["frames"], 3, 4, mode)
    f_ref, c_ref = orc.process_batch_avg(d["frames"], s, 4, mode)
    _check(f, c, f_ref, c_ref)


def test_avg_layouts_give_identical_bits():
    s = syn.setup_batching()
    seq = syn.make_avg_frames(s, 3, 3, 0, seed=131)["frames"]
    inter = np.stack([seq[g * 3 + j] for j in range(3) for g in range(3)])
    a = _run_avg(s, seq, 3, 3, 0)
    b = _run_avg(s, inter, 3, 3, 1)
    c = _run_avg(s, seq, 3, 3, 2)
    for x in (b, c):
        assert np.array_equal(a[0].view(np.uint32), x[0].view(np.uint32))
        assert np.array_equal(a[1].view(np.uint32), x[1].view(np.uint32))


def test_avg_count_one_is_plain_processing():
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.setup_batching()
    fr = syn.make_frames(s, 4, seed=132)["frames"]
    f1, c1 = _run_avg(s, fr, 4, 1, 0)
    f0, c0 = _run_avg(s, fr, 4, 0, 1)             # avg_count < 1 is treated as 1
    f_ref, c_ref = orc.process_batch(fr, s)
    _check(f1, c1, f_ref, c_ref)
    assert np.array_equal(f1.view(np.uint32), f0.view(np.uint32))


def test_avg_precision_geometry_lg_and_split_bf16():
    s = syn.with_(syn.setup_precision(), basis="lg")
    d = syn.make_avg_frames(s, 1, 3, 0, seed=133)
    f_ref, c_ref = orc.process_batch_avg(d["frames"], s, 3, 0)
    f, c = _run_avg(s, d["frames"], 1, 3, 0)
    _check(f, c, f_ref, c_ref)
    f, c = _run_avg(s, d["frames"], 1, 3, 0, precision=1)
    _check(f, c, f_ref, c_ref, coef_tol=SPLIT_COEF_TOL)


def test_avg_fill_factor_and_large_window():
    s = syn.with_(syn.serving_geometry("1024x1024_1pol", np.random.default_rng(134)), fill_factor=True)
    d = syn.make_avg_frames(s, 2, 2, 1, seed=135)
    f, c = _run_avg(s, d["frames"], 2, 2, 1)
    f_ref, c_ref = orc.process_batch_avg(d["frames"], s, 2, 1)
    _check(f, c, f_ref, c_ref)


def test_avg_many_groups_span_several_chunks():
    # 420 groups of 2 on the batching geometry: more groups than one scratch chunk holds (8 x SMs / 4, 304 on 152 SMs); the oracle
    # checks groups from the first chunk, across the boundary and from the last chunk
    s = syn.setup_batching()
    G, A = 420, 2
    d = syn.make_avg_frames(s, G, A, 1, seed=136, drift=2.0)
    f, c = _run_avg(s, d["frames"], G, A, 1)
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(c))
    for g in (0, 303, 304, 419):
        sub = np.stack([d["frames"][j * G + g] for j in range(A)])
        f_ref, c_ref = orc.process_batch_avg(sub, s, A, 0)
        _check(f[g:g + 1], c[g:g + 1], f_ref, c_ref)


def test_avg_with_reference_calibration():
    s0 = syn.setup_batching()
    cal, amp = syn.reference_profile(s0, sigma_fraction=0.15, floor=200)
    s = syn.with_(s0, ref_amplitude=amp, ref_cal=cal)
    d = syn.make_avg_frames(s, 2, 3, 0, seed=137)
    f, c = _run_avg(s, d["frames"], 2, 3, 0)
    f_ref, c_ref = orc.process_batch_avg(d["frames"], s, 3, 0)
    _check(f, c, f_ref, c_ref)


def test_avg_batching_split_bf16_fused():
    # the fused kernel's forward-only mode, the averaging kernels and its tensor-core inverse-only mode
    s = syn.setup_batching()
    d = syn.make_avg_frames(s, 3, 3, 0, seed=135)
    f_ref, c_ref = orc.process_batch_avg(d["frames"], s, 3, 0)
    f, c = _run_avg(s, d["frames"], 3, 3, 0, precision=1)
    _check(f, c, f_ref, c_ref, coef_tol=SPLIT_COEF_TOL)

