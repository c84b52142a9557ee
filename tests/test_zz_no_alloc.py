"""The allocation-free entry point dh_process_batch_noalloc against dh_process_batch.

dh_process_batch_noalloc is for callers that cannot let the library allocate device memory while they
process (their device memory belongs to another allocator, or their acquisition loop must not stall on
cudaMalloc / cudaFree).  It takes its plan tables and scratch from a static device array shared by all calls,
so two calls in a row with different geometries must each match the allocating entry point: stale contents
left by the previous call must not leak into the next.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpu_util import COEF_TOL, FIELD_TOL, rel_l2
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(setup, frames_np, noalloc, precision=None):
    import torch
    import paper_2204_02348_gb300 as dh
    fr = torch.from_numpy(frames_np).cuda()
    dt = dh.DH_DTYPE_U16 if frames_np.dtype == np.uint16 else dh.DH_DTYPE_F32
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        if precision is not None:
            dh.dh_set_precision(h, precision)
        m, modes, _ = dh.dh_get_output_dims(h)
        B, P = frames_np.shape[0], setup.pol_count
        nan = complex(float("nan"), float("nan"))
        f = torch.full((B, P, m, m), nan, dtype=torch.complex64, device="cuda")
        c = torch.full((B, P, modes), nan, dtype=torch.complex64, device="cuda")
        if noalloc:
            free_before = torch.cuda.mem_get_info()[0]
            dh.dh_process_batch_noalloc(h, fr, dt, B, f, c)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
        else:
            dh.dh_process_batch(h, fr, dt, B, f, c)
            torch.cuda.synchronize()
            free_before = free_after = None
        return f.cpu().numpy(), c.cpu().numpy(), (free_before, free_after)
    finally:
        dh.dh_destroy(h)


def test_noalloc_matches_allocating_entry_on_two_calls_in_a_row():
    # call 1: the batching workload, 200 frames -> several chunks of the 15 MiB static scratch
    s1 = syn.setup_batching()
    fr1 = syn.make_frames(s1, 200, seed=77)["frames"]
    # call 2: a different geometry (1024x1024 window, 336x336 field) -> one frame per chunk, overwriting
    # the tables and scratch left by call 1
    s2 = syn.serving_geometry("1024x1024_1pol", np.random.default_rng(78))
    fr2 = syn.make_frames(s2, 3, seed=79)["frames"]

    ref1 = _run(s1, fr1, noalloc=False)
    ref2 = _run(s2, fr2, noalloc=False)
    got1 = _run(s1, fr1, noalloc=True)
    got2 = _run(s2, fr2, noalloc=True)
    for got, ref in ((got1, ref1), (got2, ref2)):
        assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[1]))
        assert rel_l2(got[0], ref[0]).max() <= FIELD_TOL
        assert rel_l2(got[1], ref[1]).max() <= COEF_TOL
    # a third call, back on the first geometry, after the second left its contents behind
    got3 = _run(s1, fr1, noalloc=True)
    assert rel_l2(got3[0], ref1[0]).max() <= FIELD_TOL
    assert rel_l2(got3[1], ref1[1]).max() <= COEF_TOL
    # once the array is resident, a call leaves the device's free memory unchanged
    before, after = got3[2]
    assert before == after


def test_noalloc_lg_basis_matches_oracle():
    from oracle import digholo_oracle as orc
    s = syn.with_(syn.setup_batching(), basis="lg")
    fr = syn.make_frames(s, 150, seed=124)["frames"]       # several chunks of the static scratch
    got = _run(s, fr, noalloc=True)
    ref = _run(s, fr, noalloc=False)
    assert np.all(np.isfinite(got[1]))
    assert rel_l2(got[1], ref[1]).max() <= COEF_TOL
    _, c_ref = orc.process_batch(fr[:3], s)
    assert rel_l2(got[1][:3], c_ref).max() <= COEF_TOL


def test_noalloc_reference_calibration_matches_oracle():
    from oracle import digholo_oracle as orc
    s0 = syn.setup_batching()
    cal, amp = syn.reference_profile(s0, sigma_fraction=0.15, floor=200)
    s = syn.with_(s0, ref_amplitude=amp, ref_cal=cal)
    fr = syn.make_frames(s, 2, seed=138)["frames"]
    got = _run(s, fr, noalloc=True)
    f_ref, c_ref = orc.process_batch(fr, s)
    assert rel_l2(got[0], f_ref).max() <= FIELD_TOL
    assert rel_l2(got[1], c_ref).max() <= COEF_TOL


def test_noalloc_split_precision_handle_gets_fp32_overlap():
    """A handle set to the split-BF16 overlap still gets the FP32 overlap from the allocation-free call (its
    static table area carries no tensor-core operand tables): the result equals the allocating call on an
    FP32 handle, and the coefficients match the oracle at the FP32 bar."""
    import paper_2204_02348_gb300 as dh
    from oracle import digholo_oracle as orc
    s_fp32 = syn.setup_precision()
    fr = syn.make_frames(s_fp32, 6, seed=141)["frames"]
    ref = _run(s_fp32, fr, noalloc=False, precision=dh.DH_PRECISION_FP32)
    got = _run(s_fp32, fr, noalloc=True, precision=dh.DH_PRECISION_SPLIT_BF16)
    assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[1]))
    assert rel_l2(got[0], ref[0]).max() <= FIELD_TOL
    assert rel_l2(got[1], ref[1]).max() <= COEF_TOL
    f_ref, c_ref = orc.process_batch(fr[:2], s_fp32)
    assert rel_l2(got[0][:2], f_ref).max() <= FIELD_TOL
    assert rel_l2(got[1][:2], c_ref).max() <= COEF_TOL
