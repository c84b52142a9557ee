"""Non-square FFT windows and fields (the guide sets the window size and the IFFT size per axis): the generic
path against the FP64 oracle, whose geometry takes every axis' own window, radius in bins and field size.  Fields
are [M_y][M_x].  Bars as the other parity tests (field and coefficient relative L2 <= 1e-5 per frame and
polarisation); the fused, tensor-core and scoring paths serve square geometries only, so these run the three
generic kernels with the FP32 overlap whatever the precision setting."""
import math

import numpy as np
import pytest

from gpu_util import COEF_TOL, FIELD_TOL, rel_l2, run_library
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu

PX = syn.PIXEL
GENERIC = 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _wide(window, ifft, **kw):
    """Two polarisations on a 640 x 512 frame, windows centred at (160, 256) and (480, 256) pixels."""
    base = syn.with_(syn.setup_batching(), frame_w=640, frame_h=512,
                     beam_centre=[(160.3 * PX, 255.6 * PX), (479.8 * PX, 256.4 * PX)])
    return syn.with_(base, window=window, ifft_size=ifft, **kw)


def _check(setup, frames, out):
    f_ref, c_ref = orc.process_batch(frames, setup)
    if out["fields"] is not None:
        assert out["fields"].shape[2:] == f_ref.shape[2:]
        assert np.all(np.isfinite(out["fields"]))
        assert rel_l2(out["fields"], f_ref).max() <= FIELD_TOL
    if out["coefs"] is not None:
        assert np.all(np.isfinite(out["coefs"]))
        assert rel_l2(out["coefs"], c_ref).max() <= COEF_TOL


CASES = {
    "window_128x64_rule": dict(window=(128, 64), ifft=0),
    "window_64x128_rule": dict(window=(64, 128), ifft=0),
    "window_256x128_fields_96x48": dict(window=(256, 128), ifft=(96, 48)),
    "square_window_fields_64x48": dict(window=128, ifft=(64, 48)),
    "square_window_fields_32x80": dict(window=128, ifft=(32, 80)),
    "window_256x512_rule": dict(window=(256, 512), ifft=0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_non_square_against_oracle(name):
    c = CASES[name]
    s = _wide(c["window"], c["ifft"])
    d = syn.make_frames(s, 3, seed=400)
    out = run_library(s, d["frames"])
    assert out["variant"] == GENERIC
    _check(s, d["frames"], out)


def test_non_square_options():
    # float32 frames, odd window origins, defocus, fill factor, the LG basis and G = 0 on a 128 x 64 window
    s0 = _wide((128, 64), 0)
    for s in (syn.with_(s0, dtype="f32", noise="gauss"),
              syn.with_(s0, beam_centre=[(161.2 * PX, 255.0 * PX), (480.5 * PX, 257.3 * PX)], defocus=[0.9, -1.4]),
              syn.with_(s0, fill_factor=True),
              syn.with_(s0, basis="lg")):
        d = syn.make_frames(s, 2, seed=401)
        _check(s, d["frames"], run_library(s, d["frames"]))
    s = syn.with_(s0, group_count=0)
    d = syn.make_frames(s, 2, seed=402)
    out = run_library(s, d["frames"])
    assert out["modes"] == 0 and out["coefs"] is None
    _check(s, d["frames"], out)


def test_non_square_partial_outputs_precision_and_variants():
    s = _wide((256, 128), (96, 48))
    d = syn.make_frames(s, 2, seed=403)
    _check(s, d["frames"], run_library(s, d["frames"], coefs=False))
    _check(s, d["frames"], run_library(s, d["frames"], fields=False))
    # the split-BF16 setting and a fused variant held: the generic path with the FP32 overlap
    for kw in (dict(precision=1), dict(variant=1), dict(variant=4)):
        out = run_library(s, d["frames"], **kw)
        assert out["variant"] == GENERIC
        _check(s, d["frames"], out)


def test_non_square_host_pipeline_noalloc_and_averaging():
    import torch
    import paper_2204_02348_gb300 as dh
    s = _wide((128, 64), (48, 32))
    d = syn.make_frames(s, 8, seed=404)
    frames = d["frames"]
    f_ref, c_ref = orc.process_batch(frames, s)
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        mx, my, _, _ = dh.dh_get_field_dims(h)
        _, modes, _ = dh.dh_get_output_dims(h)
        B, P = frames.shape[0], s.pol_count
        nan = complex(math.nan, math.nan)
        # host buffers in and out
        fh = torch.full((B, P, my, mx), nan, dtype=torch.complex64).pin_memory()
        ch = torch.full((B, P, modes), nan, dtype=torch.complex64).pin_memory()
        dh.dh_process_batch_host(h, torch.from_numpy(frames).pin_memory(), dh.DH_DTYPE_U16, B, fh, ch)
        assert rel_l2(fh.numpy(), f_ref).max() <= FIELD_TOL and rel_l2(ch.numpy(), c_ref).max() <= COEF_TOL
        # the allocation-free entry point
        fr = torch.from_numpy(frames).cuda()
        fd = torch.full((B, P, my, mx), nan, dtype=torch.complex64, device="cuda")
        cd = torch.full((B, P, modes), nan, dtype=torch.complex64, device="cuda")
        dh.dh_process_batch_noalloc(h, fr, dh.DH_DTYPE_U16, B, fd, cd)
        torch.cuda.synchronize()
        assert rel_l2(fd.cpu().numpy(), f_ref).max() <= FIELD_TOL and rel_l2(cd.cpu().numpy(), c_ref).max() <= COEF_TOL
        # batch averaging of pairs (sequential layout)
        fa = torch.full((B // 2, P, my, mx), nan, dtype=torch.complex64, device="cuda")
        ca = torch.full((B // 2, P, modes), nan, dtype=torch.complex64, device="cuda")
        dh.dh_process_batch_avg(h, fr, dh.DH_DTYPE_U16, B // 2, 2, 0, fa, ca)
        torch.cuda.synchronize()
        fa_ref, ca_ref = orc.process_batch_avg(frames, s, 2, 0)
        assert rel_l2(fa.cpu().numpy(), fa_ref).max() <= FIELD_TOL
        assert rel_l2(ca.cpu().numpy(), ca_ref).max() <= COEF_TOL
        # candidate scoring serves square geometries only
        st = [dh.dh_setting()]
        power = torch.empty((B, 1), dtype=torch.float32, device="cuda")
        with pytest.raises(dh.DigHoloError) as ei:
            dh.dh_score_settings(h, fr, dh.DH_DTYPE_U16, B, st, power)
        assert ei.value.code == dh.DH_ERROR_INVALIDDIMENSION
        assert dh.dh_get_device_status(h) == 0
    finally:
        dh.dh_destroy(h)
