"""dh_process_batch_host: host buffers in and out through the chunked three-stream pipeline, against
dh_process_batch on device buffers (bit-identical: the same kernels on the same frames) and the oracle."""
import math

import numpy as np
import pytest

from gpu_util import COEF_TOL, FIELD_TOL, rel_l2
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _device(dh, torch, h, setup, frames):
    m, modes, _ = dh.dh_get_output_dims(h)
    fr = torch.from_numpy(frames).cuda()
    dt = dh.DH_DTYPE_U16 if frames.dtype == np.uint16 else dh.DH_DTYPE_F32
    f = torch.empty((frames.shape[0], setup.pol_count, m, m), dtype=torch.complex64, device="cuda")
    c = torch.empty((frames.shape[0], setup.pol_count, modes), dtype=torch.complex64, device="cuda") if modes else None
    dh.dh_process_batch(h, fr, dt, frames.shape[0], f, c)
    torch.cuda.synchronize()
    return f.cpu().numpy(), (None if c is None else c.cpu().numpy())


def _host(dh, torch, h, setup, frames, pinned=True, fields=True):
    m, modes, _ = dh.dh_get_output_dims(h)
    dt = dh.DH_DTYPE_U16 if frames.dtype == np.uint16 else dh.DH_DTYPE_F32
    nan = complex(math.nan, math.nan)
    if pinned:
        hin = torch.from_numpy(frames).pin_memory()
        f = torch.full((frames.shape[0], setup.pol_count, m, m), nan, dtype=torch.complex64).pin_memory()
        c = torch.full((frames.shape[0], setup.pol_count, modes), nan, dtype=torch.complex64).pin_memory()
    else:
        hin = np.ascontiguousarray(frames)
        f = np.full((frames.shape[0], setup.pol_count, m, m), nan, dtype=np.complex64)
        c = np.full((frames.shape[0], setup.pol_count, modes), nan, dtype=np.complex64)
    dh.dh_process_batch_host(h, hin, dt, frames.shape[0], f if fields else None, c)
    f = np.asarray(f) if not pinned else f.numpy()
    c = np.asarray(c) if not pinned else c.numpy()
    return f, c


@pytest.mark.parametrize("name,count", [("batching", 300), ("plain", 5), ("precision", 70)])
def test_host_pipeline_equals_device_entry(name, count):
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.WORKLOADS[name]()
    fr = syn.make_frames(s, count, seed=140)["frames"]
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        fd, cd = _device(dh, torch, h, s, fr)
        fh, ch = _host(dh, torch, h, s, fr)
        assert np.array_equal(fh.view(np.uint32), fd.view(np.uint32))
        assert np.array_equal(ch.view(np.uint32), cd.view(np.uint32))
        # a second call reuses the pipeline buffers; pageable numpy buffers copy synchronously, same results
        fh2, ch2 = _host(dh, torch, h, s, fr[: max(1, count // 2)], pinned=False)
        assert np.array_equal(fh2.view(np.uint32), fd[: max(1, count // 2)].view(np.uint32))
        assert np.array_equal(ch2.view(np.uint32), cd[: max(1, count // 2)].view(np.uint32))
    finally:
        dh.dh_destroy(h)
    f_ref, c_ref = orc.process_batch(fr[:2], s)
    assert rel_l2(fh[:2], f_ref).max() <= FIELD_TOL
    assert rel_l2(ch[:2], c_ref).max() <= COEF_TOL


def test_host_pipeline_generic_geometry_lg_basis_coefficients_only():
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.with_(syn.serving_geometry("1024x1024_1pol", np.random.default_rng(141)), basis="lg")
    fr = syn.make_frames(s, 40, seed=142)["frames"]
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        fd, cd = _device(dh, torch, h, s, fr)
        _, ch = _host(dh, torch, h, s, fr, fields=False)
        assert np.array_equal(ch.view(np.uint32), cd.view(np.uint32))
    finally:
        dh.dh_destroy(h)


def test_async_host_calls_match_the_device_entry():
    """dh_process_batch_host_async: three calls back to back into the same host buffers, then one with another
    batch size (another staging layout) into other buffers, one wait: every output bit-identical to
    dh_process_batch on device buffers."""
    import torch
    import paper_2204_02348_gb300 as dh
    for name, count in (("batching", 300), ("precision", 70)):
        s = syn.WORKLOADS[name]()
        fr = syn.make_frames(s, count, seed=142)["frames"]
        h = dh.dh_create()
        try:
            dh.configure(h, s)
            fd, cd = _device(dh, torch, h, s, fr)
            m, modes, _ = dh.dh_get_output_dims(h)
            hin = torch.from_numpy(fr).pin_memory()
            nan = complex(math.nan, math.nan)
            f = torch.full((count, s.pol_count, m, m), nan, dtype=torch.complex64).pin_memory()
            c = torch.full((count, s.pol_count, modes), nan, dtype=torch.complex64).pin_memory()
            part = max(1, count // 3)
            f2 = torch.full((part, s.pol_count, m, m), nan, dtype=torch.complex64).pin_memory()
            c2 = torch.full((part, s.pol_count, modes), nan, dtype=torch.complex64).pin_memory()
            for _ in range(3):
                dh.dh_process_batch_host_async(h, hin, dh.DH_DTYPE_U16, count, f, c)
            dh.dh_process_batch_host_async(h, hin[:part], dh.DH_DTYPE_U16, part, f2, c2)
            dh.dh_process_batch_host_wait(h)
            assert np.array_equal(f.numpy().view(np.uint32), fd.view(np.uint32))
            assert np.array_equal(c.numpy().view(np.uint32), cd.view(np.uint32))
            assert np.array_equal(f2.numpy().view(np.uint32), fd[:part].view(np.uint32))
            assert np.array_equal(c2.numpy().view(np.uint32), cd[:part].view(np.uint32))
            dh.dh_process_batch_host_wait(h)   # nothing in flight: returns at once
        finally:
            dh.dh_destroy(h)


def test_async_host_calls_generic_path_with_scratch_and_lg_basis():
    """The asynchronous entry on a geometry that runs the generic kernels (1024 x 1024 window, spectra in each
    staging slot's scratch) with the LG output basis (HG coefficients in scratch before the transform): two calls
    into the same host buffers, one wait, bit-identical to dh_process_batch."""
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.with_(syn.serving_geometry("1024x1024_1pol", np.random.default_rng(143)), basis="lg")
    fr = syn.make_frames(s, 6, seed=144)["frames"]
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        assert dh.dh_get_variant(h) == dh.DH_VARIANT_GENERIC
        fd, cd = _device(dh, torch, h, s, fr)
        m, modes, _ = dh.dh_get_output_dims(h)
        nan = complex(math.nan, math.nan)
        hin = torch.from_numpy(fr).pin_memory()
        f = torch.full((6, 1, m, m), nan, dtype=torch.complex64).pin_memory()
        c = torch.full((6, 1, modes), nan, dtype=torch.complex64).pin_memory()
        for _ in range(2):
            dh.dh_process_batch_host_async(h, hin, dh.DH_DTYPE_U16, 6, f, c)
        dh.dh_process_batch_host_wait(h)
        assert np.array_equal(f.numpy().view(np.uint32), fd.view(np.uint32))
        assert np.array_equal(c.numpy().view(np.uint32), cd.view(np.uint32))
    finally:
        dh.dh_destroy(h)


def test_host_pipeline_windows_at_different_heights():
    """Two 256 x 256 windows 100 rows apart (the fused 256 x 256 kernel): the host pipeline uploads the 356 rows
    that hold both, and each polarisation's window starts at its own row of the cropped frames; blocking and
    asynchronous calls bit-identical to dh_process_batch."""
    import torch
    import paper_2204_02348_gb300 as dh
    px = syn.PIXEL
    s = syn.with_(syn.setup_precision(), beam_centre=[(160.0 * px, 200.0 * px), (480.0 * px, 300.0 * px)])
    fr = syn.make_frames(s, 40, seed=145)["frames"]
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        assert dh.dh_get_variant(h) == dh.DH_VARIANT_FUSED
        fd, cd = _device(dh, torch, h, s, fr)
        fh, ch = _host(dh, torch, h, s, fr)
        assert np.array_equal(fh.view(np.uint32), fd.view(np.uint32))
        assert np.array_equal(ch.view(np.uint32), cd.view(np.uint32))
        m, modes, _ = dh.dh_get_output_dims(h)
        hin = torch.from_numpy(fr).pin_memory()
        f = torch.empty((40, 2, m, m), dtype=torch.complex64).pin_memory()
        c = torch.empty((40, 2, modes), dtype=torch.complex64).pin_memory()
        dh.dh_process_batch_host_async(h, hin, dh.DH_DTYPE_U16, 40, f, c)
        dh.dh_process_batch_host_wait(h)
        assert np.array_equal(f.numpy().view(np.uint32), fd.view(np.uint32))
        assert np.array_equal(c.numpy().view(np.uint32), cd.view(np.uint32))
    finally:
        dh.dh_destroy(h)
    f_ref, c_ref = orc.process_batch(fr[:2], s)
    assert rel_l2(fd[:2], f_ref).max() <= FIELD_TOL
    assert rel_l2(cd[:2], c_ref).max() <= COEF_TOL
