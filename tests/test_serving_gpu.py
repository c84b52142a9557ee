"""Serving loop: requests of mixed geometries arrive while others run; each result must equal the same
request processed alone (the kernels are deterministic and requests never share device memory)."""
import threading
import time

import numpy as np
import pytest

from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _alone(dh, torch, h, setup, frames):
    m, modes, _ = dh.dh_get_output_dims(h)
    fr = torch.from_numpy(frames).cuda()
    f = torch.empty((frames.shape[0], setup.pol_count, m, m), dtype=torch.complex64, device="cuda")
    c = torch.empty((frames.shape[0], setup.pol_count, modes), dtype=torch.complex64, device="cuda")
    dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, frames.shape[0], f, c)
    torch.cuda.synchronize()
    return f.cpu().numpy(), c.cpu().numpy()


def _geometries():
    rng = np.random.default_rng(90)
    out = []
    for kind in syn.SERVING_KINDS:
        s = syn.serving_geometry(kind, rng)
        out.append(s)
    return out


def test_mixed_requests_equal_alone_and_overlap():
    import torch
    import paper_2204_02348_gb300 as dh
    geos = _geometries()
    handles = []
    for s in geos:
        h = dh.dh_create()
        dh.configure(h, s)
        handles.append(h)
    rng = np.random.default_rng(91)
    reqs = []
    for k in range(18):
        gi = int(rng.integers(0, len(geos)))
        n = int(rng.integers(1, 5))
        fr = syn.make_frames(geos[gi], n, seed=1000 + k)["frames"]
        m, modes, _ = dh.dh_get_output_dims(handles[gi])
        host_in = torch.from_numpy(fr).pin_memory()
        f = torch.full((n, geos[gi].pol_count, m, m), complex(float("nan"), 0), dtype=torch.complex64).pin_memory()
        c = torch.full((n, geos[gi].pol_count, modes), complex(float("nan"), 0), dtype=torch.complex64).pin_memory()
        reqs.append((gi, fr, host_in, f, c))
    alone = [_alone(dh, torch, handles[gi], geos[gi], fr) for gi, fr, _, _, _ in reqs]
    srv = dh.dh_server_create(2 << 30, 4)
    try:
        tickets = [None] * len(reqs)

        def producer():
            arr = np.random.default_rng(92)
            for i, (gi, fr, hin, f, c) in enumerate(reqs):
                tickets[i] = dh.dh_server_submit(srv, handles[gi], hin, dh.DH_DTYPE_U16, fr.shape[0], f, c)
                if i % 3 == 2:
                    time.sleep(float(arr.exponential(0.002)))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for t in tickets:
            dh.dh_server_wait(srv, t, -1)
        st = dh.dh_server_stats(srv)
    finally:
        dh.dh_server_destroy(srv)
        for h in handles:
            dh.dh_destroy(h)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert st["peak_inflight"] >= 2, st
    for (gi, fr, hin, f, c), (fa, ca) in zip(reqs, alone):
        assert np.array_equal(f.numpy().view(np.uint32), fa.view(np.uint32))
        assert np.array_equal(c.numpy().view(np.uint32), ca.view(np.uint32))


def test_small_budget_chunks_a_large_request():
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.serving_geometry("1024x1024_1pol", np.random.default_rng(93))
    fr = syn.make_frames(s, 10, seed=94)["frames"]
    h = dh.dh_create()
    dh.configure(h, s)
    try:
        fa, ca = _alone(dh, torch, h, s, fr)
        srv = dh.dh_server_create(48 << 20, 2)
        try:
            hin = torch.from_numpy(fr).pin_memory()
            f = torch.empty(fa.shape, dtype=torch.complex64).pin_memory()
            c = torch.empty(ca.shape, dtype=torch.complex64).pin_memory()
            t = dh.dh_server_submit(srv, h, hin, dh.DH_DTYPE_U16, 10, f, c)
            dh.dh_server_wait(srv, t, -1)
            st = dh.dh_server_stats(srv)
        finally:
            dh.dh_server_destroy(srv)
        assert st["peak_bytes"] <= st["budget_bytes"] == 48 << 20
        assert np.array_equal(f.numpy().view(np.uint32), fa.view(np.uint32))
        assert np.array_equal(c.numpy().view(np.uint32), ca.view(np.uint32))
    finally:
        dh.dh_destroy(h)


def test_budget_errors_and_timeouts():
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.serving_geometry("1024x1024_1pol", np.random.default_rng(95))
    h = dh.dh_create()
    dh.configure(h, s)
    fr = torch.from_numpy(syn.make_frames(s, 1, seed=96)["frames"]).pin_memory()
    try:
        srv0 = dh.dh_server_create(0, 1)
        try:
            with pytest.raises(dh.DigHoloError) as ei:
                dh.dh_server_submit(srv0, h, fr, dh.DH_DTYPE_U16, 1)
            assert ei.value.code == dh.DH_ERROR_MEMORYALLOCATION
            with pytest.raises(dh.DigHoloError) as ei:
                dh.dh_server_wait(srv0, 12345, 0)
            assert ei.value.code == dh.DH_ERROR_INVALIDARGUMENT
        finally:
            dh.dh_server_destroy(srv0)
        big = torch.from_numpy(np.repeat(fr.numpy(), 48, axis=0)).pin_memory()
        m, modes, _ = dh.dh_get_output_dims(h)
        flds = [torch.empty((48, 1, m, m), dtype=torch.complex64).pin_memory() for _ in range(3)]
        srv = dh.dh_server_create(1 << 30, 1)
        try:
            # the last of three queued requests (48 frames of 1024 x 1024 with fields each, milliseconds of GPU
            # work apiece) cannot have finished when a zero timeout is asked right after its submission
            ts = [dh.dh_server_submit(srv, h, big, dh.DH_DTYPE_U16, 48, flds[k]) for k in range(3)]
            with pytest.raises(dh.DigHoloError) as ei:
                dh.dh_server_wait(srv, ts[-1], 0)
            assert ei.value.code == dh.DH_ERROR_TIMEOUT
            for t in ts:
                dh.dh_server_wait(srv, t, -1)
        finally:
            dh.dh_server_destroy(srv)
    finally:
        dh.dh_destroy(h)


@pytest.mark.parametrize("kind", ["batching", "512x512_2pol", "1024x1024_1pol"])
def test_lg_basis_request_equals_alone(kind):
    # the HG coefficients of the transform sit in the request's own scratch: the fused path (no other
    # scratch) on the 320x256 batching geometry, the generic path on the others; the 1024 window chunks
    import torch
    import paper_2204_02348_gb300 as dh
    base = syn.setup_batching() if kind == "batching" else syn.serving_geometry(kind, np.random.default_rng(125))
    s = syn.with_(base, basis="lg")
    fr = syn.make_frames(s, 6, seed=126)["frames"]
    h = dh.dh_create()
    dh.configure(h, s)
    try:
        fa, ca = _alone(dh, torch, h, s, fr)
        srv = dh.dh_server_create(48 << 20, 2)
        try:
            hin = torch.from_numpy(fr).pin_memory()
            f = torch.empty(fa.shape, dtype=torch.complex64).pin_memory()
            c = torch.empty(ca.shape, dtype=torch.complex64).pin_memory()
            t = dh.dh_server_submit(srv, h, hin, dh.DH_DTYPE_U16, fr.shape[0], f, c)
            dh.dh_server_wait(srv, t, -1)
        finally:
            dh.dh_server_destroy(srv)
        assert np.array_equal(f.numpy().view(np.uint32), fa.view(np.uint32))
        assert np.array_equal(c.numpy().view(np.uint32), ca.view(np.uint32))
    finally:
        dh.dh_destroy(h)


def test_mixed_precisions_equal_alone():
    # requests on the batching geometry with the FP32 and the split-BF16 overlap (the fused kernel's two
    # variants) interleaved with a split-BF16 256 x 256 geometry (generic path): each equals its lone run
    import torch
    import paper_2204_02348_gb300 as dh
    geos = [syn.setup_batching(), syn.setup_batching(), syn.serving_geometry("256x256_1pol", np.random.default_rng(97))]
    precs = [dh.DH_PRECISION_FP32, dh.DH_PRECISION_SPLIT_BF16, dh.DH_PRECISION_SPLIT_BF16]
    handles = []
    for s, p in zip(geos, precs):
        h = dh.dh_create()
        dh.configure(h, s)
        dh.dh_set_precision(h, p)
        handles.append(h)
    try:
        reqs = []
        for k in range(9):
            gi = k % 3
            n = 2 + k % 4
            fr = syn.make_frames(geos[gi], n, seed=1100 + k)["frames"]
            m, modes, _ = dh.dh_get_output_dims(handles[gi])
            hin = torch.from_numpy(fr).pin_memory()
            f = torch.empty((n, geos[gi].pol_count, m, m), dtype=torch.complex64).pin_memory()
            c = torch.empty((n, geos[gi].pol_count, modes), dtype=torch.complex64).pin_memory()
            reqs.append((gi, fr, hin, f, c))
        alone = [_alone(dh, torch, handles[gi], geos[gi], fr) for gi, fr, _, _, _ in reqs]
        srv = dh.dh_server_create(1 << 30, 3)
        try:
            tickets = [dh.dh_server_submit(srv, handles[gi], hin, dh.DH_DTYPE_U16, fr.shape[0], f, c)
                       for gi, fr, hin, f, c in reqs]
            for t in tickets:
                dh.dh_server_wait(srv, t, -1)
        finally:
            dh.dh_server_destroy(srv)
        for (gi, fr, hin, f, c), (fa, ca) in zip(reqs, alone):
            assert np.array_equal(f.numpy().view(np.uint32), fa.view(np.uint32))
            assert np.array_equal(c.numpy().view(np.uint32), ca.view(np.uint32))
    finally:
        for h in handles:
            dh.dh_destroy(h)


def test_small_requests_pass_one_that_does_not_fit_and_report_device_time():
    """Three large requests and a budget that holds two of them (a request reserves at most half the budget):
    the third large one waits, and small requests submitted behind it are admitted first (no head-of-line
    blocking); it still completes (its wait is bounded).  Every result equals the lone run; stats report device
    times."""
    import torch
    import paper_2204_02348_gb300 as dh
    rng = np.random.default_rng(95)
    big_s = syn.serving_geometry("1024x1024_1pol", rng)
    small_s = syn.serving_geometry("256x256_1pol", rng)
    hb, hs = dh.dh_create(), dh.dh_create()
    dh.configure(hb, big_s)
    dh.configure(hs, small_s)
    big = [syn.make_frames(big_s, 48, seed=1100 + k)["frames"] for k in range(3)]
    small = [syn.make_frames(small_s, 1, seed=1200 + k)["frames"] for k in range(10)]
    alone_b = [_alone(dh, torch, hb, big_s, fr) for fr in big]
    alone_s = [_alone(dh, torch, hs, small_s, fr) for fr in small]

    def bufs(h, s, fr):
        m, modes, _ = dh.dh_get_output_dims(h)
        n = fr.shape[0]
        return (torch.from_numpy(fr).pin_memory(),
                torch.full((n, s.pol_count, m, m), complex(float("nan"), 0), dtype=torch.complex64).pin_memory(),
                torch.full((n, s.pol_count, modes), complex(float("nan"), 0), dtype=torch.complex64).pin_memory())

    bb = [bufs(hb, big_s, fr) for fr in big]
    sb = [bufs(hs, small_s, fr) for fr in small]
    # per large frame: its rows, field, coefficients and the generic path's scratch (r1 and the window); a budget
    # of 62.4 such frames gives each large request one chunk of 31 frames, so two run and the third waits, and
    # 0.4 of a large frame stays free, room for the small requests
    m, modes, _ = dh.dh_get_output_dims(hb)
    n = big_s.window
    per_frame = big_s.frame_w * big_s.frame_h * 2 + m * m * 8 + modes * 8 + (m * n + m * m) * 8
    srv = dh.dh_server_create(int(62.4 * per_frame), 8)
    try:
        tb = [dh.dh_server_submit(srv, hb, b[0], dh.DH_DTYPE_U16, 48, b[1], b[2]) for b in bb]
        ts = [dh.dh_server_submit(srv, hs, b[0], dh.DH_DTYPE_U16, 1, b[1], b[2]) for b in sb]
        for t in tb + ts:
            dh.dh_server_wait(srv, t, -1)
        st = dh.dh_server_stats(srv)
    finally:
        dh.dh_server_destroy(srv)
        dh.dh_destroy(hb)
        dh.dh_destroy(hs)
    assert st["completed"] == 13 and st["failed"] == 0
    assert 1 <= st["bypassed"] <= 10
    for (f, c), b in zip(alone_b + alone_s, bb + sb):
        assert np.array_equal(b[1].numpy(), f) and np.array_equal(b[2].numpy(), c)
    assert 0 < st["kernel_p50_ms"] <= st["kernel_p99_ms"] <= st["span_p99_ms"] + 1e-3
    assert st["kernel_ms_total"] > 0 and st["wait_p99_ms"] >= st["wait_p50_ms"] >= 0
