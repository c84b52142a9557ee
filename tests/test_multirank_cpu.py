"""The multi-rank bench logic on CPU: world size 2 over gloo (127.0.0.1).  Each rank processes a contiguous
shard of the job's one seeded frame stream; the shards are disjoint and together cover the global range, the
job's time is the maximum over ranks, and the whole-job rate counts every rank's frames."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

FRAMES_PER_RANK = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import bench
    from synth import holograms as syn
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
        m = bench.max_over_ranks(local_ms, ws)
        rate = bench.whole_job_rate(ws, 1000, 4, m)
        s = syn.setup_batching()
        first, count = bench.rank_shard(FRAMES_PER_RANK, rank)
        fr = syn.make_frames(s, count, seed=syn.BASE_SEED, first=first)["frames"]
        sums = [int(f.astype("int64").sum()) for f in fr]
        gathered = [None] * ws
        dist.all_gather_object(gathered, (first, count, sums))
        out[rank] = (m, rate, gathered)
    finally:
        dist.destroy_process_group()


def test_two_rank_max_timing_and_disjoint_contiguous_shards():
    from synth import holograms as syn
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    (m0, r0, g0), (m1, r1, g1) = out[0], out[1]
    assert m0 == m1 == 15.0
    assert r0 == r1 == pytest.approx(2 * 1000 * 4 / 0.015)
    assert g0 == g1
    # the shards tile [0, ws F) without overlap, in rank order
    ranges = sorted((first, first + count) for first, count, _ in g0)
    assert ranges[0][0] == 0 and ranges[-1][1] == ws * FRAMES_PER_RANK
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    # every rank's frames are its slice of the one global stream a single process generates
    whole = syn.make_frames(syn.setup_batching(), ws * FRAMES_PER_RANK, seed=syn.BASE_SEED)["frames"]
    ref = [int(f.astype("int64").sum()) for f in whole]
    for first, count, sums in g0:
        assert sums == ref[first:first + count]
    assert len(set(ref)) == len(ref)          # distinct frames, so a repeated shard would have been seen


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 1000, 10, 200.0) == pytest.approx(50000.0)
    assert bench.rank_shard(1000, 0) == (0, 1000) and bench.rank_shard(1000, 3) == (3000, 1000)
    assert np.all(np.diff([bench.rank_shard(7, r)[0] for r in range(5)]) == 7)
