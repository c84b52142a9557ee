"""The multi-rank bench logic on CPU: world size 2 over gloo (127.0.0.1).  Each rank draws its own frames,
the job's time is the maximum over ranks, and the whole-job rate counts every rank's frames."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


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
        fr = syn.make_frames(s, 1, seed=bench.rank_seed(syn.BASE_SEED, rank))["frames"]
        gathered = [None] * ws
        dist.all_gather_object(gathered, int(fr.astype("int64").sum()))
        out[rank] = (m, rate, gathered)
    finally:
        dist.destroy_process_group()


def test_two_rank_max_timing_and_disjoint_shards():
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    (m0, r0, g0), (m1, r1, g1) = out[0], out[1]
    assert m0 == m1 == 15.0
    assert r0 == r1 == pytest.approx(2 * 1000 * 4 / 0.015)
    assert g0 == g1 and g0[0] != g0[1]          # the ranks processed different synthetic frames


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 1000, 10, 200.0) == pytest.approx(50000.0)
