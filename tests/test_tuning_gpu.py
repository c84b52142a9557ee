"""Every candidate the tuner can pick, run against the FP64 oracle (fields and coefficients at the FP32 bars,
coefficients at the split-BF16 bar with that overlap), and dh_autotune's choice written to a cache file that a
fresh handle reads back."""
import json
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


def _geometries():
    rng = np.random.default_rng(401)
    return {
        "batching": syn.setup_batching(),
        "precision": syn.setup_precision(),
        "serving_1024": syn.serving_geometry("1024x1024_1pol", rng),
    }


def _run(setup, frames, tuning=None, precision=0, autotune_cache=None):
    import torch
    import paper_2204_02348_gb300 as dh
    dev = torch.device("cuda", 0)
    fr = torch.from_numpy(np.ascontiguousarray(frames)).to(dev)
    dt = dh.DH_DTYPE_U16 if frames.dtype == np.uint16 else dh.DH_DTYPE_F32
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        dh.dh_set_precision(h, precision)
        m, modes, _ = dh.dh_get_output_dims(h)
        B, P = frames.shape[0], setup.pol_count
        nan = complex(math.nan, math.nan)
        f = torch.full((B, P, m, m), nan, dtype=torch.complex64, device=dev)
        c = torch.full((B, P, modes), nan, dtype=torch.complex64, device=dev)
        if autotune_cache is not None:
            dh.dh_set_tuning_cache(h, autotune_cache)
            dh.dh_autotune(h, fr, dt, B, f, c, reps=2)
        else:
            if tuning is not None:
                dh.dh_set_tuning(h, tuning)
            dh.dh_process_batch(h, fr, dt, B, f, c)
        torch.cuda.synchronize()
        return f.cpu().numpy(), c.cpu().numpy(), dh.dh_get_tuning(h), dh.dh_get_variant(h), dh.dh_tuning_key(h)
    finally:
        dh.dh_destroy(h)


@pytest.mark.parametrize("name,precision", [("batching", 0), ("precision", 0), ("precision", 1), ("serving_1024", 0)])
def test_every_candidate_against_oracle(name, precision):
    import paper_2204_02348_gb300 as dh
    s = _geometries()[name]
    frames = syn.make_frames(s, 2, seed=402)["frames"]
    f_ref, c_ref = orc.process_batch(frames, s)
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        dh.dh_set_precision(h, precision)
        cands = dh.dh_tuning_candidates(h)
    finally:
        dh.dh_destroy(h)
    assert len(cands) >= 3
    for cand in cands:
        f, c, tun, variant, _ = _run(s, frames, cand, precision)
        assert tun == cand
        if cand["variant"] != 0:
            assert variant == cand["variant"], cand
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(c)), cand
        assert rel_l2(f, f_ref).max() <= FIELD_TOL, cand
        assert rel_l2(c, c_ref).max() <= (SPLIT_COEF_TOL if precision else COEF_TOL), cand


def test_autotune_writes_cache_that_a_fresh_handle_reads(tmp_path):
    s = _geometries()["precision"]
    frames = syn.make_frames(s, 16, seed=403)["frames"]
    path = str(tmp_path / "tuning.json")
    f, c, tun, _, key = _run(s, frames, autotune_cache=path)
    # the outputs of the tuning call are the chosen candidate's
    f_ref, c_ref = orc.process_batch(frames[:2], s)
    assert rel_l2(f[:2], f_ref).max() <= FIELD_TOL and rel_l2(c[:2], c_ref).max() <= COEF_TOL
    doc = json.load(open(path))
    assert doc["format"] == "digholo-gb300-tuning"
    ent = [e for e in doc["entries"] if e["key"] == key]
    assert len(ent) == 1 and ent[0]["candidates"] == 13 and ent[0]["ms"] > 0
    assert {"variant": ent[0]["variant"], "chunk_mb": ent[0]["chunk_mb"], "radix": ent[0]["radix"]} == tun
    # a fresh handle loading the cache runs the same choice, with the same results to rounding
    import torch
    import paper_2204_02348_gb300 as dh
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        dh.dh_set_tuning_cache(h, path)
        assert dh.dh_get_tuning(h) == tun
        dev = torch.device("cuda", 0)
        fr = torch.from_numpy(frames).to(dev)
        m, modes, _ = dh.dh_get_output_dims(h)
        f2 = torch.empty((16, 2, m, m), dtype=torch.complex64, device=dev)
        c2 = torch.empty((16, 2, modes), dtype=torch.complex64, device=dev)
        dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, 16, f2, c2)
        torch.cuda.synchronize()
        assert np.array_equal(f2.cpu().numpy(), f) and np.array_equal(c2.cpu().numpy(), c)
    finally:
        dh.dh_destroy(h)
