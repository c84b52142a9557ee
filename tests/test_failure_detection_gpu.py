"""Failure detection without a GPU fault: the kernels' bounded mbarrier wait runs out on a barrier nothing
completes, reports it, and leaves the context usable; normal processing leaves the status word clear."""
import numpy as np
import pytest

from gpu_util import COEF_TOL, rel_l2, run_library
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bounded_wait_expires_and_context_stays_usable():
    import paper_2204_02348_gb300 as dh
    assert dh.dh_check_bounded_wait(2000) is True
    s = syn.setup_plain()
    d = syn.make_frames(s, 1, seed=90)
    out = run_library(s, d["frames"])
    _, c_ref = orc.process_batch(d["frames"], s)
    assert rel_l2(out["coefs"], c_ref).max() <= COEF_TOL


def test_status_word_clear_after_normal_work():
    import torch
    import paper_2204_02348_gb300 as dh
    for name, prec in (("batching", 0), ("precision", 1)):
        s = syn.WORKLOADS[name]()
        d = syn.make_frames(s, 2, seed=91)
        h = dh.dh_create()
        try:
            dh.configure(h, s)
            dh.dh_set_precision(h, prec)
            m, modes, _ = dh.dh_get_output_dims(h)
            fr = torch.from_numpy(d["frames"]).cuda()
            c = torch.empty((2, s.pol_count, modes), dtype=torch.complex64, device="cuda")
            dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, 2, None, c)
            assert dh.dh_get_device_status(h) == 0
            assert np.all(np.isfinite(c.cpu().numpy()))
        finally:
            dh.dh_destroy(h)
