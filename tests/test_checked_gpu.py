"""The bounds-checked build (libdigholo_gb300_checked.so, DH_CHECKED=1): its guard records a refused access
instead of touching memory outside a buffer, and the whole GPU suite runs under it without a guard firing (each
destroyed handle's status word and guard record are checked, tests/conftest.py).  The normal build's guards
compile away: the same probe records nothing there."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _checked_env():
    env = dict(os.environ)
    env["DH_CHECKED"] = "1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


PROBE = """
import paper_2204_02348_gb300 as dh
from synth import holograms as syn
assert dh.dh_checked_build()
h = dh.dh_create()
dh.configure(h, syn.setup_plain())
assert dh.dh_get_check_record(h) == (0, 0, 0)
dh.dh_check_bounds_probe(h)
st = dh.dh_get_device_status(h)
rec = dh.dh_get_check_record(h)
print(st, rec)
assert st & dh.DH_STATUS_BOUNDS, st
assert rec == (99, 4, 4), rec
assert dh.dh_get_check_record(h) == (0, 0, 0)   # read and cleared
dh.dh_destroy(h)
"""


def test_probe_records_in_the_checked_build_only():
    import paper_2204_02348_gb300 as dh
    from synth import holograms as syn
    assert not dh.dh_checked_build()
    h = dh.dh_create()
    try:
        dh.configure(h, syn.setup_plain())
        dh.dh_check_bounds_probe(h)
        assert dh.dh_get_device_status(h) & dh.DH_STATUS_BOUNDS == 0
        assert dh.dh_get_check_record(h) == (0, 0, 0)
    finally:
        dh.dh_destroy(h)
    r = subprocess.run([sys.executable, "-c", PROBE], cwd=ROOT, env=_checked_env(), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr


def test_gpu_suite_under_bounds_guards():
    """Every other GPU test file, run against the checked build: parity as in the normal build, no guard fired."""
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider",
                        "--ignore=tests/test_checked_gpu.py"], cwd=ROOT, env=_checked_env(), capture_output=True,
                       text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
