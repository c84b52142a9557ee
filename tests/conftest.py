import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def _ensure_native_library():
    """Build the native library in-tree if it is missing or older than its sources (host compile only)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_dh_build", os.path.join(ROOT, "paper_2204_02348_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


_ensure_native_library()


@pytest.fixture(autouse=True)
def _bounds_guards_stay_quiet(monkeypatch):
    """Under the bounds-checked build (DH_CHECKED=1 in the environment), every handle a test destroys must have
    passed all of its kernels' guards: its status word and guard record are read before it is destroyed."""
    if os.environ.get("DH_CHECKED", "") in ("", "0"):
        yield
        return
    import paper_2204_02348_gb300 as dh
    orig = dh.dh_destroy

    def destroy(h):
        try:
            st = dh.dh_get_device_status(h)
            rec = dh.dh_get_check_record(h)
        finally:
            orig(h)
        if (st & dh.DH_STATUS_BOUNDS) or rec[0]:
            raise AssertionError(f"bounds guard fired: site {rec[0]}, offset {rec[1]}, extent {rec[2]}")

    monkeypatch.setattr(dh, "dh_destroy", destroy)
    yield
