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
