"""FP64 CPU oracle for the reconstruction path: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` may import
this package.  The library (``paper_2204_02348_gb300``) never imports it and has no CPU fallback.
"""
from . import digholo_oracle  # noqa: F401
