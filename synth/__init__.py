"""Seeded synthetic hologram generator shared by the tests, the oracle checks and the benchmark.

This package is the *forward model* only: it forms camera frames |S + R|^2 from a known signal S (a sum of
Hermite-Gaussian modes) and a tilted, defocused plane-wave reference R, then adds camera noise.  It holds
none of the reconstruction arithmetic (no Fourier transforms, windows, tilt removal or overlaps), so that
the FP64 oracle and the CUDA path can both consume its frames without sharing any code of the method.
It plays the role of the paper's frame simulator (digHoloFrameSimulatorCreate, "Frame simulator").
"""
from .holograms import (  # noqa: F401
    Setup,
    setup_plain,
    setup_batching,
    setup_precision,
    setup_large_batch,
    serving_geometry,
    make_frames,
    hg_closed_form,
    random_unit_coefs,
    haar_unitary,
    candidate_settings,
    defocus_from_waves,
    WORKLOADS,
)
