"""Helpers for the GPU parity tests: run the library through its C ABI and compare with the oracle."""
import math

import numpy as np

FIELD_TOL = 1e-5       # FP32 path: field relative L2 per (frame, pol)
COEF_TOL = 1e-5        # FP32 path: coefficient relative L2 per (frame, pol)
SPLIT_COEF_TOL = 1e-4  # split-BF16 overlap: coefficient relative L2 per (frame, pol)
WINDOW_TOL = 2e-6      # masked Fourier window relative L2 per (frame, pol)


def rel_l2(a, b):
    """Relative L2 error of a against b over the trailing axes, per leading (frame, pol) entry."""
    a = np.asarray(a)
    b = np.asarray(b)
    ax = tuple(range(2, a.ndim))
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=ax))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=ax))
    return num / np.maximum(den, 1e-300)


def run_library(setup, frames, precision=0, fields=True, coefs=True, window=False, batch=None, variant=0):
    """Process frames (numpy [B][H][W]) on cuda:0 through dh_process_batch[_window]; returns numpy outputs.
    Outputs are pre-filled with NaN so unwritten elements fail the comparison.  variant: DH_VARIANT_* the handle
    is held to; the result's "variant" is the one dh_get_variant reports for the call's settings."""
    import torch
    import paper_2204_02348_gb300 as dh
    dev = torch.device("cuda", 0)
    fr = torch.from_numpy(np.ascontiguousarray(frames)).to(dev)
    dt = dh.DH_DTYPE_U16 if frames.dtype == np.uint16 else dh.DH_DTYPE_F32
    h = dh.dh_create()
    try:
        dh.configure(h, setup)
        dh.dh_set_precision(h, precision)
        dh.dh_set_variant(h, variant)
        m, modes, _ = dh.dh_get_output_dims(h)
        my = dh.dh_get_field_dims(h)[1]   # fields are [M_y][M_x]
        B = frames.shape[0] if batch is None else max(batch, 1)
        P = setup.pol_count
        nan = complex(math.nan, math.nan)
        f = torch.full((B, P, my, m), nan, dtype=torch.complex64, device=dev) if fields else None
        c = torch.full((B, P, modes), nan, dtype=torch.complex64, device=dev) if (coefs and modes) else None
        w = torch.full((B, P, my, m), nan, dtype=torch.complex64, device=dev) if window else None
        nb = frames.shape[0] if batch is None else batch
        if window:
            dh.dh_process_batch_window(h, fr, dt, nb, w, f, c)
        else:
            dh.dh_process_batch(h, fr, dt, nb, f, c)
        torch.cuda.synchronize()
        out = {"fields": None if f is None else f.cpu().numpy(),
               "coefs": None if c is None else c.cpu().numpy(),
               "window": None if w is None else w.cpu().numpy(), "m": m, "modes": modes,
               "variant": dh.dh_get_variant(h)}
    finally:
        dh.dh_destroy(h)
    return out


def oracle_window(frame, geo):
    """The library's window output as the oracle defines it: (-1)^(p+q) mask F(klo + p, klo + q) / N^2."""
    from oracle import digholo_oracle as orc
    f_box, mask, _, _ = orc.process_window(frame, geo)
    m = geo.x.m
    sign = (-1.0) ** (np.arange(m)[:, None] + np.arange(m)[None, :])
    return sign * mask * f_box / (geo.x.n * geo.y.n)
