"""GB300-native batched off-axis hologram reconstruction (digHolo's processing pipeline).

Thin ctypes binding over the C ABI in ``include/digholo.h``: the functions keep the ABI's names and only
marshal arguments (torch tensors become device pointers, streams become ``cudaStream_t`` handles).  Every
step of the reconstruction runs in the library's CUDA kernels; importing this package without the built
native library raises ImportError (there is no CPU fallback).  Build with ``python
paper_2204_02348_gb300/_build.py`` or ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# DH_CHECKED=1 in the environment selects the bounds-checked build of the same library (csrc/check.cuh)
CHECKED = os.environ.get("DH_CHECKED", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "_native", "libdigholo_gb300_checked.so" if CHECKED else "libdigholo_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"native library missing at {LIB_PATH}; build it with `python paper_2204_02348_gb300/_build.py`")

_lib = ctypes.CDLL(LIB_PATH)

# constants (include/digholo.h)
DH_SUCCESS = 0
DH_ERROR_ERROR = 1
DH_ERROR_INVALIDHANDLE = 2
DH_ERROR_NULLPOINTER = 3
DH_ERROR_INVALIDDIMENSION = 5
DH_ERROR_INVALIDPOLARISATION = 6
DH_ERROR_INVALIDAXIS = 7
DH_ERROR_INVALIDARGUMENT = 8
DH_ERROR_MEMORYALLOCATION = 9
DH_ERROR_TIMEOUT = 12
DH_ERROR_CUDA = 13
DH_DTYPE_U16 = 0
DH_DTYPE_F32 = 1
DH_PRECISION_FP32 = 0
DH_PRECISION_SPLIT_BF16 = 1
DH_VARIANT_AUTO = 0
DH_VARIANT_FUSED = 1
DH_VARIANT_FUSED_PRUNED = 2
DH_VARIANT_GENERIC = 3
DH_VARIANT_FUSED_GROUPS = 4
DH_BASIS_HG = 0
DH_BASIS_LG = 1
DH_BASIS_CUSTOM = 2
DH_AVGMODE_SEQUENTIAL = 0
DH_AVGMODE_INTERLACED = 1
DH_AVGMODE_SEQUENTIALSWEEP = 2
DH_MAX_AVG_COUNT = 4096
DH_MAX_POLS = 2


class DigHoloError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"digholo error {code}: {msg}")
        self.code = code


DH_MAX_RADICES = 6


class dh_tuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("chunk_mb", ctypes.c_int), ("nradix", ctypes.c_int),
                ("radix", ctypes.c_int * DH_MAX_RADICES)]

    def as_dict(self):
        return {"variant": self.variant, "chunk_mb": self.chunk_mb, "radix": list(self.radix[:self.nradix])}


def make_tuning(variant=0, chunk_mb=0, radix=()):
    t = dh_tuning()
    t.variant, t.chunk_mb, t.nradix = int(variant), int(chunk_mb), len(radix)
    for i, r in enumerate(radix):
        t.radix[i] = int(r)
    return t


class dh_setting(ctypes.Structure):
    _fields_ = [("tilt_deg", (ctypes.c_double * 2) * DH_MAX_POLS),
                ("defocus", ctypes.c_double * DH_MAX_POLS),
                ("waist", ctypes.c_double * DH_MAX_POLS)]


class dh_request(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("h_frames", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("batch", ctypes.c_int), ("h_fields", ctypes.c_void_p), ("h_coefs", ctypes.c_void_p)]


class dh_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("frames", ctypes.c_longlong), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("frames_per_s", ctypes.c_double), ("budget_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int), ("peak_inflight", ctypes.c_int),
                ("wait_p50_ms", ctypes.c_double), ("wait_p99_ms", ctypes.c_double),
                ("kernel_p50_ms", ctypes.c_double), ("kernel_p99_ms", ctypes.c_double),
                ("span_p50_ms", ctypes.c_double), ("span_p99_ms", ctypes.c_double),
                ("kernel_ms_total", ctypes.c_double), ("bypassed", ctypes.c_longlong)]


_i, _d, _p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_PROTOS = {
    "dh_create": [ctypes.POINTER(_i)],
    "dh_destroy": [_i],
    "dh_set_frame": [_i, _i, _i, _i, _d],
    "dh_set_wavelength": [_i, _d],
    "dh_set_fft_window": [_i, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "dh_set_beam_centre": [_i, _i, _i, _d],
    "dh_set_fourier_window_radius": [_i, _d],
    "dh_set_ifft_size": [_i, _i, _i],
    "dh_set_tilt": [_i, _i, _i, _d],
    "dh_set_defocus": [_i, _i, _d],
    "dh_set_basis": [_i, _i, _d, _i],
    "dh_set_precision": [_i, _i],
    "dh_set_variant": [_i, _i],
    "dh_get_variant": [_i, ctypes.POINTER(_i)],
    "dh_tuning_key": [_i, ctypes.c_char_p, _i],
    "dh_tuning_candidates": [_i, ctypes.POINTER(dh_tuning), _i, ctypes.POINTER(_i)],
    "dh_set_tuning": [_i, ctypes.POINTER(dh_tuning)],
    "dh_get_tuning": [_i, ctypes.POINTER(dh_tuning)],
    "dh_set_tuning_cache": [_i, ctypes.c_char_p],
    "dh_autotune": [_i, _p, _i, _i, _p, _p, _p, _i],
    "dh_set_fill_factor_correction": [_i, _i],
    "dh_set_basis_type": [_i, _i],
    "dh_set_ref_calibration": [_i, _p, _i, _i, _i],
    "dh_set_ref_calibration_enabled": [_i, _i],
    "dh_set_basis_transform": [_i, _i, _i, _p],
    "dh_get_output_dims": [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_d)],
    "dh_get_axes": [_i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d)],
    "dh_get_field_dims": [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_d)],
    "dh_process_batch": [_i, _p, _i, _i, _p, _p, _p],
    "dh_process_batch_window": [_i, _p, _i, _i, _p, _p, _p, _p],
    "dh_process_batch_noalloc": [_i, _p, _i, _i, _p, _p, _p],
    "dh_process_batch_avg": [_i, _p, _i, _i, _i, _i, _p, _p, _p],
    "dh_process_batch_host": [_i, _p, _i, _i, _p, _p, _p],
    "dh_process_batch_host_async": [_i, _p, _i, _i, _p, _p, _p],
    "dh_process_batch_host_wait": [_i],
    "dh_get_alignment": [_i, ctypes.POINTER(dh_setting)],
    "dh_calc_metrics": [_i, _p, _i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), _p],
    "dh_auto_align": [_i, _p, _i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), _i, ctypes.POINTER(_d),
                      ctypes.POINTER(_i), _p],
    "dh_score_settings": [_i, _p, _i, _i, ctypes.POINTER(dh_setting), _i, _p, _p],
    "dh_set_profiling": [_i, _i],
    "dh_get_device_status": [_i, ctypes.POINTER(_i)],
    "dh_check_bounded_wait": [ctypes.c_longlong, ctypes.POINTER(_i)],
    "dh_get_check_record": [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "dh_checked_build": [ctypes.POINTER(_i)],
    "dh_check_bounds_probe": [_i],
    "dh_server_create": [ctypes.c_size_t, _i, ctypes.POINTER(_p)],
    "dh_server_submit": [_p, ctypes.POINTER(dh_request), ctypes.POINTER(ctypes.c_uint64)],
    "dh_server_set_admission": [_p, _i, _i],
    "dh_server_wait": [_p, ctypes.c_uint64, _i],
    "dh_server_stats": [_p, ctypes.POINTER(dh_stats)],
    "dh_server_destroy": [_p],
    "dh_get_profile": [_i, _i, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_d),
                       ctypes.POINTER(_i)],
}
_lib.dh_last_error.restype = ctypes.c_char_p
_lib.dh_last_error.argtypes = []
for _name, _args in _PROTOS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _i

# every C-ABI name exported by the library, as declared in include/digholo.h
ABI_NAMES = tuple(_PROTOS) + ("dh_last_error",)


def dh_last_error() -> str:
    return _lib.dh_last_error().decode()


def _check(rc: int) -> None:
    if rc != DH_SUCCESS:
        raise DigHoloError(rc, dh_last_error())


def _frames_ptr(frames, dtype: int) -> int:
    """Address of a frame buffer, after checking that its elements are as wide as dtype says (2 bytes for
    DH_DTYPE_U16, 4 for DH_DTYPE_F32): a mismatch would make the kernels read twice (or half) the buffer."""
    if frames is not None and not isinstance(frames, int):
        width = frames.element_size() if hasattr(frames, "element_size") else getattr(frames, "itemsize", None)
        want = {DH_DTYPE_U16: 2, DH_DTYPE_F32: 4}.get(dtype)
        if width is not None and want is not None and width != want:
            raise ValueError(f"frames have {width}-byte elements but dtype {dtype} needs {want}-byte elements")
    return _ptr(frames)


def _ptr(t) -> int:
    """Device (or host) address of a tensor / integer / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("numpy arrays passed to the library must be C-contiguous")
    return t.ctypes.data


def _stream(s) -> int:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------------------------------ ABI calls


def dh_create() -> int:
    h = _i()
    _check(_lib.dh_create(ctypes.byref(h)))
    return h.value


def dh_destroy(h: int) -> None:
    _check(_lib.dh_destroy(h))


def dh_set_frame(h: int, width: int, height: int, pol_count: int, pixel_size: float) -> None:
    _check(_lib.dh_set_frame(h, width, height, pol_count, pixel_size))


def dh_set_wavelength(h: int, wavelength: float) -> None:
    _check(_lib.dh_set_wavelength(h, wavelength))


def dh_set_fft_window(h: int, nx: int, ny: int):
    a, b = _i(), _i()
    _check(_lib.dh_set_fft_window(h, nx, ny, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def dh_set_beam_centre(h: int, axis: int, pol: int, centre: float) -> None:
    _check(_lib.dh_set_beam_centre(h, axis, pol, centre))


def dh_set_fourier_window_radius(h: int, radius_deg: float) -> None:
    _check(_lib.dh_set_fourier_window_radius(h, radius_deg))


def dh_set_ifft_size(h: int, mx: int, my: int) -> None:
    _check(_lib.dh_set_ifft_size(h, mx, my))


def dh_set_tilt(h: int, axis: int, pol: int, tilt_deg: float) -> None:
    _check(_lib.dh_set_tilt(h, axis, pol, tilt_deg))


def dh_set_defocus(h: int, pol: int, dioptre: float) -> None:
    _check(_lib.dh_set_defocus(h, pol, dioptre))


def dh_set_basis(h: int, pol: int, waist: float, group_count: int) -> None:
    _check(_lib.dh_set_basis(h, pol, waist, group_count))


def dh_set_fill_factor_correction(h: int, enabled: bool) -> None:
    _check(_lib.dh_set_fill_factor_correction(h, 1 if enabled else 0))


def dh_set_ref_calibration(h: int, cal) -> None:
    """cal: uint16 array [height][width] or [wavelengths][height][width] (copied by the library)."""
    import numpy as np
    c = np.ascontiguousarray(np.asarray(cal, dtype=np.uint16))
    if c.ndim == 2:
        c = c[None]
    _check(_lib.dh_set_ref_calibration(h, c.ctypes.data_as(_p), c.shape[0], c.shape[2], c.shape[1]))


def dh_set_ref_calibration_enabled(h: int, enabled: bool) -> None:
    _check(_lib.dh_set_ref_calibration_enabled(h, 1 if enabled else 0))


def dh_set_basis_type(h: int, basis: int) -> None:
    _check(_lib.dh_set_basis_type(h, basis))


def dh_set_basis_transform(h: int, transform) -> None:
    """transform: complex matrix [modes_out][modes_in] (anything numpy converts); copied by the library."""
    import numpy as np
    t = np.ascontiguousarray(np.asarray(transform, dtype=np.complex64))
    if t.ndim != 2:
        raise ValueError("transform must be a 2-D matrix [modes_out][modes_in]")
    _check(_lib.dh_set_basis_transform(h, t.shape[1], t.shape[0], t.ctypes.data_as(_p)))


def dh_set_precision(h: int, precision: int) -> None:
    _check(_lib.dh_set_precision(h, precision))


def dh_set_variant(h: int, variant: int) -> None:
    _check(_lib.dh_set_variant(h, variant))


def dh_get_variant(h: int) -> int:
    v = _i()
    _check(_lib.dh_get_variant(h, ctypes.byref(v)))
    return v.value


def dh_tuning_key(h: int) -> str:
    buf = ctypes.create_string_buffer(256)
    _check(_lib.dh_tuning_key(h, buf, 256))
    return buf.value.decode()


def dh_tuning_candidates(h: int):
    n = _i()
    _check(_lib.dh_tuning_candidates(h, None, 0, ctypes.byref(n)))
    arr = (dh_tuning * max(n.value, 1))()
    _check(_lib.dh_tuning_candidates(h, arr, n.value, ctypes.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def dh_set_tuning(h: int, tuning=None) -> None:
    """tuning: None (defaults and the cache), a dh_tuning, or a dict with variant / chunk_mb / radix."""
    if tuning is None:
        _check(_lib.dh_set_tuning(h, None))
        return
    t = tuning if isinstance(tuning, dh_tuning) else make_tuning(**tuning)
    _check(_lib.dh_set_tuning(h, ctypes.byref(t)))


def dh_get_tuning(h: int) -> dict:
    t = dh_tuning()
    _check(_lib.dh_get_tuning(h, ctypes.byref(t)))
    return t.as_dict()


def dh_set_tuning_cache(h: int, path) -> None:
    _check(_lib.dh_set_tuning_cache(h, None if path is None else os.fsencode(path)))


def dh_autotune(h: int, frames, dtype: int, batch: int, fields=None, coefs=None, stream=None, reps: int = 3) -> None:
    """Time every tuning candidate on these device frames, keep the fastest; fields / coefs receive its results."""
    _check(_lib.dh_autotune(h, _frames_ptr(frames, dtype), dtype, batch, _ptr(fields), _ptr(coefs), _stream(stream), reps))


def dh_get_output_dims(h: int):
    m, modes, dx = _i(), _i(), _d()
    _check(_lib.dh_get_output_dims(h, ctypes.byref(m), ctypes.byref(modes), ctypes.byref(dx)))
    return m.value, modes.value, dx.value


def dh_get_field_dims(h: int):
    """(M_x, M_y, dx', dy'): fields are [M_y][M_x] per polarisation."""
    mx, my, dx, dy = _i(), _i(), _d(), _d()
    _check(_lib.dh_get_field_dims(h, ctypes.byref(mx), ctypes.byref(my), ctypes.byref(dx), ctypes.byref(dy)))
    return mx.value, my.value, dx.value, dy.value


def dh_get_axes(h: int, pol: int):
    mx, my, _, _ = dh_get_field_dims(h)
    x, y = (_d * mx)(), (_d * my)()
    _check(_lib.dh_get_axes(h, pol, x, y))
    return list(x), list(y)


def dh_process_batch(h: int, frames, dtype: int, batch: int, fields=None, coefs=None, stream=None) -> None:
    _check(_lib.dh_process_batch(h, _frames_ptr(frames, dtype), dtype, batch, _ptr(fields), _ptr(coefs), _stream(stream)))


def dh_process_batch_window(h: int, frames, dtype: int, batch: int, window, fields=None, coefs=None,
                            stream=None) -> None:
    _check(_lib.dh_process_batch_window(h, _frames_ptr(frames, dtype), dtype, batch, _ptr(window), _ptr(fields), _ptr(coefs),
                                        _stream(stream)))


def dh_process_batch_host(h: int, frames, dtype: int, batch: int, fields=None, coefs=None, stream=None) -> None:
    """frames, fields, coefs: host tensors or numpy arrays (page-locked for overlapped copies)."""
    _check(_lib.dh_process_batch_host(h, _frames_ptr(frames, dtype), dtype, batch, _ptr(fields), _ptr(coefs), _stream(stream)))


def dh_process_batch_host_async(h: int, frames, dtype: int, batch: int, fields=None, coefs=None, stream=None) -> None:
    """As dh_process_batch_host, returning once queued: the outputs are valid after dh_process_batch_host_wait
    (page-locked host tensors; keep them alive and unread until then)."""
    _check(_lib.dh_process_batch_host_async(h, _frames_ptr(frames, dtype), dtype, batch, _ptr(fields), _ptr(coefs),
                                            _stream(stream)))


def dh_process_batch_host_wait(h: int) -> None:
    _check(_lib.dh_process_batch_host_wait(h))


def dh_process_batch_avg(h: int, frames, dtype: int, batch: int, avg_count: int, avg_mode: int, fields=None,
                         coefs=None, stream=None) -> None:
    _check(_lib.dh_process_batch_avg(h, _frames_ptr(frames, dtype), dtype, batch, avg_count, avg_mode, _ptr(fields), _ptr(coefs),
                                     _stream(stream)))


METRIC_NAMES = ("IL", "MDL", "DIAG", "SNRAVG", "DIAGBEST", "DIAGWORST", "SNRBEST", "SNRWORST", "SNRMG")
NOT_CALCULATED = -3.4028234663852886e38      # -FLT_MAX


def dh_calc_metrics(h: int, coefs, batch: int, mul_conj_trans: bool = False, stream=None):
    """Transfer-matrix metrics (dB) of a device coefficient tensor [batch][pol][modes]: (dict name -> value,
    None when not calculated; the Gram eigenvalues as a list)."""
    rows = min(batch, int(coefs.shape[1]) * int(coefs.shape[2]))
    out = (ctypes.c_double * 9)()
    eig = (ctypes.c_double * max(rows, 1))()
    _check(_lib.dh_calc_metrics(h, _ptr(coefs), batch, 1 if mul_conj_trans else 0, out, eig, _stream(stream)))
    vals = {n: (None if out[i] == NOT_CALCULATED else out[i]) for i, n in enumerate(METRIC_NAMES)}
    return vals, list(eig)[:rows]


def dh_get_alignment(h: int):
    """Current (tilt_deg [P][2], defocus [P], waist [P]) of every polarisation slot (DH_MAX_POLS)."""
    out = dh_setting()
    _check(_lib.dh_get_alignment(h, ctypes.byref(out)))
    return ([[out.tilt_deg[p][0], out.tilt_deg[p][1]] for p in range(DH_MAX_POLS)],
            [out.defocus[p] for p in range(DH_MAX_POLS)], [out.waist[p] for p in range(DH_MAX_POLS)])


def dh_auto_align(h: int, frames, dtype: int, batch: int, steps=None, min_steps=None, max_iter: int = 40,
                  stream=None):
    """Fine-alignment search; returns (total power, scorings).  The final settings are written to the handle."""
    st = None if steps is None else (ctypes.c_double * 3)(*steps)
    lo = None if min_steps is None else (ctypes.c_double * 3)(*min_steps)
    power, its = _d(), _i()
    _check(_lib.dh_auto_align(h, _frames_ptr(frames, dtype), dtype, batch, st, lo, max_iter, ctypes.byref(power), ctypes.byref(its),
                              _stream(stream)))
    return power.value, its.value


def dh_process_batch_noalloc(h: int, frames, dtype: int, batch: int, fields=None, coefs=None, stream=None) -> None:
    """dh_process_batch without device allocation: tables and scratch come from the library's static
    16 MiB device array (see include/digholo.h for the limits and the sharing rules)."""
    _check(_lib.dh_process_batch_noalloc(h, _frames_ptr(frames, dtype), dtype, batch, _ptr(fields), _ptr(coefs), _stream(stream)))


def dh_score_settings(h: int, frames, dtype: int, batch: int, settings, power, stream=None) -> None:
    arr = (dh_setting * len(settings))(*settings)
    _check(_lib.dh_score_settings(h, _frames_ptr(frames, dtype), dtype, batch, arr, len(settings), _ptr(power), _stream(stream)))


def dh_get_device_status(h: int) -> int:
    """Bits of the handle's device status word since the last call (0: no bounded wait ran out)."""
    st = _i()
    _check(_lib.dh_get_device_status(h, ctypes.byref(st)))
    return st.value


DH_STATUS_WAIT_COPY = 1
DH_STATUS_WAIT_MMA = 2
DH_STATUS_BOUNDS = 4


def dh_get_check_record(h: int):
    """The first failed bounds guard since the last call, as (site, offset, extent); (0, 0, 0) when none."""
    a, b, c = _i(), _i(), _i()
    _check(_lib.dh_get_check_record(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def dh_checked_build() -> bool:
    """Whether the loaded library is the bounds-checked build."""
    v = _i()
    _check(_lib.dh_checked_build(ctypes.byref(v)))
    return bool(v.value)


def dh_check_bounds_probe(h: int) -> None:
    _check(_lib.dh_check_bounds_probe(h))


def dh_check_bounded_wait(limit: int) -> bool:
    """Run the kernels' bounded mbarrier wait on a barrier nothing completes; True when it expired."""
    ex = _i()
    _check(_lib.dh_check_bounded_wait(limit, ctypes.byref(ex)))
    return bool(ex.value)


def dh_set_profiling(h: int, enable: bool) -> None:
    _check(_lib.dh_set_profiling(h, 1 if enable else 0))


def dh_get_profile(h: int, max_kernels: int = 16):
    """{kernel name: (launches, total milliseconds)} since the last dh_set_profiling."""
    names = ctypes.create_string_buffer(64 * max_kernels)
    launches = (ctypes.c_longlong * max_kernels)()
    total = (_d * max_kernels)()
    count = _i()
    _check(_lib.dh_get_profile(h, max_kernels, names, launches, total, ctypes.byref(count)))
    out = {}
    for i in range(min(count.value, max_kernels)):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(total[i]))
    return out


def dh_server_create(hbm_budget: int, max_inflight: int = 8) -> int:
    out = _p()
    _check(_lib.dh_server_create(hbm_budget, max_inflight, ctypes.byref(out)))
    return out.value


def dh_server_set_admission(server: int, max_bypass: int, max_wait_ms: int) -> None:
    _check(_lib.dh_server_set_admission(server, max_bypass, max_wait_ms))


def dh_server_submit(server: int, geometry: int, frames, dtype: int, batch: int, fields=None, coefs=None) -> int:
    """Queue a request on host buffers (tensors or addresses); returns its ticket."""
    req = dh_request(geometry, _frames_ptr(frames, dtype), dtype, batch, _ptr(fields), _ptr(coefs))
    t = ctypes.c_uint64()
    _check(_lib.dh_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def dh_server_wait(server: int, ticket: int, timeout_ms: int = -1) -> None:
    _check(_lib.dh_server_wait(server, ticket, timeout_ms))


def dh_server_stats(server: int) -> dict:
    st = dh_stats()
    _check(_lib.dh_server_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in dh_stats._fields_}


def dh_server_destroy(server: int) -> None:
    _check(_lib.dh_server_destroy(server))


# ------------------------------------------------------------------------------------------ convenience


def make_setting(tilt_deg, defocus, waist) -> dh_setting:
    """dh_setting from per-polarisation sequences: tilt_deg[p] = (x, y), defocus[p], waist[p]."""
    s = dh_setting()
    for p in range(len(defocus)):
        s.tilt_deg[p][0] = float(tilt_deg[p][0])
        s.tilt_deg[p][1] = float(tilt_deg[p][1])
        s.defocus[p] = float(defocus[p])
        s.waist[p] = float(waist[p])
    return s


def configure(h: int, setup) -> None:
    """Apply an acquisition description (attributes frame_w, frame_h, pol_count, pixel, wavelength, window,
    beam_centre, tilt_deg, defocus, radius_deg, ifft_size, group_count, waist and optionally precision,
    fill_factor, basis, basis_transform and ref_cal) to a handle through the setters."""
    dh_set_frame(h, setup.frame_w, setup.frame_h, setup.pol_count, setup.pixel)
    dh_set_wavelength(h, setup.wavelength)
    # window and ifft_size: one size for both axes, or (x, y)
    nx, ny = (setup.window, setup.window) if isinstance(setup.window, int) else tuple(setup.window)
    mx, my = (setup.ifft_size, setup.ifft_size) if isinstance(setup.ifft_size, int) else tuple(setup.ifft_size)
    dh_set_fft_window(h, nx, ny)
    dh_set_fourier_window_radius(h, setup.radius_deg)
    dh_set_ifft_size(h, mx, my)
    for p in range(setup.pol_count):
        for ax in range(2):
            dh_set_beam_centre(h, ax, p, setup.beam_centre[p][ax])
            dh_set_tilt(h, ax, p, setup.tilt_deg[p][ax])
        dh_set_defocus(h, p, setup.defocus[p])
        dh_set_basis(h, p, setup.waist[p], setup.group_count)
    dh_set_precision(h, getattr(setup, "precision", DH_PRECISION_FP32))
    dh_set_fill_factor_correction(h, bool(getattr(setup, "fill_factor", False)))
    cal = getattr(setup, "ref_cal", None)
    if cal is not None:
        dh_set_ref_calibration(h, cal)
    basis = getattr(setup, "basis", "hg")
    if basis == "custom":
        dh_set_basis_transform(h, setup.basis_transform)
    else:
        dh_set_basis_type(h, DH_BASIS_LG if basis == "lg" else DH_BASIS_HG)


class Reconstructor:
    """A handle plus output allocation: ``rec(frames)`` returns (fields, coefs) as torch tensors."""

    def __init__(self, setup, precision: int = DH_PRECISION_FP32):
        self.h = dh_create()
        configure(self.h, setup)
        dh_set_precision(self.h, precision)
        self.m, self.modes, self.dx = dh_get_output_dims(self.h)
        self.my = dh_get_field_dims(self.h)[1]
        self.pols = setup.pol_count

    def __call__(self, frames, fields: bool = True, coefs: bool = True, stream=None):
        import torch
        b = frames.shape[0]
        dt = DH_DTYPE_U16 if frames.dtype == torch.uint16 else DH_DTYPE_F32
        f = torch.empty((b, self.pols, self.my, self.m), dtype=torch.complex64, device=frames.device) if fields else None
        c = torch.empty((b, self.pols, self.modes), dtype=torch.complex64, device=frames.device) \
            if (coefs and self.modes) else None
        dh_process_batch(self.h, frames, dt, b, f, c, stream)
        return f, c

    def close(self) -> None:
        if self.h is not None:
            dh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
