"""Host-only tests of the C ABI: the library loads, exports every declared symbol, validates settings with
the guide's error codes and derives the same geometry as the oracle.  No GPU work is queued here."""
import math
import os
import re

import numpy as np
import pytest

import paper_2204_02348_gb300 as dh
from oracle import digholo_oracle as orc
from synth import holograms as syn

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "digholo.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(dh_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(dh._lib, n), n
    assert set(names) <= set(dh.ABI_NAMES)


def test_error_codes_match_guide_values():
    txt = open(HEADER).read()
    codes = dict(re.findall(r"#define (DH_(?:SUCCESS|ERROR_\w+))\s+(\d+)", txt))
    assert codes == {"DH_SUCCESS": "0", "DH_ERROR_ERROR": "1", "DH_ERROR_INVALIDHANDLE": "2",
                     "DH_ERROR_NULLPOINTER": "3", "DH_ERROR_INVALIDDIMENSION": "5",
                     "DH_ERROR_INVALIDPOLARISATION": "6", "DH_ERROR_INVALIDAXIS": "7",
                     "DH_ERROR_INVALIDARGUMENT": "8", "DH_ERROR_MEMORYALLOCATION": "9",
                     "DH_ERROR_TIMEOUT": "12", "DH_ERROR_CUDA": "13"}


def _code(fn, *a):
    with pytest.raises(dh.DigHoloError) as ei:
        fn(*a)
    return ei.value.code


def test_invalid_handle_and_arguments():
    assert _code(dh.dh_set_frame, 12345, 64, 64, 1, 20e-6) == dh.DH_ERROR_INVALIDHANDLE
    h = dh.dh_create()
    try:
        assert _code(dh.dh_set_frame, h, 0, 64, 1, 20e-6) == dh.DH_ERROR_INVALIDDIMENSION
        assert _code(dh.dh_set_frame, h, 64, 64, 3, 20e-6) == dh.DH_ERROR_INVALIDPOLARISATION
        assert _code(dh.dh_set_frame, h, 64, 64, 1, -1.0) == dh.DH_ERROR_INVALIDARGUMENT
        assert _code(dh.dh_set_beam_centre, h, 2, 0, 0.0) == dh.DH_ERROR_INVALIDAXIS
        assert _code(dh.dh_set_tilt, h, 0, 2, 1.0) == dh.DH_ERROR_INVALIDPOLARISATION
        assert _code(dh.dh_set_wavelength, h, 0.0) == dh.DH_ERROR_INVALIDARGUMENT
        assert _code(dh.dh_set_fourier_window_radius, h, -1.0) == dh.DH_ERROR_INVALIDARGUMENT
        assert _code(dh.dh_set_ifft_size, h, 40, 40) == dh.DH_ERROR_INVALIDDIMENSION
        assert _code(dh.dh_set_ifft_size, h, 16 * 23, 16 * 23) == dh.DH_ERROR_INVALIDDIMENSION  # prime 23
        assert _code(dh.dh_set_basis, h, 0, 100e-6, 40) == dh.DH_ERROR_INVALIDDIMENSION
        assert _code(dh.dh_set_precision, h, 7) == dh.DH_ERROR_INVALIDARGUMENT
        assert _code(dh.dh_set_fft_window, h, 64, 96) == dh.DH_ERROR_INVALIDDIMENSION   # 96: not a power of two
        assert _code(dh.dh_set_fft_window, h, 15, 15) == dh.DH_ERROR_INVALIDDIMENSION
        assert "16" in dh.dh_last_error()
        assert _code(dh.dh_set_ifft_size, h, 32, 40) == dh.DH_ERROR_INVALIDDIMENSION
        # frame geometry never set
        assert _code(dh.dh_get_output_dims, h) == dh.DH_ERROR_INVALIDDIMENSION
    finally:
        dh.dh_destroy(h)
    assert _code(dh.dh_destroy, h) == dh.DH_ERROR_INVALIDHANDLE


def test_fft_window_floors_to_pixel_quanta():
    h = dh.dh_create()
    try:
        assert dh.dh_set_fft_window(h, 130, 140) == (128, 128)   # floor to multiples of 16
        assert dh.dh_set_fft_window(h, 260, 140) == (256, 128)   # each axis on its own
        assert _code(dh.dh_set_fft_window, h, 100, 100) == dh.DH_ERROR_INVALIDDIMENSION  # 96: not a power of two
    finally:
        dh.dh_destroy(h)


@pytest.mark.parametrize("name", ["plain", "batching", "precision", "large_batch"])
def test_output_dims_and_axes_match_oracle(name):
    s = syn.WORKLOADS[name]()
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        m, modes, dx = dh.dh_get_output_dims(h)
        geos = orc.geometries(s)
        assert m == geos[0].x.m
        assert modes == len(orc.mode_list(s.group_count))
        assert dx == pytest.approx(geos[0].x.dx, rel=1e-15)
        for p in range(s.pol_count):
            x, y = dh.dh_get_axes(h, p)
            ox, oy = orc.output_axes(geos[p])
            assert max(abs(a - b) for a, b in zip(x, ox)) == 0.0
            assert max(abs(a - b) for a, b in zip(y, oy)) == 0.0
    finally:
        dh.dh_destroy(h)
    expected_m = {"plain": 32, "batching": 64, "precision": 96, "large_batch": 176}[name]
    assert m == expected_m


def test_window_outside_frame_and_half_plane_rejected():
    s = syn.setup_plain()
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        dh.dh_set_beam_centre(h, 0, 0, 10 * s.pixel)     # window would start at x = -54
        assert _code(dh.dh_get_output_dims, h) == dh.DH_ERROR_INVALIDARGUMENT
        dh.dh_set_beam_centre(h, 0, 0, s.beam_centre[0][0])
        dh.dh_set_tilt(h, 0, 0, -1.0)                     # off-axis term in the missing half plane
        assert _code(dh.dh_get_output_dims, h) == dh.DH_ERROR_INVALIDARGUMENT
        dh.dh_set_tilt(h, 0, 0, 1.0)
        dh.dh_set_ifft_size(h, 0, 0)                      # the guide's rule: 48 for a 128 window at 0.32 w_max
        assert dh.dh_get_output_dims(h)[0] == 48
        dh.dh_set_basis(h, 0, 150e-6, 0)                  # no modal decomposition
        assert dh.dh_get_output_dims(h)[1] == 0
    finally:
        dh.dh_destroy(h)


def test_serving_geometries_are_accepted():
    import numpy as np
    rng = np.random.default_rng(4)
    for kind in syn.SERVING_KINDS:
        for _ in range(5):
            s = syn.serving_geometry(kind, rng)
            h = dh.dh_create()
            try:
                dh.configure(h, s)
                m, modes, _ = dh.dh_get_output_dims(h)
                assert m == orc.geometries(s)[0].x.m and m % 16 == 0
                assert modes == s.group_count * (s.group_count + 1) // 2
            finally:
                dh.dh_destroy(h)


def test_paper_size_rule_table_through_abi():
    # FFT [IFFT] sizes of the Benchmarks table, with the window radius at the non-overlap limit
    for n, m in [(64, 32), (128, 48), (256, 96), (512, 176), (1024, 336)]:
        h = dh.dh_create()
        try:
            px, lam = 20e-6, 1565e-9
            dh.dh_set_frame(h, n, n, 1, px)
            dh.dh_set_wavelength(h, lam)
            dh.dh_set_fft_window(h, n, n)
            dh.dh_set_beam_centre(h, 0, 0, n / 2 * px)
            dh.dh_set_beam_centre(h, 1, 0, n / 2 * px)
            wmax = math.degrees(lam / (2 * px))
            rad = orc.window_radius_fraction() * wmax
            dh.dh_set_fourier_window_radius(h, rad)
            dh.dh_set_tilt(h, 0, 0, orc.rule_tilt(rad))
            dh.dh_set_tilt(h, 1, 0, orc.rule_tilt(rad))
            assert dh.dh_get_output_dims(h)[0] == m
        finally:
            dh.dh_destroy(h)


def test_server_entry_points_fail_cleanly_without_device_work():
    with pytest.raises(dh.DigHoloError) as ei:
        dh.dh_server_submit(0, 0, 0, dh.DH_DTYPE_U16, 1)
    assert ei.value.code == dh.DH_ERROR_INVALIDHANDLE
    with pytest.raises(dh.DigHoloError) as ei:
        dh.dh_server_create(1 << 20, 0)
    assert ei.value.code == dh.DH_ERROR_INVALIDARGUMENT
    with pytest.raises(dh.DigHoloError) as ei:
        dh.dh_server_stats(0)
    assert ei.value.code == dh.DH_ERROR_INVALIDHANDLE


def test_basis_selection_and_output_mode_counts():
    s = syn.setup_plain()                       # G = 4: 10 HG modes
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        modes_hg = s.group_count * (s.group_count + 1) // 2
        assert dh.dh_get_output_dims(h)[1] == modes_hg
        assert _code(dh.dh_set_basis_type, h, 3) == dh.DH_ERROR_INVALIDARGUMENT
        assert _code(dh.dh_set_basis_type, h, -1) == dh.DH_ERROR_INVALIDARGUMENT
        dh.dh_set_basis_type(h, dh.DH_BASIS_CUSTOM)          # no matrix yet: HG coefficients
        assert dh.dh_get_output_dims(h)[1] == modes_hg
        dh.dh_set_basis_type(h, dh.DH_BASIS_LG)
        assert dh.dh_get_output_dims(h)[1] == modes_hg
        dh.dh_set_basis_transform(h, [[1.0] * 12] * 5)        # 5 outputs from 12 inputs
        assert dh.dh_get_output_dims(h)[1] == 5
        dh.dh_set_basis_type(h, dh.DH_BASIS_HG)
        assert dh.dh_get_output_dims(h)[1] == modes_hg
        dh.dh_set_basis_type(h, dh.DH_BASIS_CUSTOM)          # the stored matrix applies again
        assert dh.dh_get_output_dims(h)[1] == 5
        assert dh._lib.dh_set_basis_transform(h, 2, 2, None) == dh.DH_ERROR_NULLPOINTER
        buf = (dh.ctypes.c_float * 8)()
        assert dh._lib.dh_set_basis_transform(h, 0, 2, buf) == dh.DH_ERROR_INVALIDDIMENSION
        assert dh._lib.dh_set_basis_transform(h, 2, -1, buf) == dh.DH_ERROR_INVALIDDIMENSION
        assert dh._lib.dh_set_basis_transform(h, 1 << 13, 1 << 12, buf) == dh.DH_ERROR_INVALIDDIMENSION
        assert dh.dh_get_output_dims(h)[1] == 5                # failed calls keep the settings
        dh.dh_set_basis(h, 0, s.waist[0], 0)                   # G = 0: no coefficients in any basis
        assert dh.dh_get_output_dims(h)[1] == 0
    finally:
        dh.dh_destroy(h)


def test_process_batch_avg_argument_errors_before_device_work():
    s = syn.setup_plain()
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        fake = 16   # never dereferenced: the arguments are rejected first
        assert dh._lib.dh_process_batch_avg(h, None, 0, 1, 2, 0, None, None, None) == dh.DH_ERROR_NULLPOINTER
        assert dh._lib.dh_process_batch_avg(h, fake, 7, 1, 2, 0, None, None, None) == dh.DH_ERROR_INVALIDARGUMENT
        assert dh._lib.dh_process_batch_avg(h, fake, 0, 1, 2, 3, None, None, None) == dh.DH_ERROR_INVALIDARGUMENT
        assert dh._lib.dh_process_batch_avg(h, fake, 0, 1, 2, -1, None, None, None) == dh.DH_ERROR_INVALIDARGUMENT
        assert dh._lib.dh_process_batch_avg(h, fake, 0, 1, dh.DH_MAX_AVG_COUNT + 1, 0, None, None, None) \
            == dh.DH_ERROR_INVALIDDIMENSION
        assert dh._lib.dh_process_batch_avg(12345, fake, 0, 1, 2, 0, None, None, None) == dh.DH_ERROR_INVALIDHANDLE
    finally:
        dh.dh_destroy(h)


def test_process_batch_host_argument_errors_before_device_work():
    h = dh.dh_create()
    try:
        dh.configure(h, syn.setup_plain())
        assert dh._lib.dh_process_batch_host(h, None, 0, 1, None, None, None) == dh.DH_ERROR_NULLPOINTER
        assert dh._lib.dh_process_batch_host(h, 16, 9, 1, None, None, None) == dh.DH_ERROR_INVALIDARGUMENT
        assert dh._lib.dh_process_batch_host(12345, 16, 0, 1, None, None, None) == dh.DH_ERROR_INVALIDHANDLE
    finally:
        dh.dh_destroy(h)


def test_reference_calibration_setters():
    import numpy as np
    s = syn.setup_batching()
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        assert _code(dh.dh_set_ref_calibration_enabled, h, True) == dh.DH_ERROR_INVALIDARGUMENT   # none set yet
        cal, _ = syn.reference_profile(s)
        dh.dh_set_ref_calibration(h, cal)
        assert dh.dh_get_output_dims(h)[0] == 64
        dh.dh_set_ref_calibration_enabled(h, False)
        dh.dh_set_ref_calibration_enabled(h, True)
        # a calibration of another size is rejected when the geometry is validated
        dh.dh_set_ref_calibration(h, np.ones((8, 16), dtype=np.uint16))
        assert _code(dh.dh_get_output_dims, h) == dh.DH_ERROR_INVALIDDIMENSION
        # invalid calls disable the calibration (and so the size mismatch disappears)
        assert _code(dh.dh_set_ref_calibration, h, np.zeros((s.frame_h, s.frame_w), dtype=np.uint16)) \
            == dh.DH_ERROR_INVALIDARGUMENT
        assert dh.dh_get_output_dims(h)[0] == 64
        assert dh._lib.dh_set_ref_calibration(h, None, 1, s.frame_w, s.frame_h) == dh.DH_ERROR_NULLPOINTER
        buf = (dh.ctypes.c_uint16 * 4)(1, 2, 3, 4)
        assert dh._lib.dh_set_ref_calibration(h, buf, 0, 2, 2) == dh.DH_ERROR_INVALIDARGUMENT
        assert dh._lib.dh_set_ref_calibration(h, buf, 1, 0, 2) == dh.DH_ERROR_INVALIDARGUMENT
    finally:
        dh.dh_destroy(h)


def test_alignment_getter_and_search_argument_errors():
    s = syn.setup_batching()
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        tilt, dfc, waist = dh.dh_get_alignment(h)
        assert tilt[1] == list(s.tilt_deg[1]) and dfc[:2] == list(s.defocus) and waist[:2] == list(s.waist)
        bad = (dh.ctypes.c_double * 3)(0.0, 0.1, 0.05)
        assert dh._lib.dh_auto_align(h, 16, 0, 1, bad, None, 10, None, None, None) == dh.DH_ERROR_INVALIDARGUMENT
        assert dh._lib.dh_auto_align(h, None, 0, 1, None, None, 10, None, None, None) == dh.DH_ERROR_NULLPOINTER
        assert dh._lib.dh_calc_metrics(h, None, 4, 0, None, None, None) == dh.DH_ERROR_NULLPOINTER
        dh.dh_set_basis(h, 0, s.waist[0], 0)
        assert dh._lib.dh_auto_align(h, 16, 0, 1, None, None, 10, None, None, None) == dh.DH_ERROR_INVALIDARGUMENT
    finally:
        dh.dh_destroy(h)


def test_frames_element_width_must_match_dtype():
    # the binding refuses frames whose element width contradicts dtype before anything reaches the library, so
    # a uint16 buffer is never read as float32 (twice its bytes)
    import numpy as np
    h = dh.dh_create()
    try:
        dh.configure(h, syn.setup_batching())
        u16 = np.zeros((1, 256, 320), np.uint16)
        f32 = np.zeros((1, 256, 320), np.float32)
        for fn in (dh.dh_process_batch, dh.dh_process_batch_host, dh.dh_process_batch_noalloc):
            with pytest.raises(ValueError):
                fn(h, u16, dh.DH_DTYPE_F32, 1)
            with pytest.raises(ValueError):
                fn(h, f32, dh.DH_DTYPE_U16, 1)
    finally:
        dh.dh_destroy(h)


def test_checked_build_exports_the_same_symbols():
    # the bounds-checked library is the same ABI; it reports itself as checked (no GPU work)
    import ctypes
    path = os.path.join(os.path.dirname(dh.LIB_PATH), "libdigholo_gb300_checked.so")
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    v = ctypes.c_int(-1)
    assert lib.dh_checked_build(ctypes.byref(v)) == 0 and v.value == 1
    assert not dh.dh_checked_build()


@pytest.mark.parametrize("window,ifft", [((128, 64), 0), ((64, 128), (32, 48)), ((256, 128), (96, 48))])
def test_non_square_dims_and_axes_match_oracle(window, ifft):
    # per-axis windows and fields: the library's field size, pitch and axes against the oracle's geometry
    s = syn.with_(syn.setup_batching(), frame_w=640, frame_h=512, window=window, ifft_size=ifft,
                  beam_centre=[(160 * syn.PIXEL, 256 * syn.PIXEL), (480 * syn.PIXEL, 256 * syn.PIXEL)])
    h = dh.dh_create()
    try:
        dh.configure(h, s)
        g = orc.pol_geometry(s, 1)
        mx, my, dx, dy = dh.dh_get_field_dims(h)
        assert (mx, my) == (g.x.m, g.y.m)
        assert dx == pytest.approx(g.x.dx, rel=1e-15) and dy == pytest.approx(g.y.dx, rel=1e-15)
        m, modes, dx1 = dh.dh_get_output_dims(h)
        assert (m, dx1) == (mx, dx) and modes == s.modes
        x, y = dh.dh_get_axes(h, 1)
        xe, ye = orc.output_axes(g)
        assert np.allclose(x, xe, rtol=0, atol=1e-15) and np.allclose(y, ye, rtol=0, atol=1e-15)
        assert len(x) == mx and len(y) == my
    finally:
        dh.dh_destroy(h)
