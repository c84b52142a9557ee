"""GPU transfer-matrix metrics (dh_calc_metrics) and the fine-alignment search (dh_auto_align) against the
oracle's definitions."""
import math

import numpy as np
import pytest

from gpu_util import COEF_TOL
from oracle import digholo_oracle as orc
from synth import holograms as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _handle(setup):
    import paper_2204_02348_gb300 as dh
    h = dh.dh_create()
    dh.configure(h, setup)
    return h


def _gpu_metrics(setup, coefs, mct=False):
    import torch
    import paper_2204_02348_gb300 as dh
    h = _handle(setup)
    try:
        d = torch.from_numpy(np.ascontiguousarray(coefs.astype(np.complex64))).cuda()
        return dh.dh_calc_metrics(h, d, coefs.shape[0], mct)
    finally:
        dh.dh_destroy(h)


def _same(got, ref):
    for name in orc.METRICS:
        g, r = got[name], ref[name]
        if r is None or g is None:
            assert g is None and r is None, name
        elif math.isinf(r):
            assert g == r, (name, g, r)
        else:
            assert abs(g - r) <= 1e-8 * max(1.0, abs(r)), (name, g, r)


@pytest.mark.parametrize("rows,mct", [(45, False), (45, True), (20, False), (20, True), (130, False)])
def test_metrics_random_batches(rows, mct):
    s = syn.setup_batching()                  # 2 pols x 45 modes = 90 columns
    rng = np.random.default_rng(160 + rows)
    c = (rng.standard_normal((rows, 2, 45)) + 1j * rng.standard_normal((rows, 2, 45))).astype(np.complex64)
    got, eig = _gpu_metrics(s, c, mct)
    ref = orc.transfer_metrics(c.astype(np.complex128), groups=s.group_count, mul_conj_trans=mct)
    _same(got, ref)
    A = c.astype(np.complex128).reshape(rows, 90)
    gram = A @ A.conj().T if rows <= 90 else A.conj().T @ A
    assert np.allclose(np.sort(eig), np.linalg.eigvalsh(gram), rtol=1e-10, atol=1e-10 * np.abs(gram).max())


def test_metrics_near_unitary_transfer_matrix_and_identity():
    s = syn.setup_batching()
    u = syn.haar_unitary(np.random.default_rng(165), 90)
    noise = np.random.default_rng(166).standard_normal((90, 90)) * 1e-3
    c = (u + noise).reshape(90, 2, 45).astype(np.complex64)
    got, _ = _gpu_metrics(s, c)
    _same(got, orc.transfer_metrics(c.astype(np.complex128), groups=s.group_count))
    eye = np.eye(90, dtype=np.complex64).reshape(90, 2, 45)
    got, _ = _gpu_metrics(s, eye)
    _same(got, orc.transfer_metrics(eye.astype(np.complex128), groups=s.group_count))
    assert got["SNRAVG"] == math.inf and got["MDL"] == 0.0


def test_metrics_custom_basis_has_no_group_metric_and_rank_deficient_mdl():
    s = syn.setup_plain()                     # 1 pol, G = 5: 15 modes
    t = np.random.default_rng(167).standard_normal((12, 15))
    c = np.random.default_rng(168).standard_normal((12, 1, 12)).astype(np.complex64)
    got, _ = _gpu_metrics(syn.with_(s, basis="custom", basis_transform=t), c)
    assert got["SNRMG"] is None
    ref = orc.transfer_metrics(c.astype(np.complex128), groups=None)
    _same(got, ref)
    dup = np.concatenate([c[:6], c[:6]]).astype(np.complex64)      # rank 6 of 12
    got, _ = _gpu_metrics(syn.with_(s, basis="custom", basis_transform=t), dup)
    assert got["MDL"] == math.inf


def test_metrics_on_reconstructed_coefficients():
    # a transfer-matrix measurement: frame b carries column b of a Haar unitary (precision workload recipe)
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.with_(syn.setup_batching(), coefs="haar")
    d = syn.make_frames(s, 45, seed=169)
    h = _handle(s)
    try:
        m, modes, _ = dh.dh_get_output_dims(h)
        fr = torch.from_numpy(d["frames"]).cuda()
        c = torch.empty((45, 2, modes), dtype=torch.complex64, device="cuda")
        dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, 45, None, c)
        got, _ = dh.dh_calc_metrics(h, c, 45)
        ref = orc.transfer_metrics(c.cpu().numpy().astype(np.complex128), groups=s.group_count)
    finally:
        dh.dh_destroy(h)
    _same(got, ref)


def test_auto_align_recovers_alignment_and_matches_oracle_power():
    import torch
    import paper_2204_02348_gb300 as dh
    s = syn.setup_plain()
    d = syn.make_frames(s, 1, seed=62)
    off = syn.with_(s, tilt_deg=[(s.tilt_deg[0][0] + 0.03, s.tilt_deg[0][1] - 0.02)], waist=[s.waist[0] * 1.06])
    h = _handle(off)
    try:
        fr = torch.from_numpy(d["frames"]).cuda()
        power, its = dh.dh_auto_align(h, fr, dh.DH_DTYPE_F32, 1, max_iter=60)
        tilt, dfc, waist = dh.dh_get_alignment(h)
    finally:
        dh.dh_destroy(h)
    t_o, d_o, w_o, p_o, its_o = orc.auto_align_tweak(d["frames"], off, max_iter=60)
    # the GPU search ends on a point whose oracle power equals its own and matches the oracle search's optimum
    assert its >= 5
    assert abs(tilt[0][0] - s.tilt_deg[0][0]) < 4e-3 and abs(tilt[0][1] - s.tilt_deg[0][1]) < 4e-3
    assert abs(waist[0] / s.waist[0] - 1.0) < 0.01
    # the oracle's power at the GPU's final settings is the power the GPU reports
    p_at = orc.score_settings(d["frames"], s, np.array([[tilt[0]]]), np.array([[dfc[0]]]), np.array([[waist[0]]])).sum()
    assert power == pytest.approx(p_at, rel=2 * COEF_TOL)
    assert power == pytest.approx(p_o, rel=1e-4)
    p_true = orc.score_settings(d["frames"], s, np.array([s.tilt_deg]), np.array([s.defocus]),
                                np.array([s.waist])).sum()
    assert power >= p_true * (1 - 1e-3)
