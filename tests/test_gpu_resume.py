"""Checkpoint and resume (pam_model_save, pam_model_load, pam_resume,
pam_resume_cells) through the C ABI on cuda:0: a fit saved after one
refinement level, loaded into a fresh model and workspace and resumed for
the remaining levels, must meet the same parity bar against the oracle's
uninterrupted fit as an uninterrupted GPU fit (binary64: the same
dictionaries, coefficients within 1e-9; mixed: final L1 within 1 %), and a
blob must survive a save -> load -> save round trip byte for byte.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

BETA_RTOL = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    return torch, pam, torch.device("cuda:0")


def _compare(got, ref):
    for s in range(len(ref["M"])):
        m = int(ref["M"][s])
        assert got["M"][s] == m, (s, got["M"][s], m)
        np.testing.assert_array_equal(got["c"][s, :m], ref["c"][s, :m])
        rb, gb = ref["beta"][s, :m], got["beta"][s, :m]
        assert np.abs(gb - rb).max() <= BETA_RTOL * max(1.0, np.abs(rb).max()), (s, np.abs(gb - rb).max())


def test_resume_binary64_grid(env):
    torch, pam, dev = env
    K = fields.voronoi_field(128, n_sites=16, seed=51)
    geo = ((128, 128), (4, 4), 2, (6, 6))
    params = dict(k_top=12, levels=3)
    Kd = torch.from_numpy(K).to(dev)
    first = pam.Fitter(*geo, device=dev, **params)
    first.fit(Kd, levels=1)
    blob = first.save()
    del first
    second = pam.Fitter(*geo, device=dev, **params)  # fresh model and workspace
    second.load(blob)
    assert second.save() == blob  # round trip
    second.resume(Kd, levels=2)
    torch.cuda.synchronize()
    ref = oracle.fit_all(K, *geo, oracle.default_params(**params))
    got = second.host_model()
    _compare(got, ref)
    assert (got["info"][:, pam.INFO_LEVELS] <= 3).all() and got["M"].max() > 36
    e_gpu, e_ref = second.errors(Kd), oracle.errors(ref, K)
    assert e_gpu["l1"] == pytest.approx(e_ref["l1"], rel=1e-9)


def test_resume_mixed_grid(env):
    torch, pam, dev = env
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    geo = ((256, 256), (8, 8), 2, (8, 8))
    params = dict(k_top=37, levels=3)
    Kd = torch.from_numpy(K).to(dev)
    first = pam.Fitter(*geo, device=dev, precision=pam.PAM_PREC_MIXED, **params)
    first.fit(Kd, levels=2)
    blob = first.save()
    second = pam.Fitter(*geo, device=dev, precision=pam.PAM_PREC_MIXED, **params)
    second.load(blob)
    second.resume(Kd, levels=1)
    torch.cuda.synchronize()
    ref = oracle.fit_all(K, *geo, oracle.default_params(**params))
    e_m, e_o = second.errors(Kd), oracle.errors(ref, K)
    assert abs(e_m["l1"] - e_o["l1"]) <= 0.01 * e_o["l1"], (e_m["l1"], e_o["l1"])
    flags = second.host_model()["info"][:, pam.INFO_FLAGS]
    assert np.count_nonzero(flags & pam.FLAG_NOT_CERTIFIED) == 0


def test_resume_binary64_triangle_mesh(env):
    torch, pam, dev = env
    x, vol = fields.triangle_mesh(64, seed=52)
    K = fields.voronoi_at(x, 10, 52)
    geo = ((64, 64), (2, 2), 2, (5, 5))
    params = dict(k_top=8, levels=2)
    Kd = torch.from_numpy(K).to(dev)
    first = pam.CellFitter(*geo, x, vol, device=dev, **params)
    first.fit(Kd, levels=1)
    blob = first.save()
    second = pam.CellFitter(*geo, x, vol, device=dev, **params)
    second.load(blob)
    second.resume(Kd, levels=1)
    torch.cuda.synchronize()
    ref = oracle.fit_cells(x, vol, K, *geo, oracle.default_params(**params))
    _compare(second.host_model(), ref)


def test_load_rejects_another_problem(env):
    torch, pam, dev = env
    K = fields.voronoi_field(64, n_sites=6, seed=53)
    a = pam.Fitter((64, 64), (2, 2), 1, (4, 4), device=dev, k_top=4, levels=1)
    a.fit(torch.from_numpy(K).to(dev))
    blob = a.save()
    b = pam.Fitter((64, 64), (2, 2), 2, (4, 4), device=dev, k_top=4, levels=1)  # another overlap
    with pytest.raises(pam.PamError):
        b.load(blob)
    bad = bytearray(blob)
    bad[0] = ord("X")
    with pytest.raises(pam.PamError):
        a.load(bytes(bad))
    with pytest.raises(pam.PamError):
        a.load(blob[:-8])
