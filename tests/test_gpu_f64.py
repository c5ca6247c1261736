"""Parity of the plain (binary64) CUDA path with the FP64 CPU oracle.

Bar (stated per test): the same dictionary sizes and centres, coefficients
within 1e-9 relative (max-norm per subdomain), identical supports where the
oracle's optimality margin exceeds 1e-9, and evaluated K* within 1e-10 of
the range of K. Everything runs through the C ABI on cuda:0.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

BETA_RTOL = 1e-9
KSTAR_RTOL = 1e-10


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    return torch, torch.device("cuda:0")


def _fit_gpu(torch, dev, K, n_cells, n_sub, overlap, g, **params):
    from paper_2605_16564_gb300 import pam
    fit = pam.Fitter(n_cells, n_sub, overlap, g, device=dev, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd)
    torch.cuda.synchronize()
    return fit, Kd


def _compare_models(got, ref, which=None):
    S = len(ref["M"])
    which = range(S) if which is None else which
    n_checked_support = 0
    for s in which:
        m = int(ref["M"][s])
        assert got["M"][s] == m, (s, got["M"][s], m)
        np.testing.assert_array_equal(got["c"][s, :m], ref["c"][s, :m])
        rb, gb = ref["beta"][s, :m], got["beta"][s, :m]
        scale = max(1.0, np.abs(rb).max())
        assert np.abs(gb - rb).max() <= BETA_RTOL * scale, (s, np.abs(gb - rb).max())
        if ref["info"][s, 4] > 1e-9:  # optimality margin of the oracle's solution
            np.testing.assert_array_equal(gb != 0, rb != 0)
            n_checked_support += 1
    return n_checked_support


def _check_eval(fit, torch, dev, ref, pts, K):
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    expect = oracle.evaluate(ref, pts)
    tol = KSTAR_RTOL * (K.max() - K.min())
    both_nan = np.isnan(out) & np.isnan(expect)
    assert np.all(both_nan | (np.abs(out - expect) <= tol)), np.nanmax(np.abs(out - expect))
    return out


def test_disc_single_subdomain_two_levels(torch_dev):
    # 64 x 64 disc, 16 x 16 initial centres, 2 refinement levels, eval on 97 x 97.
    torch, dev = torch_dev
    K = fields.disc_field(64)
    params = dict(k_top=51, levels=2)
    fit, Kd = _fit_gpu(torch, dev, K, (64, 64), (1, 1), 0, (16, 16), **params)
    ref = oracle.fit_all(K, (64, 64), (1, 1), 0, (16, 16), oracle.default_params(**params))
    got = fit.host_model()
    assert got["M"][0] == 256 + 2 * 3 * 51
    _compare_models(got, ref)
    _check_eval(fit, torch, dev, ref, fields.cell_centred_points((97, 97), (1.0, 1.0)), K)
    e_gpu, e_ref = fit.errors(Kd), oracle.errors(ref, K)
    for k in ("l1", "l2", "l1_log", "max_log10"):
        assert e_gpu[k] == pytest.approx(e_ref[k], rel=1e-9)


def test_voronoi_batched_64_subdomains(torch_dev):
    # 256 x 256 Voronoi (32 sites), 8 x 8 subdomains with a 2-cell overlap,
    # 8 x 8 initial centres, 3 levels: every subdomain against the oracle.
    torch, dev = torch_dev
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    params = dict(k_top=37, levels=3)
    fit, Kd = _fit_gpu(torch, dev, K, (256, 256), (8, 8), 2, (8, 8), **params)
    ref = oracle.fit_all(K, (256, 256), (8, 8), 2, (8, 8), oracle.default_params(**params))
    got = fit.host_model()
    n_sup = _compare_models(got, ref)
    assert n_sup >= 60
    assert got["M"].min() >= 64 and got["M"].max() <= 64 + 3 * 3 * 37
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 1, size=(20000, 2))
    _check_eval(fit, torch, dev, ref, pts, K)


def test_layered_3d_full_size_sampled_subdomains(torch_dev):
    # 60 x 220 x 85 layered field, 6 x 22 x 17 subdomains, overlap 1, 4 x 4 x 2
    # initial centres, 3 levels: the GPU fits all 2244 subdomains, the oracle a
    # sample of them; evaluation is checked at points inside the sample.
    torch, dev = torch_dev
    shape = (60, 220, 85)
    K = fields.layered_field(shape, seed=5)
    params = dict(k_top=30, levels=3)
    fit, Kd = _fit_gpu(torch, dev, K, shape, (6, 22, 17), 1, (4, 4, 2), **params)
    which = list(range(0, 2244, 101)) + [2243]
    ref = oracle.fit_all(K, shape, (6, 22, 17), 1, (4, 4, 2), oracle.default_params(**params),
                         which=which)
    got = fit.host_model()
    _compare_models(got, ref, which)
    h = 1.0 / 220
    rng = np.random.default_rng(6)
    pts = []
    for s in which:
        b = ref["boxes"][s]
        lo, hi = b[0:3] * h, b[3:6] * h
        pts.append(lo + rng.uniform(0, 1, size=(200, 3)) * (hi - lo))
    pts = np.concatenate(pts)
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    expect = oracle.evaluate(ref, pts)
    assert np.abs(out - expect).max() <= KSTAR_RTOL * (K.max() - K.min())


def test_ragged_grid_and_odd_dictionary(torch_dev):
    # cores of unequal size (37 x 23 split 4 x 3), a 3 x 5 lattice (M not a
    # multiple of any tile), overlap 3.
    torch, dev = torch_dev
    K = fields.voronoi_field(37, n_sites=7, seed=8)[:23, :]
    params = dict(k_top=4, levels=2)
    fit, Kd = _fit_gpu(torch, dev, K, (37, 23), (4, 3), 3, (3, 5), **params)
    ref = oracle.fit_all(K, (37, 23), (4, 3), 3, (3, 5), oracle.default_params(**params))
    _compare_models(fit.host_model(), ref)
    rng = np.random.default_rng(9)
    pts = rng.uniform(0, 1, size=(5000, 2)) * np.array([1.0, 23 / 37])
    edge = np.array([[0.0, 0.0], [1.0, 23 / 37], [-0.01, 0.1], [0.5, 0.7]])
    _check_eval(fit, torch, dev, ref, np.concatenate([pts, edge]), K)


def test_one_cell_subdomains_1d(torch_dev):
    # every subdomain holds one cell and one centre (N_i = M_i = 1).
    torch, dev = torch_dev
    K = fields.step_field_1d(16, 5)
    params = dict(k_top=1, levels=1)
    fit, Kd = _fit_gpu(torch, dev, K, (16,), (16,), 0, (1,), **params)
    ref = oracle.fit_all(K, (16,), (16,), 0, (1,), oracle.default_params(**params))
    _compare_models(fit.host_model(), ref)


def test_step_1d_refinement_and_nothing_marked(torch_dev):
    torch, dev = torch_dev
    K = fields.step_field_1d(256, 128)
    for eps in (1e-3, 1e3):  # 1e3: every indicator is below tolerance -> stops at once
        params = dict(k_top=2, levels=3, eps_tol_rel=eps)
        fit, Kd = _fit_gpu(torch, dev, K, (256,), (1,), 0, (2,), **params)
        ref = oracle.fit_all(K, (256,), (1,), 0, (2,), oracle.default_params(**params))
        got = fit.host_model()
        _compare_models(got, ref)
        if eps > 1:
            assert got["M"][0] == 2


def test_bad_cell_values_are_reported(torch_dev):
    torch, dev = torch_dev
    from paper_2605_16564_gb300 import pam
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        K = fields.voronoi_field(16, n_sites=3, seed=1)
        K[3, 4] = bad
        fit = pam.Fitter((16, 16), (2, 2), 1, (2, 2), device=dev)
        code = fit.fit(torch.from_numpy(K).to(dev), check=False)
        assert code == 2


def test_two_runs_are_bitwise_identical(torch_dev):
    torch, dev = torch_dev
    K = fields.voronoi_field(128, n_sites=16, seed=10)
    params = dict(k_top=20, levels=2)
    a, _ = _fit_gpu(torch, dev, K, (128, 128), (4, 4), 2, (6, 6), **params)
    b, _ = _fit_gpu(torch, dev, K, (128, 128), (4, 4), 2, (6, 6), **params)
    ma, mb = a.host_model(), b.host_model()
    for k in ("M", "c", "beta"):
        np.testing.assert_array_equal(ma[k], mb[k])


def test_empty_evaluation_is_a_noop(torch_dev):
    torch, dev = torch_dev
    K = fields.voronoi_field(16, n_sites=3, seed=1)
    fit, _ = _fit_gpu(torch, dev, K, (16, 16), (2, 2), 1, (2, 2), k_top=2, levels=1)
    out = fit.eval(torch.zeros((0, 2), dtype=torch.float64, device=dev))
    assert out.numel() == 0


def test_channel_field_1024_sampled_subdomains(torch_dev):
    # 1024 x 1024 channelised field, 32 x 32 subdomains, overlap 2, 8 x 8
    # initial centres, 3 levels: the GPU fits all 1024 subdomains, the oracle
    # a sample of them.
    torch, dev = torch_dev
    K = fields.channel_field(1024, seed=3)
    params = dict(k_top=37, levels=3)
    fit, Kd = _fit_gpu(torch, dev, K, (1024, 1024), (32, 32), 2, (8, 8), **params)
    which = list(range(0, 1024, 53)) + [1023]
    ref = oracle.fit_all(K, (1024, 1024), (32, 32), 2, (8, 8), oracle.default_params(**params), which=which)
    _compare_models(fit.host_model(), ref, which)
    h = 1.0 / 1024
    rng = np.random.default_rng(14)
    pts = np.concatenate([ref["boxes"][s, 0:2] * h + rng.uniform(0, 1, size=(100, 2)) * 32 * h for s in which])
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    assert np.abs(out - oracle.evaluate(ref, pts)).max() <= KSTAR_RTOL * (K.max() - K.min())
    # the workload's own target: the non-matching 1536 x 1536 mesh, every
    # point the sampled subdomains own
    mesh = fields.cell_centred_points((1536, 1536), (1.0, 1.0))
    ko, own = oracle.evaluate(ref, mesh, return_owner=True)
    sel = np.isin(own, which)
    assert sel.sum() == len(which) * 48 * 48
    kg = fit.eval(torch.from_numpy(mesh).to(dev)).cpu().numpy()
    assert np.abs(kg[sel] - ko[sel]).max() <= KSTAR_RTOL * (K.max() - K.min())


@pytest.mark.parametrize("case", ["voronoi2d", "layered3d"])
def test_gauss_legendre_indicators_match_the_oracle(torch_dev, case):
    # pam_params.quad = 1: the indicators R_T (and the errors) on the
    # 2^dim-point Gauss-Legendre rule; same decisions as the oracle's.
    torch, dev = torch_dev
    if case == "voronoi2d":
        K = fields.voronoi_field(64, n_sites=8, seed=34)
        geo = ((64, 64), (2, 2), 1, (4, 4))
    else:
        K = fields.layered_field((24, 44, 17), seed=7)
        geo = ((24, 44, 17), (2, 4, 1), 1, (4, 4, 2))
    params = dict(k_top=5, levels=2, quad=1)
    fit, Kd = _fit_gpu(torch, dev, K, *geo, **params)
    ref = oracle.fit_all(K, *geo, oracle.default_params(**params))
    assert ref["failed"] == 0
    _compare_models(fit.host_model(), ref)
    e_gpu, e_ref = fit.errors(Kd), oracle.errors(ref, K, quad=1)
    for k in ("l1", "l2", "l1_log", "max_log10"):
        assert e_gpu[k] == pytest.approx(e_ref[k], rel=1e-9), k
    # the midpoint errors of the same model differ (the rule is really applied)
    assert fit.errors(Kd, quad=0)["l1"] != pytest.approx(e_gpu["l1"], rel=1e-6)
