"""Subdomain groups of the refinement levels (pam_tuning.level_groups).

With two groups the even and the odd subdomains run their refinement levels
(marking, statistics, Gram, solve, binary64 fallback) on two streams. The
subdomains of section 2 are independent, so the fit must be the same bits as
one pipeline's: dictionaries, coefficients, info words and the evaluation,
in eager launches and in a replayed CUDA graph, for an odd number of
subdomains, and with the binary64 fallback taking subdomains in both groups.
"""
import numpy as np
import pytest

from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    yield torch, pam, torch.device("cuda:0")
    pam.pam_tuning_set(reset=True)


def _fit(env, K, geo, groups, pts, **params):
    torch, pam, dev = env
    pam.pam_tuning_set(level_groups=groups)
    try:
        fit = pam.Fitter(*geo, device=dev, precision=pam.PAM_PREC_MIXED, **params)
        Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
        code = fit.fit(Kd, check=False)
        out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        pam.pam_tuning_set(reset=True)
    return fit, code, fit.host_model(), out


def _same(a, b):
    for key in ("M", "c", "beta", "info"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_two_groups_match_one_pipeline_2d(env):
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    geo = ((256, 256), (8, 8), 2, (8, 8))
    pts = np.random.default_rng(5).uniform(0, 1, size=(20000, 2))
    _, c1, one, o1 = _fit(env, K, geo, 1, pts, k_top=37, levels=3)
    _, c2, two, o2 = _fit(env, K, geo, 2, pts, k_top=37, levels=3)
    assert c1 == c2 == 0
    _same(one, two)
    np.testing.assert_array_equal(o1, o2)


def test_two_groups_with_gauss_legendre_indicators(env):
    # quad = 1: the indicators come from their own kernel at the start of
    # each refinement round, launched per group
    K = fields.voronoi_field(192, n_sites=24, seed=3)
    geo = ((192, 192), (6, 6), 2, (6, 6))
    pts = np.random.default_rng(7).uniform(0, 1, size=(10000, 2))
    _, c1, one, o1 = _fit(env, K, geo, 1, pts, k_top=20, levels=2, quad=1)
    _, c2, two, o2 = _fit(env, K, geo, 2, pts, k_top=20, levels=2, quad=1)
    assert c1 == c2 == 0
    _same(one, two)
    np.testing.assert_array_equal(o1, o2)


def test_two_groups_odd_count_3d(env):
    # 5 x 3 x 3 = 45 subdomains: 23 in the even group, 22 in the odd one
    shape = (40, 24, 18)
    K = fields.layered_field(shape, seed=7)
    geo = (shape, (5, 3, 3), 1, (3, 3, 2))
    pts = np.random.default_rng(6).uniform(0, 1, size=(20000, 3)) * (np.array(shape) / max(shape))
    _, c1, one, o1 = _fit(env, K, geo, 1, pts, k_top=12, levels=2)
    _, c2, two, o2 = _fit(env, K, geo, 2, pts, k_top=12, levels=2)
    assert c1 == c2 == 0
    _same(one, two)
    np.testing.assert_array_equal(o1, o2)


def test_two_groups_in_a_cuda_graph(env):
    torch, pam, dev = env
    K = fields.voronoi_field(192, n_sites=24, seed=9)
    geo = ((192, 192), (6, 6), 2, (6, 6))
    pts = np.random.default_rng(8).uniform(0, 1, size=(10000, 2))
    _, _, one, o1 = _fit(env, K, geo, 1, pts, k_top=20, levels=2)
    pam.pam_tuning_set(level_groups=2)
    try:
        fit = pam.Fitter(*geo, device=dev, precision=pam.PAM_PREC_MIXED, k_top=20, levels=2)
        Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
        ptsd = torch.from_numpy(pts).to(dev)
        out = torch.empty(pts.shape[0], dtype=torch.float64, device=dev)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # one eager pass before capture
            fit.fit(Kd, deferred=True)
            fit.eval(ptsd, out=out)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fit.fit(Kd, deferred=True)
            fit.eval(ptsd, out=out)
        for _ in range(2):
            out.fill_(0)
            g.replay()
        torch.cuda.synchronize()
        assert fit.status() == 0
        _same(one, fit.host_model())
        np.testing.assert_array_equal(out.cpu().numpy(), o1)
        del g
    finally:
        pam.pam_tuning_set(reset=True)


def test_two_groups_with_the_binary64_fallback(env):
    # lambda1 small enough that fp32 solves fail their check: the fallback
    # runs in both groups, each on its share of the slots (5 x 5 = 25
    # subdomains and 25 slots: 13 even subdomains with 13 slots, 12 odd with
    # 12, so every uncertified subdomain finds a slot, as in the one list)
    _, pam, _ = env
    K = fields.voronoi_field(100, n_sites=14, seed=42)
    geo = ((100, 100), (5, 5), 2, (6, 6))
    pts = np.random.default_rng(4).uniform(0, 1, size=(5000, 2))
    params = dict(k_top=8, levels=2, lambda1_hat=1e-5)
    _, c1, one, o1 = _fit(env, K, geo, 1, pts, **params)
    _, c2, two, o2 = _fit(env, K, geo, 2, pts, **params)
    assert c1 == c2 == 0
    div = (two["info"][:, pam.INFO_FLAGS] & pam.FLAG_REFINE_DIVERGED) != 0
    assert div[0::2].any() and div[1::2].any(), "the fallback did not run in both groups"
    _same(one, two)
    np.testing.assert_array_equal(o1, o2)
