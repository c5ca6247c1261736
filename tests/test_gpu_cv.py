"""Per-subdomain cross-validation of the Elastic Net weights (pam_lambda_cv)
on the GPU against the oracle's cv_lambda on the same dictionary.

Bar, binary64 form: cross-validation errors within 1e-8 relative (solves
that agree to the certification tolerance), the same chosen grid index
wherever the oracle's best and second-best errors differ by more than 1e-6
relative (elsewhere the GPU's choice is within that band of the least
error), and the refit coefficients within 1e-9 relative (max-norm per
subdomain) where the choices agree. Mixed form: cross-validation errors
within 1e-4 relative (the fp32-certified solves; the largest deviation
measured over all 2,244 subdomains of the 3-D workload was 1e-5), the same
choice wherever the oracle's gap exceeds 1e-3, and the refit log-field on
the patch cells within 1e-3 max(1, |log10 K*|) per cell.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

CV_RTOL = 1e-8
GAP = 1e-6
BETA_RTOL = 1e-9
GRID = [(4.59e-4 * f, 4.64e-6 * f) for f in (0.25, 1.0, 4.0)] + [(1e-5, 1e-6)]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    return torch, pam, torch.device("cuda:0")


MX_CV_RTOL = 1e-4
MX_GAP = 1e-3
MX_LOG10_RTOL = 1e-3


def _run(env, K, n_cells, n_sub, overlap, g, grid, folds, which=None, **params):
    torch, pam, dev = env
    fit = pam.Fitter(n_cells, n_sub, overlap, g, device=dev, precision=pam.PAM_PREC_FP64, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd, check=False)
    before = fit.host_model()
    cv, choice, code = fit.lambda_cv(Kd, grid, folds)
    assert code == 0
    got = fit.host_model()
    cv, choice = cv.cpu().numpy(), choice.cpu().numpy()
    model = dict(before, n_cells=tuple(n_cells), n_sub=tuple(n_sub), m_cap=fit.plan.m_cap)
    ref = oracle.cv_lambda(model, K, grid, folds, which=which)
    which = range(len(choice)) if which is None else which
    agree = 0
    for s in which:
        rc = ref["cv"][s]
        np.testing.assert_allclose(cv[s], rc, rtol=CV_RTOL, err_msg=f"subdomain {s}")
        order = np.argsort(rc, kind="stable")
        gap = (rc[order[1]] - rc[order[0]]) / rc[order[0]] if len(rc) > 1 else np.inf
        if gap > GAP:
            assert choice[s] == ref["choice"][s], (s, choice[s], ref["choice"][s])
        else:
            assert rc[choice[s]] <= rc[order[0]] * (1 + GAP)
        assert ref["certified"][s]
        if choice[s] == ref["choice"][s]:
            m = int(got["M"][s])
            rb, gb = ref["beta"][s, :m], got["beta"][s, :m]
            assert np.abs(gb - rb).max() <= BETA_RTOL * max(1.0, np.abs(rb).max()), s
            agree += 1
        # the dictionary is kept
        np.testing.assert_array_equal(got["c"][s], before["c"][s])
    return cv, choice, agree


def test_voronoi_2d_three_folds(env):
    K = fields.voronoi_field(n=128, n_sites=24, seed=5)
    cv, choice, agree = _run(env, K, (128, 128), (4, 4), 2, (4, 4), GRID, 3, k_top=12, levels=1)
    assert agree >= 12


def test_layered_3d_ragged_folds(env):
    # patches of 8 x 13 x 7 ... cells: fold sizes differ by one (N mod 4 != 0)
    shape = (30, 44, 17)
    K = fields.layered_field(shape=shape, seed=9)
    _run(env, K, shape, (3, 4, 3), 1, (3, 3, 2), GRID[:3], 4, k_top=8, levels=1)


def test_single_pair_refit_is_the_plain_fit(env):
    torch, pam, dev = env
    K = fields.voronoi_field(n=64, n_sites=12, seed=3)
    fit = pam.Fitter((64, 64), (2, 2), 2, (4, 4), device=dev, precision=pam.PAM_PREC_FP64, levels=1, k_top=8)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd)
    ref = fit.host_model()
    cv, choice, code = fit.lambda_cv(Kd, [(fit.params.lambda1_hat, fit.params.lambda2_hat)], 2)
    assert code == 0 and (choice.cpu().numpy() == 0).all()
    got = fit.host_model()
    for s in range(4):
        m = int(ref["M"][s])
        scale = max(1.0, np.abs(ref["beta"][s, :m]).max())
        assert np.abs(got["beta"][s, :m] - ref["beta"][s, :m]).max() <= BETA_RTOL * scale


def test_full_size_layered_workload_sampled(env):
    # the 60 x 220 x 85 workload (2,244 subdomains), checked on a sample
    shape = (60, 220, 85)
    K = fields.layered_field(shape=shape, seed=5)
    which = [0, 517, 1122, 1800, 2243]
    _run(env, K, shape, (6, 22, 17), 1, (4, 4, 2), GRID[:3], 3, which=which, k_top=30, levels=3)


def _run_mixed(env, K, n_cells, n_sub, overlap, g, grid, folds, which=None, **params):
    torch, pam, dev = env
    fit = pam.Fitter(n_cells, n_sub, overlap, g, device=dev, precision=pam.PAM_PREC_MIXED, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd, check=False)
    before = fit.host_model()
    cv, choice, code = fit.lambda_cv(Kd, grid, folds)
    assert code in (0, 5)
    got = fit.host_model()
    n_unc = int(((got["info"][:, 4].astype(np.int64) & 1) != 0).sum())
    assert n_unc <= max(1, len(got["M"]) // 200), n_unc
    cv, choice = cv.cpu().numpy(), choice.cpu().numpy()
    model = dict(before, n_cells=tuple(n_cells), n_sub=tuple(n_sub), m_cap=fit.plan.m_cap)
    ref = oracle.cv_lambda(model, K, grid, folds, which=which)
    which = range(len(choice)) if which is None else which
    dim = len(n_cells)
    worst = 0.0
    for s in which:
        rc = ref["cv"][s]
        worst = max(worst, float(np.max(np.abs(cv[s] - rc) / rc)))
        np.testing.assert_allclose(cv[s], rc, rtol=MX_CV_RTOL, err_msg=f"subdomain {s}")
        order = np.argsort(rc, kind="stable")
        gap = (rc[order[1]] - rc[order[0]]) / rc[order[0]] if len(rc) > 1 else np.inf
        if gap > MX_GAP:
            assert choice[s] == ref["choice"][s], (s, choice[s], ref["choice"][s])
        else:
            assert rc[choice[s]] <= rc[order[0]] * (1 + MX_GAP)
        if choice[s] == ref["choice"][s]:
            b = got["boxes"][s]
            x, _, _ = oracle.box_cells(n_cells, b[6:9], b[9:12], K)
            m = int(got["M"][s])
            W = oracle.assemble(dim, x, got["c"][s, :m])
            lg = (W @ got["beta"][s, :m]) / np.log(10.0)
            lr = (W @ ref["beta"][s, :m]) / np.log(10.0)
            assert np.all(np.abs(lg - lr) <= MX_LOG10_RTOL * np.maximum(1.0, np.abs(lr))), s
        np.testing.assert_array_equal(got["c"][s], before["c"][s])
    return worst


def test_mixed_voronoi_2d_three_folds(env):
    # the mixed form certifies for lambda1_hat down to ~1e-4: below, the fp32
    # rounding of its exact gradient (~1e-6 over ~1e3 cells) exceeds the
    # 1e-4 lambda1 stationarity band, so the 1e-5 pair is left to the binary64 form
    K = fields.voronoi_field(n=128, n_sites=24, seed=5)
    worst = _run_mixed(env, K, (128, 128), (4, 4), 2, (4, 4), GRID[:3], 3, k_top=12, levels=1)
    print("mixed cv max relative deviation", worst)


def test_mixed_full_size_layered_workload_sampled(env):
    shape = (60, 220, 85)
    K = fields.layered_field(shape=shape, seed=5)
    which = [0, 517, 1122, 1800, 2243]
    worst = _run_mixed(env, K, shape, (6, 22, 17), 1, (4, 4, 2), GRID[:3], 3, which=which, k_top=30, levels=3)
    print("mixed cv max relative deviation", worst)
