"""The autotuner (pam_autotune) and the process-wide launch tuning on
cuda:0: the tuned knobs change launch shapes only, so a fit and an
evaluation under the tuned settings are bit-identical to those under the
built-in settings, and every tuned choice is one of the candidates."""
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


def _run(env, K, geo, pts, precision, **params):
    torch, pam, dev = env
    fit = pam.Fitter(*geo, device=dev, precision=precision, **params)
    Kd = torch.from_numpy(K).to(dev)
    fit.fit(Kd)
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    return fit, Kd, fit.host_model(), out


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_choices_and_bitwise_invariance(env, precision):
    torch, pam, dev = env
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    geo = ((256, 256), (8, 8), 2, (8, 8))
    params = dict(k_top=37, levels=3)
    pts = np.random.default_rng(71).uniform(0, 1, size=(30000, 2))
    pam.pam_tuning_set(reset=True)
    fit, Kd, base, out0 = _run(env, K, geo, pts, precision, **params)
    choice, ms = fit.autotune(Kd, torch.from_numpy(pts).to(dev))
    assert choice == pam.pam_tuning_get()
    assert choice["eval_block"] in (0, 128, 512, 1024) and (ms[8:12] > 0).all()  # 0: the built-in 256
    if precision == 1:
        assert choice["gram_stages"] in (2, 3) and choice["factor_kb"] in (0, 64, 48, 32, 24, 16)
        assert (ms[:2] > 0).all() and (ms[2:8] != 0).all() and (ms[12:14] > 0).all()
        assert choice["solve_persistent"] in (0, 1)
    else:
        assert (ms[:8] == -1).all() and (ms[12:14] == -1).all()
    # force the non-default candidates too: results must not move
    for tuned in (choice, dict(factor_kb=16, gram_stages=2, eval_block=1024, solve_persistent=1),
                  dict(solve_persistent=1)):
        pam.pam_tuning_set(**tuned)
        _, _, got, out = _run(env, K, geo, pts, precision, **params)
        for key in ("M", "c", "beta"):
            np.testing.assert_array_equal(got[key], base[key])
        np.testing.assert_array_equal(out, out0)
    pam.pam_tuning_set(reset=True)


def test_autotune_on_a_triangle_mesh(env):
    torch, pam, dev = env
    x, vol = fields.triangle_mesh(96, seed=72)
    K = fields.voronoi_at(x, 20, 72)
    geo = ((96, 96), (4, 4), 2, (6, 6))
    params = dict(k_top=12, levels=2, precision=pam.PAM_PREC_MIXED)
    pts = np.random.default_rng(73).uniform(0, 1, size=(20000, 2))
    Kd = torch.from_numpy(K).to(dev)
    P = torch.from_numpy(pts).to(dev)
    pam.pam_tuning_set(reset=True)
    a = pam.CellFitter(*geo, x, vol, device=dev, **params)
    a.fit(Kd)
    base, out0 = a.host_model(), a.eval(P).cpu().numpy()
    choice, ms = a.autotune(Kd, P)
    assert choice == pam.pam_tuning_get() and (ms[:2] > 0).all()
    b = pam.CellFitter(*geo, x, vol, device=dev, **params)
    b.fit(Kd)
    got = b.host_model()
    for key in ("M", "c", "beta"):
        np.testing.assert_array_equal(got[key], base[key])
    np.testing.assert_array_equal(b.eval(P).cpu().numpy(), out0)
    pam.pam_tuning_set(reset=True)
