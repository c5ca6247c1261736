"""Parity of the fit on general meshes given as cells (pam_fit_cells,
pam_refine_cells, pam_errors_cells) with the oracle's oracle.fit_cells,
through the C ABI on cuda:0.

Bars as for grids: binary64 form, the same dictionaries (centres bit for
bit), coefficients within 1e-9 (max-norm per subdomain), identical supports
where the oracle's optimality margin exceeds 1e-9, errors within 1e-9
relative and evaluated K* within 1e-10 of the range of K; mixed form, final
L1 within 1 % of the oracle's and per element 1e-3 on log10 where the
dictionaries agree.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

BETA_RTOL = 1e-9
KSTAR_RTOL = 1e-10
LOG10_RTOL = 1e-3
L1_RTOL = 0.01


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    return torch, pam, torch.device("cuda:0")


def _fit(env, x, vol, K, geo, precision=0, **params):
    torch, pam, dev = env
    fit = pam.CellFitter(*geo, x, vol, device=dev, precision=precision, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd)
    torch.cuda.synchronize()
    return fit, Kd


def _compare(got, ref, which=None):
    which = range(len(ref["M"])) if which is None else which
    n_sup = 0
    for s in which:
        m = int(ref["M"][s])
        assert got["M"][s] == m, (s, got["M"][s], m)
        np.testing.assert_array_equal(got["c"][s, :m], ref["c"][s, :m])
        rb, gb = ref["beta"][s, :m], got["beta"][s, :m]
        assert np.abs(gb - rb).max() <= BETA_RTOL * max(1.0, np.abs(rb).max()), (s, np.abs(gb - rb).max())
        if ref["info"][s, 4] > 1e-9:
            np.testing.assert_array_equal(gb != 0, rb != 0)
            n_sup += 1
    return n_sup


def _case(name):
    if name == "grid2d":  # a structured grid handed over as cells
        K2 = fields.voronoi_field(128, n_sites=16, seed=21)
        x, vol, K = fields.grid_as_cells(K2, (128, 128))
        return x, vol, K, ((128, 128), (4, 4), 2, (6, 6)), dict(k_top=12, levels=2)
    if name == "triangles":
        x, vol = fields.triangle_mesh(96, seed=22)
        return x, vol, fields.voronoi_at(x, 20, 22), ((96, 96), (4, 4), 2, (6, 6)), dict(k_top=12, levels=2)
    if name == "graded3d":
        shape = (24, 28, 12)
        x, vol = fields.graded_mesh(shape, seed=23)
        Kg = fields.layered_field(shape, seed=23).reshape(-1)  # one value per element, layered structure
        return x, vol, Kg, (shape, (2, 2, 2), 1, (4, 4, 2)), dict(k_top=6, levels=2)
    if name == "graded1d":
        x, vol = fields.graded_mesh((300,), seed=24)
        K = np.where(x[:, 0] < 0.43, 1e-4, 1e-1) * np.where(x[:, 0] > 0.8, 30.0, 1.0)
        return x, vol, K, ((300,), (3,), 4, (5,)), dict(k_top=4, levels=3)
    raise ValueError(name)


@pytest.mark.parametrize("name", ["grid2d", "triangles", "graded3d", "graded1d"])
def test_cells_binary64_match_the_oracle(env, name):
    torch, pam, dev = env
    x, vol, K, geo, params = _case(name)
    fit, Kd = _fit(env, x, vol, K, geo, **params)
    ref = oracle.fit_cells(x, vol, K, *geo, oracle.default_params(**params))
    assert ref["failed"] == 0
    got = fit.host_model()
    n_sup = _compare(got, ref)
    assert n_sup >= len(ref["M"]) // 2
    assert got["M"].max() > int(np.prod(geo[3]))  # refinement happened
    e_gpu, e_ref = fit.errors(Kd), oracle.errors_cells(ref, x, vol, K)
    for k in ("l1", "l2", "l1_log", "max_log10"):
        assert e_gpu[k] == pytest.approx(e_ref[k], rel=1e-9), k
    rng = np.random.default_rng(25)
    ext = np.asarray(geo[0]) / max(geo[0])
    pts = rng.uniform(0, 1, size=(8000, len(geo[0]))) * ext
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    assert np.abs(out - oracle.evaluate(ref, pts)).max() <= KSTAR_RTOL * (K.max() - K.min())


def test_cells_triangles_sampled_subdomains_of_a_large_mesh(env):
    # 256 x 256 squares cut into 131,072 triangles, 8 x 8 subdomains
    # (overlap 2, about 2,600 elements per patch), 8 x 8 initial centres,
    # 3 levels: the GPU fits all 64, the oracle a sample
    torch, pam, dev = env
    x, vol = fields.triangle_mesh(256, seed=26)
    K = fields.voronoi_at(x, 32, 2)
    geo = ((256, 256), (8, 8), 2, (8, 8))
    params = dict(k_top=37, levels=3)
    fit, Kd = _fit(env, x, vol, K, geo, **params)
    which = [0, 9, 27, 36, 54, 63]
    ref = oracle.fit_cells(x, vol, K, *geo, oracle.default_params(**params), which=which)
    _compare(fit.host_model(), ref, which)


def test_cells_mixed_form(env):
    torch, pam, dev = env
    x, vol = fields.triangle_mesh(128, seed=27)
    K = fields.voronoi_at(x, 24, 27)
    geo = ((128, 128), (4, 4), 2, (8, 8))
    params = dict(k_top=20, levels=3)
    fit, Kd = _fit(env, x, vol, K, geo, precision=pam.PAM_PREC_MIXED, **params)
    ref = oracle.fit_cells(x, vol, K, *geo, oracle.default_params(**params))
    got = fit.host_model()
    flags = got["info"][:, pam.INFO_FLAGS]
    assert np.count_nonzero(flags & pam.FLAG_NOT_CERTIFIED) == 0
    e_m = fit.errors(Kd)
    e_o = oracle.errors_cells(ref, x, vol, K)
    assert abs(e_m["l1"] - e_o["l1"]) <= L1_RTOL * e_o["l1"], (e_m["l1"], e_o["l1"])
    # per element where the refinement made the same decisions
    km = fit.eval(torch.from_numpy(x).to(dev)).cpu().numpy()
    ko = oracle.evaluate(ref, x)
    _, own = oracle.evaluate(ref, x, return_owner=True)
    same = 0
    for s in range(len(ref["M"])):
        m = ref["M"][s]
        if got["M"][s] == m and np.array_equal(got["c"][s, :m], ref["c"][s, :m]):
            same += 1
            sel = own == s
            lg, lo = np.log10(km[sel]), np.log10(ko[sel])
            assert np.all(np.abs(lg - lo) <= LOG10_RTOL * np.maximum(1.0, np.abs(lo))), s
    assert same >= 0.75 * len(ref["M"])


def test_cells_bad_values_and_measures_are_reported(env):
    torch, pam, dev = env
    x, vol = fields.triangle_mesh(16, seed=28)
    K0 = fields.voronoi_at(x, 4, 28)
    for which, bad in (("K", 0.0), ("K", float("nan")), ("vol", 0.0), ("vol", -1.0), ("vol", float("inf"))):
        K, v = K0.copy(), vol.copy()
        (K if which == "K" else v)[37] = bad
        fit = pam.CellFitter((16, 16), (2, 2), 1, (2, 2), x, v, device=dev)
        assert fit.fit(torch.from_numpy(K).to(dev), check=False) == pam.PAM_ERR_NONPOSITIVE_K, (which, bad)


@pytest.mark.parametrize("precision", [0, 1])
def test_cells_mesh_with_a_hole_that_empties_a_patch(env, precision):
    # a subdomain without elements: beta = 0, stopped at level 0, K* = 1 in
    # its core, nothing flagged; the others as the oracle
    torch, pam, dev = env
    h = 1 / 64
    x, vol = fields.triangle_mesh(64, seed=61)
    x, vol = fields.cut_box(x, vol, (14.5 * h, 30.5 * h), (33.5 * h, 49.5 * h))
    K = fields.voronoi_at(x, 10, 61)
    geo = ((64, 64), (4, 4), 1, (4, 4))
    params = dict(k_top=6, levels=2)
    fit, Kd = _fit(env, x, vol, K, geo, precision=precision, **params)
    ref = oracle.fit_cells(x, vol, K, *geo, oracle.default_params(**params))
    got = fit.host_model()
    assert got["info"][9, pam.INFO_N_CELLS] == 0 and got["info"][9, pam.INFO_STOPPED] == 1
    assert not got["beta"][9].any() and got["M"][9] == 16
    assert np.count_nonzero(got["info"][:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED) == 0
    pts = np.array([[24.0 * h, 40.0 * h], [0.5, 0.1], [0.9, 0.9]])
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    assert out[0] == pytest.approx(1.0, rel=1e-6)
    if precision == 0:
        _compare(got, ref)
        np.testing.assert_allclose(out, oracle.evaluate(ref, pts), rtol=1e-10)
        e_gpu, e_ref = fit.errors(Kd), oracle.errors_cells(ref, x, vol, K)
        assert e_gpu["l1"] == pytest.approx(e_ref["l1"], rel=1e-9)
    else:
        e_m, e_o = fit.errors(Kd), oracle.errors_cells(ref, x, vol, K)
        assert abs(e_m["l1"] - e_o["l1"]) <= L1_RTOL * e_o["l1"]


@pytest.mark.parametrize("precision", [0, 1])
def test_cells_warm_start_written_on_a_side_stream(env, precision):
    # pam_fit_cells with warm_start and pam_params.warm_start_event: the
    # coefficients copied into model.beta on another stream after the fit is
    # enqueued are the ones the level-0 solve starts from (the wait comes
    # before the dictionary set-up on element lists): the same bits as the
    # in-line warm start, although beta holds NaN when the fit is enqueued
    torch, pam, dev = env
    x, vol = fields.triangle_mesh(64, seed=62)
    K = fields.voronoi_at(x, 12, 62)
    geo, params = ((64, 64), (4, 4), 1, (4, 4)), dict(k_top=6, levels=0)
    fit, Kd = _fit(env, x, vol, K, geo, precision=precision, **params)
    seed = fit.model.beta.clone()
    seed[:, ::2] = 0.0  # a partial warm start: half the coefficients
    fit.model.beta.copy_(seed)
    assert fit.fit(Kd, levels=0, warm_start=True, check=False) == 0
    b_seq, i_seq = fit.model.beta.cpu().numpy().copy(), fit.model.info.cpu().numpy().copy()
    fit.model.beta.fill_(float("nan"))
    side, ev = torch.cuda.Stream(device=dev), torch.cuda.Event()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        torch.cuda._sleep(20_000_000)  # the copy lands well after the fit is enqueued
        fit.model.beta.copy_(seed)
        ev.record(side)
    assert fit.fit(Kd, levels=0, warm_start=True, warm_start_event=ev, check=False) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fit.model.beta.cpu().numpy(), b_seq)
    np.testing.assert_array_equal(fit.model.info.cpu().numpy(), i_seq)
