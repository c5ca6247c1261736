"""Parity of the glued evaluation (pam_eval_glued) with the oracle's
oracle.evaluate_glued, through the C ABI on cuda:0.

The GPU fits with the CUDA path and the oracle fits independently (the fit
parity itself is covered by test_gpu_f64.py); both glued evaluations then
run on their own models. Bars: binary64 form, K* within 1e-10 of the range
of K and ln K* within 1e-9 max(1, |ln K*|) (the coefficient tolerance
carried through a convex combination); the mixed form, ln K* per point
within 1e-3 max(1, |log10 K*|) on log10 (the mixed-form tolerance) and the
L1 of a mixed fit's glued field within 1 % of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

KSTAR_RTOL = 1e-10
LOG_RTOL = 1e-9
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


def _fit(env, K, geo, precision=0, **params):
    torch, pam, dev = env
    fit = pam.Fitter(*geo, device=dev, precision=precision, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd)
    torch.cuda.synchronize()
    return fit, Kd


_VORONOI = {}


def _voronoi(env, precision=0):
    """The 256 x 256 Voronoi workload (8 x 8 subdomains, overlap 2, 3 levels):
    the GPU fit in the given form and the oracle's fit, made once."""
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    geo = ((256, 256), (8, 8), 2, (8, 8))
    params = dict(k_top=37, levels=3)
    if "ref" not in _VORONOI:
        _VORONOI["ref"] = oracle.fit_all(K, *geo, oracle.default_params(**params))
    if precision not in _VORONOI:
        _VORONOI[precision] = _fit(env, K, geo, precision=precision, **params)[0]
    return K, _VORONOI[precision], _VORONOI["ref"]


def _interface_points(n_cells, n_sub, band, rng, per_face=64):
    """Points on, beside and across every interior core face (and the
    corners where they meet), plus the band edges exactly."""
    dim = len(n_cells)
    h = 1.0 / max(n_cells)
    ext = np.asarray(n_cells) * h
    out = []
    for a in range(dim):
        for j in range(1, n_sub[a]):
            f = (j * n_cells[a]) // n_sub[a] * h
            p = rng.uniform(0, 1, size=(per_face, dim)) * ext
            offs = np.concatenate([[0.0, band * h, -band * h, 1e-12], rng.uniform(-1.2, 1.2, per_face - 4) * band * h])
            p[:, a] = f + offs
            out.append(p)
    faces = [[(j * n_cells[a]) // n_sub[a] * h for j in range(1, n_sub[a])] or [0.5 * ext[a]] for a in range(dim)]
    corners = np.array(np.meshgrid(*faces, indexing="ij")).reshape(dim, -1).T
    for c in corners[:16]:
        out.append(c + rng.uniform(-1, 1, size=(16, dim)) * band * h)
        out.append(c[None, :])
    pts = np.concatenate(out)
    return np.clip(pts, 0.0, ext)


def _check_fp64(env, fit, ref, K, pts, band):
    torch, pam, dev = env
    P = torch.from_numpy(pts).to(dev)
    got = fit.eval_glued(P, band).cpu().numpy()
    want = oracle.evaluate_glued(ref, pts, band)
    nan_mismatch = np.flatnonzero(np.isnan(got) != np.isnan(want))
    assert nan_mismatch.size == 0, (band, nan_mismatch.size, pts[nan_mismatch[:5]], got[nan_mismatch[:5]],
                                    want[nan_mismatch[:5]])
    both_nan = np.isnan(got) & np.isnan(want)
    tol = KSTAR_RTOL * (K.max() - K.min())
    err = np.where(both_nan, 0.0, np.abs(got - want))
    assert np.all(err <= tol), (band, np.nanmax(err), tol)
    gl = fit.eval_glued(P, band, log_space=True).cpu().numpy()
    wl = oracle.evaluate_glued(ref, pts, band, log_space=True)
    ok = (np.isnan(gl) & np.isnan(wl)) | (np.abs(gl - wl) <= LOG_RTOL * np.maximum(1.0, np.abs(wl)))
    assert ok.all(), (band, np.nanmax(np.abs(gl - wl)))
    return got


def test_glued_voronoi_2d_matches_the_oracle(env):
    # 256 x 256 Voronoi, 8 x 8 subdomains (cores of 32), overlap 2, 3 levels;
    # bands from one cell up to the largest allowed (half a core).
    torch, pam, dev = env
    K, fit, ref = _voronoi(env)
    rng = np.random.default_rng(41)
    for band in (1.0, 2.5, 16.0):
        pts = np.concatenate([rng.uniform(0, 1, size=(6000, 2)), _interface_points((256, 256), (8, 8), band, rng),
                              np.array([[-0.01, 0.5], [0.5, 1.01], [0.0, 0.0], [1.0, 1.0]])])
        got = _check_fp64(env, fit, ref, K, pts, band)
        assert np.isnan(got[-4:-2]).all() and np.isfinite(got[:-4]).all() and np.isfinite(got[-2:]).all()


def test_glued_equals_piecewise_away_from_the_bands(env):
    # farther than the band from every interior face the weight of the owner
    # is exactly 1 and the others 0: the glued value is the piecewise value
    # (the same local evaluation; equal up to the compiler's contraction)
    torch, pam, dev = env
    K = fields.voronoi_field(128, n_sites=12, seed=42)
    fit, _ = _fit(env, K, ((128, 128), (4, 4), 2, (6, 6)), k_top=10, levels=2)
    rng = np.random.default_rng(43)
    pts = rng.uniform(0, 1, size=(40000, 2))
    band = 3.0
    d = np.abs(((pts * 128) + 16) % 32 - 16)  # cells to the nearest core face
    far = pts[np.all(d > band + 1e-6, axis=1)]
    P = torch.from_numpy(far).to(dev)
    for prec in (pam.PAM_PREC_FP64, pam.PAM_PREC_MIXED):
        a = fit.eval_glued(P, band, precision=prec).cpu().numpy()
        b = fit.eval(P, precision=prec).cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)


def test_glued_3d_ragged_cores_and_corners(env):
    # ragged cores (24 x 44 x 17 split 3 x 4 x 2), eight subdomains meeting
    # at interior corners; the largest band is limited by the 8-cell cores
    torch, pam, dev = env
    n_cells = (24, 44, 17)
    K = fields.layered_field(n_cells, seed=44)
    geo = (n_cells, (3, 4, 2), 1, (4, 4, 2))
    params = dict(k_top=6, levels=2)
    fit, _ = _fit(env, K, geo, **params)
    ref = oracle.fit_all(K, *geo, oracle.default_params(**params))
    rng = np.random.default_rng(45)
    h = 1.0 / 44
    for band in (0.75, 4.0):
        pts = np.concatenate([rng.uniform(0, 1, size=(4000, 3)) * np.asarray(n_cells) * h,
                              _interface_points(n_cells, (3, 4, 2), band, rng, per_face=48)])
        _check_fp64(env, fit, ref, K, pts, band)


def test_glued_1d(env):
    torch, pam, dev = env
    K = fields.step_field_1d(300, 140)
    geo = ((300,), (3,), 4, (5,))
    params = dict(k_top=4, levels=2)
    fit, _ = _fit(env, K, geo, **params)
    ref = oracle.fit_all(K, *geo, oracle.default_params(**params))
    pts = np.linspace(-0.01, 1.01, 5001)[:, None]
    _check_fp64(env, fit, ref, K, pts, 50.0)
    _check_fp64(env, fit, ref, K, pts, 0.5)


def test_glued_full_size_layered_3d_sampled(env):
    # the 60 x 220 x 85 workload (2,244 subdomains, 3 levels) fitted on the
    # GPU; the oracle fits two 3 x 3 x 3 blocks of subdomains, and points in
    # the central core of each block (whose weights involve only the block)
    # are compared, the band at its largest (2.5 cells: cores of 5 along z)
    torch, pam, dev = env
    shape, n_sub = (60, 220, 85), (6, 22, 17)
    K = fields.layered_field(shape, seed=5)
    geo = (shape, n_sub, 1, (4, 4, 2))
    params = dict(k_top=30, levels=3)
    fit, _ = _fit(env, K, geo, **params)
    centres = [(2, 10, 8), (4, 17, 3)]
    which = sorted({(i + di) + 6 * ((j + dj) + 22 * (k + dk)) for (i, j, k) in centres
                    for di in (-1, 0, 1) for dj in (-1, 0, 1) for dk in (-1, 0, 1)})
    ref = oracle.fit_all(K, *geo, oracle.default_params(**params), which=which)
    h = 1.0 / 220
    rng = np.random.default_rng(46)
    pts = []
    for (i, j, k) in centres:
        s = i + 6 * (j + 22 * k)
        lo, hi = ref["boxes"][s, 0:3] * h, ref["boxes"][s, 3:6] * h
        pts.append(lo + rng.uniform(0, 1, size=(1500, 3)) * (hi - lo))
        pts.append(np.array([lo, hi - 1e-12, 0.5 * (lo + hi)]))
    pts = np.concatenate(pts)
    _check_fp64(env, fit, ref, K, pts, 2.5)
    _check_fp64(env, fit, ref, K, pts, 0.5)


def test_glued_mixed_evaluation_of_a_binary64_fit(env):
    # the same binary64 model evaluated glued in the mixed form (local
    # surrogates in fp32) against the oracle's glued field
    torch, pam, dev = env
    K, fit, ref = _voronoi(env)
    rng = np.random.default_rng(47)
    band = 4.0
    pts = np.concatenate([rng.uniform(0, 1, size=(20000, 2)), _interface_points((256, 256), (8, 8), band, rng)])
    P = torch.from_numpy(pts).to(dev)
    got = fit.eval_glued(P, band, precision=pam.PAM_PREC_MIXED).cpu().numpy()
    want = oracle.evaluate_glued(ref, pts, band)
    lg, lw = np.log10(got), np.log10(want)
    assert np.all(np.abs(lg - lw) <= LOG10_RTOL * np.maximum(1.0, np.abs(lw))), np.abs(lg - lw).max()
    assert np.abs(np.log(got) - np.log(want)).max() <= 1e-4


def test_glued_mixed_fit_l1_within_one_percent(env):
    # a mixed-form fit (tensor-core Gram, fp32 solve) evaluated glued at every
    # cell centroid: its L1 error against K within 1 % of the oracle's glued L1
    torch, pam, dev = env
    K, fit, ref = _voronoi(env, pam.PAM_PREC_MIXED)
    pts = fields.cell_centred_points((256, 256), (1.0, 1.0))
    band = 2.0
    got = fit.eval_glued(torch.from_numpy(pts).to(dev), band).cpu().numpy()
    want = oracle.evaluate_glued(ref, pts, band)
    k = K.reshape(-1)
    l1m, l1o = np.abs(k - got).sum() / np.abs(k).sum(), np.abs(k - want).sum() / np.abs(k).sum()
    assert abs(l1m - l1o) <= L1_RTOL * l1o, (l1m, l1o)


def test_glued_empty_outside_and_deterministic(env):
    torch, pam, dev = env
    K = fields.voronoi_field(64, n_sites=6, seed=48)
    fit, _ = _fit(env, K, ((64, 64), (4, 4), 1, (4, 4)), k_top=5, levels=1)
    assert fit.eval_glued(torch.zeros((0, 2), dtype=torch.float64, device=dev), 2.0).numel() == 0
    pts = np.array([[-0.1, 0.5], [0.5, 1.2], [np.nan, 0.5], [0.5, 0.5], [1.0, 1.0], [0.0, 0.0], [0.25, 0.25]])
    out = fit.eval_glued(torch.from_numpy(pts).to(dev), 2.0).cpu().numpy()
    assert np.isnan(out[:3]).all() and np.isfinite(out[3:]).all()
    rng = np.random.default_rng(49)
    P = torch.from_numpy(rng.uniform(0, 1, size=(50000, 2))).to(dev)
    a = fit.eval_glued(P, 8.0).cpu().numpy()
    b = fit.eval_glued(P, 8.0).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    with pytest.raises(pam.PamError):
        fit.eval_glued(P, 8.5)  # more than half a 16-cell core
    with pytest.raises(pam.PamError):
        fit.eval_glued(P, 0.0)
