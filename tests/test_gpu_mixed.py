"""The mixed-precision building blocks on the GPU against the FP64 oracle.

The tensor-core Gram (bf16 hi/lo split, fp32 accumulation) must reproduce
G = W^T W to about 2^-16 relative per entry and b = W^T ln K to fp32
accuracy; the binary64 Gram of the plain form to 1e-12.
"""
import numpy as np
import pytest

import oracle
from oracle_refit import oracle_on_gpu_dictionary
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

G_TC_RTOL = 1e-4      # max |dG| / max |G|: three bf16 products, fp32 accumulation
G_TC_FRO = 3e-5       # Frobenius-relative
B_TC_RTOL = 2e-5      # fp32 accumulation over ~1e3 cells
G_F64_RTOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    return torch, pam, torch.device("cuda:0")


def _gram_case(env, K, n_cells, n_sub, overlap, g, levels_done, which, **params):
    torch, pam, dev = env
    fit = pam.Fitter(n_cells, n_sub, overlap, g, device=dev, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    pam.pam_fit_subdomains(fit.problem, fit.params, fit.plan, Kd, fit.model, fit.workspace)
    if levels_done:
        pam.pam_refine(fit.problem, fit.params, fit.plan, Kd, fit.model, levels_done, fit.workspace)
    S, mc = fit.plan.n_subdomains, fit.plan.m_cap
    out = {}
    for prec in (pam.PAM_PREC_MIXED, pam.PAM_PREC_FP64):
        par = pam.make_params(precision=prec, **params)
        G = torch.zeros((S, mc, mc), dtype=torch.float64, device=dev)
        b = torch.zeros((S, mc), dtype=torch.float64, device=dev)
        pam.pam_gram(fit.problem, par, fit.plan, Kd, fit.model, G, b, fit.workspace)
        out[prec] = (G.cpu().numpy(), b.cpu().numpy())
    model = fit.host_model()
    boxes = model["boxes"]
    checked = 0
    for s in which:
        m = int(model["M"][s])
        bx = boxes[s]
        x, y, _ = oracle.box_cells(n_cells, bx[6:9], bx[9:12], K)
        W = oracle.assemble(len(n_cells), x, model["c"][s, :m])
        Gr, br = oracle.gram(W, y)
        Gt, bt = out[pam.PAM_PREC_MIXED][0][s, :m, :m], out[pam.PAM_PREC_MIXED][1][s, :m]
        gmax = np.abs(Gr).max()
        assert np.abs(Gt - Gr).max() <= G_TC_RTOL * gmax, (s, m, np.abs(Gt - Gr).max() / gmax)
        assert np.linalg.norm(Gt - Gr) <= G_TC_FRO * np.linalg.norm(Gr), (s, m)
        assert np.abs(bt - br).max() <= B_TC_RTOL * np.abs(br).max(), (s, m)
        G6, b6 = out[pam.PAM_PREC_FP64][0][s, :m, :m], out[pam.PAM_PREC_FP64][1][s, :m]
        assert np.abs(G6 - Gr).max() <= G_F64_RTOL * gmax
        assert np.abs(b6 - br).max() <= G_F64_RTOL * np.abs(br).max()
        # nothing written past the dictionary
        assert np.all(out[pam.PAM_PREC_MIXED][0][s, m:, :] == 0)
        checked += 1
    return model, checked


def test_tensor_core_gram_voronoi_multi_strip(env):
    # after 2 refinement levels M reaches 64 + 2 * 111 = 286: three 128-row
    # strips, the last one 32 rows wide
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    model, n = _gram_case(env, K, (256, 256), (8, 8), 2, (8, 8), 2, range(0, 64, 7), k_top=37, levels=3)
    assert model["M"].max() > 256 and n == 10


def test_tensor_core_gram_two_strip_groups(env):
    # after 3 refinement levels M reaches 64 + 3 * 111 = 397 > 384: the padded
    # dictionary (416) needs four 128-row strips whose D blocks do not fit the
    # 512 TMEM columns together, so two CTAs per subdomain each generate W for
    # their own strip group (the benchmark's 3-D dictionaries, M = 392, take
    # the same path)
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    model, n = _gram_case(env, K, (256, 256), (8, 8), 2, (8, 8), 3, range(0, 64, 5), k_top=37, levels=3)
    assert model["M"].max() > 384 and n == 13
    assert sum(int(model["M"][s] > 384) for s in range(0, 64, 5)) >= 3


def test_tensor_core_gram_3d_and_1d(env):
    K = fields.layered_field((20, 30, 12), seed=31)
    _gram_case(env, K, (20, 30, 12), (2, 3, 2), 1, (3, 3, 2), 1, range(12), k_top=10, levels=2)
    K1 = fields.step_field_1d(300, 140)
    _gram_case(env, K1, (300,), (3,), 4, (5,), 1, range(3), k_top=4, levels=2)


def test_tensor_core_gram_single_chunk_and_ragged(env):
    # patches smaller than one 32-cell chunk, and a dictionary of 3 x 5
    K = fields.voronoi_field(37, n_sites=6, seed=32)[:23, :]
    _gram_case(env, K, (37, 23), (8, 6), 0, (3, 5), 0, range(48), k_top=3, levels=1)


# ------------------------------------------------------------------ the fit --
LOG10_RTOL = 1e-3   # per cell: |dlog10 K*| <= 1e-3 max(1, |log10 K*_oracle|)
L1_RTOL = 0.01      # final L1 within 1 % of the oracle's


def _mixed_fit(env, K, n_cells, n_sub, overlap, g, n_refine, **params):
    torch, pam, dev = env
    fit = pam.Fitter(n_cells, n_sub, overlap, g, device=dev, precision=pam.PAM_PREC_MIXED, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    pam.pam_fit_subdomains(fit.problem, fit.params, fit.plan, Kd, fit.model, fit.workspace)
    if n_refine:
        pam.pam_refine(fit.problem, fit.params, fit.plan, Kd, fit.model, n_refine, fit.workspace)
    torch.cuda.synchronize()
    return fit, Kd


def _log10_close(a, b):
    la, lb = np.log10(a), np.log10(b)
    return np.abs(la - lb) <= LOG10_RTOL * np.maximum(1.0, np.abs(lb))


def _cell_centroids(n_cells):
    h = 1.0 / max(n_cells)
    return fields.cell_centred_points(n_cells, [n * h for n in n_cells])


def test_mixed_level0_matches_oracle_per_cell(env):
    torch, pam, dev = env
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    params = dict(k_top=37, levels=3)
    fit, Kd = _mixed_fit(env, K, (256, 256), (8, 8), 2, (8, 8), 0, **params)
    ref = oracle.fit_all(K, (256, 256), (8, 8), 2, (8, 8), oracle.default_params(k_top=37, levels=0))
    got = fit.host_model()
    np.testing.assert_array_equal(got["M"], ref["M"])
    pts = _cell_centroids((256, 256))
    km = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    ko = oracle.evaluate(ref, pts)
    ok = _log10_close(km, ko)
    assert ok.all(), (np.count_nonzero(~ok), np.abs(np.log10(km) - np.log10(ko)).max())
    # the fp64 evaluation of the same mixed model agrees with its fp32 evaluation
    k64 = fit.eval(torch.from_numpy(pts).to(dev), precision=pam.PAM_PREC_FP64).cpu().numpy()
    assert np.abs(np.log(km) - np.log(k64)).max() <= 1e-4


def test_mixed_full_fit_voronoi(env):
    torch, pam, dev = env
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    params = dict(k_top=37, levels=3)
    fit, Kd = _mixed_fit(env, K, (256, 256), (8, 8), 2, (8, 8), 3, **params)
    ref = oracle.fit_all(K, (256, 256), (8, 8), 2, (8, 8), oracle.default_params(**params))
    got = fit.host_model()
    e_m = fit.errors(Kd)
    e_o = oracle.errors(ref, K)
    assert abs(e_m["l1"] - e_o["l1"]) <= L1_RTOL * e_o["l1"], (e_m["l1"], e_o["l1"])
    # where the refinement made the same decisions the surrogates agree per cell
    same = [s for s in range(64) if got["M"][s] == ref["M"][s]
            and np.array_equal(got["c"][s, :ref["M"][s]], ref["c"][s, :ref["M"][s]])]
    assert len(same) >= 48, len(same)
    boxes = ref["boxes"]
    h = 1.0 / 256
    pts = []
    for s in same:
        b = boxes[s]
        xs = (np.arange(b[0], b[3]) + 0.5) * h
        ys = (np.arange(b[1], b[4]) + 0.5) * h
        X, Y = np.meshgrid(xs, ys)
        pts.append(np.stack([X.ravel(), Y.ravel()], 1))
    pts = np.concatenate(pts)
    km = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    ko = oracle.evaluate(ref, pts)
    ok = _log10_close(km, ko)
    assert ok.all(), (np.count_nonzero(~ok), np.abs(np.log10(km) - np.log10(ko)).max())
    # the others: against the oracle's fit of the GPU's own refined dictionary
    for s in sorted(set(range(64)) - set(same)):
        b = boxes[s]
        X, Y = np.meshgrid((np.arange(b[0], b[3]) + 0.5) * h, (np.arange(b[1], b[4]) + 0.5) * h)
        ps = np.stack([X.ravel(), Y.ravel()], 1)
        km = fit.eval(torch.from_numpy(ps).to(dev)).cpu().numpy()
        ko = oracle_on_gpu_dictionary((256, 256), ref, got, s, K, ps)
        assert _log10_close(km, ko).all(), (s, np.abs(np.log10(km) - np.log10(ko)).max())
    flags = got["info"][:, pam.INFO_FLAGS]
    assert np.count_nonzero(flags & pam.FLAG_NOT_CERTIFIED) == 0


def test_mixed_3d_layered_sample(env):
    torch, pam, dev = env
    shape = (60, 220, 85)
    K = fields.layered_field(shape, seed=5)
    params = dict(k_top=30, levels=3)
    fit, Kd = _mixed_fit(env, K, shape, (6, 22, 17), 1, (4, 4, 2), 3, **params)
    which = list(range(0, 2244, 97))
    ref = oracle.fit_all(K, shape, (6, 22, 17), 1, (4, 4, 2), oracle.default_params(**params), which=which)
    got = fit.host_model()
    h = 1.0 / 220
    same, l1m, l1o, den = 0, 0.0, 0.0, 0.0
    bad = 0
    for s in which:
        b = ref["boxes"][s]
        ax = [(np.arange(b[a], b[3 + a]) + 0.5) * h for a in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        km = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
        ko = oracle.evaluate(ref, pts)
        kt = K[b[2]:b[5], b[1]:b[4], b[0]:b[3]].ravel()
        l1m += np.abs(kt - km).sum(); l1o += np.abs(kt - ko).sum(); den += np.abs(kt).sum()
        m = ref["M"][s]
        if got["M"][s] == m and np.array_equal(got["c"][s, :m], ref["c"][s, :m]):
            same += 1
            bad += np.count_nonzero(~_log10_close(km, ko))
        else:  # the oracle's fit of the GPU's own refined dictionary
            kr = oracle_on_gpu_dictionary(shape, ref, got, s, K, pts)
            bad += np.count_nonzero(~_log10_close(km, kr))
    assert same >= 0.75 * len(which), same
    assert bad == 0
    assert abs(l1m - l1o) <= L1_RTOL * l1o, (l1m / den, l1o / den)


def test_mixed_eval_outside_and_empty(env):
    torch, pam, dev = env
    K = fields.voronoi_field(64, n_sites=6, seed=33)
    fit, Kd = _mixed_fit(env, K, (64, 64), (4, 4), 1, (4, 4), 1, k_top=5, levels=1)
    pts = np.array([[-0.1, 0.5], [0.5, 1.2], [0.5, 0.5], [1.0, 1.0], [0.0, 0.0]])
    out = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    assert np.isnan(out[:2]).all() and np.isfinite(out[2:]).all()
    assert fit.eval(torch.zeros((0, 2), dtype=torch.float64, device=dev)).numel() == 0


def test_mixed_channel_field_1024_sample(env):
    torch, pam, dev = env
    K = fields.channel_field(1024, seed=3)
    params = dict(k_top=37, levels=3)
    fit, Kd = _mixed_fit(env, K, (1024, 1024), (32, 32), 2, (8, 8), 3, **params)
    which = list(range(0, 1024, 37))
    ref = oracle.fit_all(K, (1024, 1024), (32, 32), 2, (8, 8), oracle.default_params(**params), which=which)
    got = fit.host_model()
    h = 1.0 / 1024
    same, bad, l1m, l1o = 0, 0, 0.0, 0.0
    for s in which:
        b = ref["boxes"][s]
        xs = (np.arange(b[0], b[3]) + 0.5) * h
        ys = (np.arange(b[1], b[4]) + 0.5) * h
        X, Y = np.meshgrid(xs, ys)
        pts = np.stack([X.ravel(), Y.ravel()], 1)
        km = fit.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
        ko = oracle.evaluate(ref, pts)
        kt = K[b[1]:b[4], b[0]:b[3]].ravel()
        l1m += np.abs(kt - km).sum(); l1o += np.abs(kt - ko).sum()
        m = ref["M"][s]
        if got["M"][s] == m and np.array_equal(got["c"][s, :m], ref["c"][s, :m]):
            same += 1
            bad += np.count_nonzero(~_log10_close(km, ko))
        else:  # the oracle's fit of the GPU's own refined dictionary
            kr = oracle_on_gpu_dictionary((1024, 1024), ref, got, s, K, pts)
            bad += np.count_nonzero(~_log10_close(km, kr))
    assert same >= 0.75 * len(which), same
    assert bad == 0
    assert abs(l1m - l1o) <= L1_RTOL * l1o
    # the workload's own target, the non-matching 1536 x 1536 mesh: every
    # point the sampled subdomains own, per point against the oracle's fit
    # (of the GPU's dictionary where the refinement decided differently)
    mesh = fields.cell_centred_points((1536, 1536), (1.0, 1.0))
    ko, own = oracle.evaluate(ref, mesh, return_owner=True)
    kg = fit.eval(torch.from_numpy(mesh).to(dev)).cpu().numpy()
    n_pts = 0
    for s in which:
        q = own == s
        n_pts += int(q.sum())
        m = ref["M"][s]
        kr = ko[q] if (got["M"][s] == m and np.array_equal(got["c"][s, :m], ref["c"][s, :m])) else \
            oracle_on_gpu_dictionary((1024, 1024), ref, got, s, K, mesh[q])
        assert _log10_close(kg[q], kr).all(), (s, np.abs(np.log10(kg[q]) - np.log10(kr)).max())
    assert n_pts == len(which) * 48 * 48


def test_mixed_gauss_legendre_indicators(env):
    # the mixed form with pam_params.quad = 1 against the oracle on the same
    # rule: final L1 (Gauss-Legendre errors) within 1 %
    torch, pam, dev = env
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    params = dict(k_top=37, levels=3, quad=1)
    fit, Kd = _mixed_fit(env, K, (256, 256), (8, 8), 2, (8, 8), 3, **params)
    ref = oracle.fit_all(K, (256, 256), (8, 8), 2, (8, 8), oracle.default_params(**params))
    e_m = fit.errors(Kd)
    e_o = oracle.errors(ref, K, quad=1)
    assert abs(e_m["l1"] - e_o["l1"]) <= L1_RTOL * e_o["l1"], (e_m["l1"], e_o["l1"])
    flags = fit.host_model()["info"][:, pam.INFO_FLAGS]
    assert np.count_nonzero(flags & pam.FLAG_NOT_CERTIFIED) == 0
