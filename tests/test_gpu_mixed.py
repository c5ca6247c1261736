"""The mixed-precision building blocks on the GPU against the FP64 oracle.

The tensor-core Gram (bf16 hi/lo split, fp32 accumulation) must reproduce
G = W^T W to about 2^-16 relative per entry and b = W^T ln K to fp32
accuracy; the binary64 Gram of the plain form to 1e-12.
"""
import numpy as np
import pytest

import oracle
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


def test_tensor_core_gram_3d_and_1d(env):
    K = fields.layered_field((20, 30, 12), seed=31)
    _gram_case(env, K, (20, 30, 12), (2, 3, 2), 1, (3, 3, 2), 1, range(12), k_top=10, levels=2)
    K1 = fields.step_field_1d(300, 140)
    _gram_case(env, K1, (300,), (3,), 4, (5,), 1, range(3), k_top=4, levels=2)


def test_tensor_core_gram_single_chunk_and_ragged(env):
    # patches smaller than one 32-cell chunk, and a dictionary of 3 x 5
    K = fields.voronoi_field(37, n_sites=6, seed=32)[:23, :]
    _gram_case(env, K, (37, 23), (8, 6), 0, (3, 5), 0, range(48), k_top=3, levels=1)
