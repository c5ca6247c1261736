"""pam_errors_noalloc: the error reduction for callers that cannot allocate.

Some host programs (a simulator that reserves the whole GPU memory in its own
pool, a real-time loop that cannot afford an allocation) can hand the
library their inputs and outputs but no scratch space. This entry point
keeps its scratch in a fixed array inside the library; its results must
agree with pam_errors (midpoint rule, quad = 0), which takes a caller
workspace, on consecutive calls, and with the FP64 oracle's error reduction
of the same coefficients. This file is collected last so that a failure here
comes after every other test has run; it passes alone in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # different summation order than pam_errors, the same logits and exps
RTOL_ORACLE = 1e-10  # the oracle: host exp/log and another summation order


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    return torch, pam, torch.device("cuda:0")


def _fitted(torch, pam, dev, K, n_cells, n_sub, overlap, g, **params):
    fit = pam.Fitter(n_cells, n_sub, overlap, g, device=dev, **params)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    fit.fit(Kd)
    return fit, Kd


def test_noalloc_errors_match_the_workspace_version_on_consecutive_calls(env):
    torch, pam, dev = env
    cases = [
        (fields.voronoi_field(128, n_sites=12, seed=21), (128, 128), (4, 4), 2, (6, 6)),
        (fields.layered_field((20, 30, 12), seed=22), (20, 30, 12), (2, 3, 2), 1, (3, 3, 2)),
    ]
    for K, n_cells, n_sub, overlap, g in cases:
        fit, Kd = _fitted(torch, pam, dev, K, n_cells, n_sub, overlap, g, k_top=8, levels=2)
        ref = torch.zeros(4, dtype=torch.float64, device=dev)
        pam.pam_errors(fit.problem, fit.plan, fit.model, Kd, ref, fit.workspace, pam.PAM_PREC_FP64, quad=0)
        orc = oracle.errors(fit.host_model(), K, quad=0)
        want = np.array([orc["l1"], orc["l2"], orc["l1_log"], orc["max_log10"]])
        outs = []
        for _ in range(2):  # two calls in a row share the library's scratch array
            out = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
            pam.pam_errors_noalloc(fit.problem, fit.plan, fit.model, Kd, out)
            outs.append(out.cpu().numpy())
        r = ref.cpu().numpy()
        for o in outs:
            np.testing.assert_allclose(o, r, rtol=RTOL, atol=0)
            np.testing.assert_allclose(o, want, rtol=RTOL_ORACLE, atol=0)
        np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_errors_reject_grids_beyond_the_scratch_limit(env):
    torch, pam, dev = env
    K = fields.voronoi_field(32, n_sites=4, seed=23)
    fit, Kd = _fitted(torch, pam, dev, K, (32, 32), (2, 2), 1, (2, 2), k_top=2, levels=1)
    big = pam.make_problem((4097, 4096), (128, 128), 1, (2, 2))  # 16,781,312 cells
    big_plan = pam.pam_plan_create(big, pam.make_params(k_top=2, levels=1))
    err = torch.zeros(4, dtype=torch.float64, device=dev)
    code = pam.lib().pam_errors_noalloc(C.byref(big), C.byref(big_plan), C.byref(fit.model.c_struct()),
                                        C.c_void_p(Kd.data_ptr()), C.c_void_p(err.data_ptr()), None)
    assert code == 6  # PAM_ERR_UNSUPPORTED, nothing launched
