"""Failure detection on cuda:0 without a GPU fault: a bounded device wait on
a flag that nothing sets gives up, reports PAM_ERR_TIMEOUT through a status
word the host reads, and leaves the context usable (a fit afterwards still
matches the oracle)."""
import time

import numpy as np
import pytest

import oracle
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
    return torch, pam, torch.device("cuda:0")


def test_a_wait_that_nothing_completes_times_out_and_the_context_survives(env):
    torch, pam, dev = env
    flag = torch.full((1,), -1, dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    code = pam.pam_selftest_wait(0, 20_000_000, flag)  # about 10 ms at 2 GHz
    dt = time.perf_counter() - t0
    assert code == pam.PAM_ERR_TIMEOUT and int(flag.item()) == 1
    assert dt < 5.0
    # the same wait with its arrival completes
    assert pam.pam_selftest_wait(1, 20_000_000, flag) == pam.PAM_OK and int(flag.item()) == 0
    # the context is still usable: a mixed fit (tensor-core Gram) and its parity
    K = fields.voronoi_field(64, n_sites=6, seed=81)
    fit = pam.Fitter((64, 64), (2, 2), 1, (4, 4), device=dev, precision=pam.PAM_PREC_MIXED, k_top=5, levels=1)
    Kd = torch.from_numpy(K).to(dev)
    assert fit.fit(Kd) == 0
    ref = oracle.fit_all(K, (64, 64), (2, 2), 1, (4, 4), oracle.default_params(k_top=5, levels=1))
    e_m, e_o = fit.errors(Kd), oracle.errors(ref, K)
    assert abs(e_m["l1"] - e_o["l1"]) <= 0.01 * e_o["l1"]
