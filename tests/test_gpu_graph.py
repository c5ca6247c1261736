"""Deferred-status fits and their capture in a CUDA graph.

With deferred_status = 1 the fit calls launch without synchronising the
host, so a whole step (fit over all levels, evaluation, error measures) can
be captured once and replayed. The replay must reproduce the eager step bit
for bit (every kernel is deterministic), and the deferred status must report
what the synchronous calls report.
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
    return torch, pam, torch.device("cuda:0")


def _fitter(env, prec, K):
    torch, pam, dev = env
    fit = pam.Fitter((128, 128), (4, 4), 2, (4, 4), device=dev, precision=prec, k_top=12, levels=2)
    return fit, torch.from_numpy(np.ascontiguousarray(K)).to(dev)


def _model(fit):
    return [t.cpu().numpy().copy() for t in (fit.model.centres, fit.model.beta, fit.model.info)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_deferred_fit_matches_the_synchronous_fit(env, prec):
    torch, pam, dev = env
    p = pam.PAM_PREC_FP64 if prec == "fp64" else pam.PAM_PREC_MIXED
    K = fields.voronoi_field(n=128, n_sites=24, seed=7)
    fit, Kd = _fitter(env, p, K)
    code = fit.fit(Kd)
    ref = _model(fit)
    fit.model.beta.zero_()
    assert fit.fit(Kd, deferred=True) == 0
    assert fit.status() == code
    for a, b in zip(ref, _model(fit)):
        np.testing.assert_array_equal(a, b)


def test_deferred_status_reports_nonpositive_k(env):
    torch, pam, dev = env
    K = fields.voronoi_field(n=128, n_sites=24, seed=7).copy()
    K[40, 77] = 0.0
    fit, Kd = _fitter(env, pam.PAM_PREC_FP64, K)
    with pytest.raises(pam.PamError) as e:
        fit.fit(Kd)
    assert e.value.code == pam.PAM_ERR_NONPOSITIVE_K
    # deferred: the launches go through (the bad cell fitted as K = 1) and
    # the status keeps the error through pam_refine
    assert fit.fit(Kd, deferred=True) == 0
    assert fit.status() == pam.PAM_ERR_NONPOSITIVE_K
    assert fit.fit(torch.from_numpy(np.ascontiguousarray(fields.voronoi_field(n=128, n_sites=24, seed=7)))
                   .to(dev), deferred=True) == 0
    assert fit.status() == 0  # a new fit starts a new status


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_reproduces_the_eager_step(env, prec):
    torch, pam, dev = env
    p = pam.PAM_PREC_FP64 if prec == "fp64" else pam.PAM_PREC_MIXED
    K = fields.voronoi_field(n=128, n_sites=24, seed=11)
    fit, Kd = _fitter(env, p, K)
    pts = torch.from_numpy(fields.cell_centred_points((96, 80), (1.0, 1.0))).to(dev)
    out = torch.empty(pts.shape[0], dtype=torch.float64, device=dev)
    err = torch.zeros(4, dtype=torch.float64, device=dev)

    def step():
        fit.fit(Kd, deferred=True)
        fit.eval(pts, out=out)
        fit.errors_device(Kd, err)

    step()  # eager, also sizes the evaluation workspace
    torch.cuda.synchronize()
    assert fit.status() == 0
    ref = _model(fit) + [out.cpu().numpy().copy(), err.cpu().numpy().copy()]

    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # a warm-up on the side stream before capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    fit.model.beta.zero_()
    out.zero_()
    err.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert fit.status() == 0
    got = _model(fit) + [out.cpu().numpy(), err.cpu().numpy()]
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    # a new field copied into the captured input buffer refits on replay
    K2 = fields.voronoi_field(n=128, n_sites=24, seed=12)
    Kd.copy_(torch.from_numpy(np.ascontiguousarray(K2)))
    g.replay()
    torch.cuda.synchronize()
    fit2, Kd2 = _fitter(env, p, K2)
    fit2.fit(Kd2)
    for a, b in zip(_model(fit2), _model(fit)):
        np.testing.assert_array_equal(a, b)
    del g


@pytest.mark.parametrize("prec,chunks", [("mixed", 1), ("mixed", 3), ("fp64", 7)])
def test_chunked_evaluation_to_host_matches_one_call(env, prec, chunks):
    # Fitter.eval_to_host: slices of the points evaluated one after another,
    # each copied to pinned host memory on a side stream; the values are
    # those of one pam_eval call, eager and replayed from a CUDA graph
    torch, pam, dev = env
    p = pam.PAM_PREC_FP64 if prec == "fp64" else pam.PAM_PREC_MIXED
    fit, Kd = _fitter(env, p, fields.voronoi_field(n=128, n_sites=24, seed=13))
    fit.fit(Kd)
    pts = torch.from_numpy(fields.cell_centred_points((97, 83), (1.0, 1.0))).to(dev)
    n = pts.shape[0]
    ref = fit.eval(pts).cpu().numpy()
    out = torch.empty(n, dtype=torch.float64, device=dev)
    host = torch.zeros(n, dtype=torch.float64).pin_memory()
    fit.eval_to_host(pts, out, host, chunks=chunks)
    torch.cuda.current_stream().synchronize()  # the current stream waited for the copies
    np.testing.assert_array_equal(host.numpy(), ref)

    side = torch.cuda.Stream(device=dev)

    def body():
        side.wait_stream(torch.cuda.current_stream())
        fit.eval_to_host(pts, out, host, chunks=chunks, copy_stream=side, join=False)
        torch.cuda.current_stream().wait_stream(side)

    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        body()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    host.zero_()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host.numpy(), ref)
    del g
