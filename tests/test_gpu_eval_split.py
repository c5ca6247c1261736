"""pam_eval in two calls (pam_eval_bucket, pam_eval_bucketed).

The bucketing reads only the points and the partition, so it may run on
another stream beside the fit; the evaluation of the bucketed points must
then equal pam_eval bit for bit, in both precisions, with NaN for points
outside the grid, eagerly and inside a replayed CUDA graph.
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


def _points(n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(-0.05, 1.05, size=(n, 2))  # some outside the grid
    pts[:50] = rng.uniform(0, 1, size=(50, 2))
    return pts


@pytest.mark.parametrize("precision", [0, 1])
def test_bucket_beside_the_fit_then_evaluate(env, precision):
    torch, pam, dev = env
    K = fields.voronoi_field(128, n_sites=20, seed=12)
    fit = pam.Fitter((128, 128), (4, 4), 2, (6, 6), device=dev, precision=precision, k_top=12, levels=2)
    Kd = torch.from_numpy(K).to(dev)
    pts = torch.from_numpy(_points(30000, 3)).to(dev)
    fit.fit(Kd)
    ref = fit.eval(pts).clone()
    out = torch.full_like(ref, 7.0)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fit.eval_bucket(pts, out)
    fit.fit(Kd)  # the same fit again on the main stream, beside the bucketing
    torch.cuda.current_stream().wait_stream(side)
    fit.eval_bucketed(pts, out)
    torch.cuda.synchronize()
    a, b = out.cpu().numpy(), ref.cpu().numpy()
    assert np.isnan(a).sum() > 0
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


def test_split_evaluation_in_a_cuda_graph(env):
    torch, pam, dev = env
    K = fields.voronoi_field(128, n_sites=20, seed=13)
    fit = pam.Fitter((128, 128), (4, 4), 2, (6, 6), device=dev, precision=1, k_top=12, levels=2)
    Kd = torch.from_numpy(K).to(dev)
    pts = torch.from_numpy(_points(20000, 4)).to(dev)
    fit.fit(Kd)
    ref = fit.eval(pts).cpu().numpy()
    out = torch.zeros(pts.shape[0], dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(device=dev)

    def body():
        cur = torch.cuda.current_stream()
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            fit.eval_bucket(pts, out)
        fit.fit(Kd, deferred=True)
        cur.wait_stream(side)
        fit.eval_bucketed(pts, out)

    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        body()
    torch.cuda.current_stream().wait_stream(cap)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    for _ in range(2):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert fit.status() == 0
    a = out.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(a), np.isnan(ref))
    np.testing.assert_array_equal(a[~np.isnan(a)], ref[~np.isnan(ref)])
    del g
