"""One field split over ranks (section 8(e)), on one GPU: each shard fits
only its contiguous block of subdomains (pam_params.sub_begin/sub_end) and
must reproduce the whole fit's coefficients for that block bit for bit (the
subdomains are independent), evaluate its points identically, and its raw
error sums (pam_error_sums) added over the shards must give the whole fit's
error measures."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_shards_reproduce_the_whole_fit(env, precision):
    import bench
    torch, pam, dev = env
    n_cells, n_sub, ov, g = (128, 128), (4, 4), 2, (6, 6)
    K = fields.voronoi_field(128, n_sites=16, seed=61)
    params = dict(k_top=8, levels=2, precision=precision)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    whole = pam.Fitter(n_cells, n_sub, ov, g, device=dev, **params)
    whole.fit(Kd)
    ref = whole.host_model()
    e_ref = whole.errors(Kd)
    W = dict(shape=n_cells, n_sub=n_sub, overlap=ov, g=g, params=dict(k_top=8, levels=2))
    ranges = bench.shard_ranges(bench.shard_costs(W), 3)
    assert ranges[0][0] == 0 and ranges[-1][1] == 16
    pts = np.random.default_rng(62).uniform(0, 1, size=(20000, 2))
    own = bench.owner_index(dict(W, shape=n_cells), pts)
    k_ref = whole.eval(torch.from_numpy(pts).to(dev)).cpu().numpy()
    total = np.zeros(8)
    for b, e in ranges:
        sh = pam.Fitter(n_cells, n_sub, ov, g, device=dev, sub_range=(b, e), **params)
        sh.fit(Kd)
        got = sh.host_model()
        for key in ("M", "c", "beta"):
            np.testing.assert_array_equal(got[key][b:e], ref[key][b:e])
        np.testing.assert_array_equal(got["info"][b:e], ref["info"][b:e])
        outside = np.r_[0:b, e:16]
        assert np.all(got["info"][outside, pam.INFO_STOPPED] == 1)
        assert np.all(got["beta"][outside] == 0) and np.all(got["M"][outside] == 36)
        q = (own >= b) & (own < e)
        np.testing.assert_array_equal(sh.eval(torch.from_numpy(np.ascontiguousarray(pts[q])).to(dev)).cpu().numpy(),
                                      k_ref[q])
        sums = torch.zeros(8, dtype=torch.float64, device=dev)
        pam.pam_error_sums(sh.problem, sh.plan, sh.model, Kd, sums, (b, e), sh.workspace, precision)
        s = sums.cpu().numpy()
        total[:6] += s[:6]
        total[6] = max(total[6], s[6])
    e_sh = pam.error_measures_from_sums(total)
    for key in ("l1", "l2", "l1_log", "max_log10"):
        assert e_sh[key] == pytest.approx(e_ref[key], rel=1e-12)
