"""The learned warm start end to end on the GPU, at the sizes of the 2-D
patch workload: about 50k seeded 32 x 32 patches (224^2 = 50,176) labelled
by the plain fit, the network trained on them with the project's kernels,
and its inference batched over 4,096 held-out patches in one forward pass.
What it gains: fewer active-set iterations for the same certified minimiser
(the plain regression stays the fallback and has the last word). Parity: on an
evenly spaced sample of the held-out patches the oracle fits each patch,
and the learned form matches it -- binary64: coefficients within 1e-9 and
the same supports; fp32 form: the patch's L1 error within 1 % of the
oracle's and no cell's log10 K* off by more than 1e-3 (relative)."""
import numpy as np
import pytest

import oracle
from oracle_refit import oracle_on_gpu_dictionary
from paper_2605_16564_gb300 import fields

pytestmark = pytest.mark.gpu

N_TRAIN = 224 * 224    # 50,176 training patches
LABEL_BATCH = 56 * 56  # labelled in 16 launches of 3,136 patches
N_HELD = 64 * 64       # 4,096 held-out patches
N_ORACLE = 96          # held-out patches the oracle fits
BETA_RTOL = 1e-9
LOG10_RTOL = 1e-3
L1_RTOL = 0.01


@pytest.fixture(scope="module")
def trained():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam, warmstart as ws
    dev = torch.device("cuda:0")
    train = fields.patch_batch(N_TRAIN, seed=4)
    beta, support = ws.label(train, dev, batch=LABEL_BATCH)
    net = ws.Network(dev, batch=256, seed=0)
    hist = net.train(ws.network_input(train), support, beta, epochs=8, lr=2e-3)
    del train, beta, support
    held = fields.patch_batch(N_HELD, seed=40)
    grid, T = ws.tile(held)
    which = np.linspace(0, N_HELD - 1, N_ORACLE).round().astype(int)
    ref = oracle.fit_all(grid, (T * ws.PATCH, T * ws.PATCH), (T, T), 0, (ws.G, ws.G),
                         oracle.default_params(k_top=1, levels=0), which=which)
    assert ref["failed"] == 0
    return dict(torch=torch, pam=pam, ws=ws, dev=dev, net=net, hist=hist, held=held, grid=grid, T=T,
                which=which, ref=ref)


def test_training_reduces_the_held_out_loss(trained):
    torch, pam, ws, dev, net, hist, held = (trained[k] for k in ("torch", "pam", "ws", "dev", "net", "hist",
                                                                 "held"))
    assert all(b[0] <= a[0] * 1.02 for a, b in zip(hist, hist[1:])), hist
    assert hist[-1][0] < hist[0][0] and hist[-1][1] < hist[0][1], hist
    hb, hs = ws.label(held, dev, batch=N_HELD)
    x = ws.network_input(held)
    untrained = ws.Network(dev, batch=256, seed=0)
    l0, l1 = untrained.mean_loss(x, hs, hb), net.mean_loss(x, hs, hb)
    print(f"held-out loss: bce {l0[0]:.4f} -> {l1[0]:.4f}, mse {l0[1]:.4f} -> {l1[1]:.4f}")
    assert l1[0] < 0.95 * l0[0] and l1[1] < 0.85 * l0[1], (l0, l1)


def _sample_cells(T, which):
    """Flat indices (x fastest) of the cells of patches `which` of a T x T
    tiling, patch by patch."""
    n = 32 * T
    r, c = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    return np.stack([((p // T) * 32 + r) * n + (p % T) * 32 + c for p in which]).reshape(len(which), -1)


def test_device_inputs_and_seed_match_the_host_forms(trained):
    # pam_nn_inputs(arch 0) gathers network_input's patches from the tiled
    # field on the device (log10 in fp32 there: a rounding apart), and
    # pam_nn_seed(arch 0) writes warm_start_coefficients of the same output
    torch, pam, ws, dev, net, held = (trained[k] for k in ("torch", "pam", "ws", "dev", "net", "held"))
    fit = ws.PatchFit(32 * 32, dev)
    sub = held[:32 * 32]
    Kd = fit.device_field(sub)
    X = torch.full((1024, 32, 32, 1), 7.0, dtype=torch.float32, device=dev)
    pam.pam_nn_inputs(fit.fitter.problem, fit.fitter.plan, Kd, X)
    x = X.cpu().numpy()[..., 0]
    np.testing.assert_allclose(x, ws.network_input(sub), rtol=0, atol=5e-7)
    out = net.forward_device(X)
    f = fit.fitter
    f.model.beta.fill_(5.0)
    pam.pam_nn_seed(f.plan, out, ws.SEED_THRESHOLD, f.model, arch=pam.PAM_NN_PATCH2D)
    o = out.cpu().numpy()
    want = ws.warm_start_coefficients(o[:, :ws.N_OUT], o[:, ws.N_OUT:] * ws.BETA_SCALE)
    got = f.model.beta[:, :ws.N_OUT].cpu().numpy()
    np.testing.assert_array_equal(got, want)
    # fewer rows than subdomains: refused, nothing written
    Xs = torch.full((992, 32, 32, 1), 7.0, dtype=torch.float32, device=dev)
    with pytest.raises(pam.PamError):
        pam.pam_nn_inputs(f.problem, f.plan, Kd, Xs)
    torch.cuda.synchronize()
    assert torch.all(Xs == 7.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_warm_start_reaches_the_plain_minimiser_in_fewer_iterations(trained, precision):
    torch, pam, ws, dev, net, held = (trained[k] for k in ("torch", "pam", "ws", "dev", "net", "held"))
    T, which, ref, grid = trained["T"], trained["which"], trained["ref"], trained["grid"]
    cold = ws.PatchFit(N_HELD, dev, precision, max_iters=400)
    b_cold, info_cold, ms_cold = cold.fit(held)
    res = ws.learned_fit(net, held, dev, precision)
    it = lambda info: (info[:, pam.INFO_ITERS] % 100).astype(float)
    assert np.all((info_cold[:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED) == 0)
    assert np.all((res["info"][:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED) == 0)
    if precision == 0:
        # the same certified minimiser (unique), to solve precision, on all
        # 4,096 patches; and the oracle's on the sample, supports included
        scale = np.maximum(1.0, np.abs(b_cold).max(axis=1, keepdims=True))
        assert np.all(np.abs(res["beta"] - b_cold) <= BETA_RTOL * scale)
        for s in which:
            rb, gb = ref["beta"][s, :ws.N_OUT], res["beta"][s]
            assert np.abs(gb - rb).max() <= BETA_RTOL * max(1.0, np.abs(rb).max()), s
            if ref["info"][s, 4] > 1e-9:
                np.testing.assert_array_equal(gb != 0, rb != 0)
    # the learned form's surrogate (evaluated by the GPU in its own
    # precision, on the cold fit's dictionary) against the oracle's, cell by
    # cell on the sampled patches
    xs = fields.cell_centred_points((T * ws.PATCH, T * ws.PATCH), (1.0, 1.0))
    idx = _sample_cells(T, which)
    pts = xs[idx.reshape(-1)]
    f = cold.fitter
    f.model.beta[:, :ws.N_OUT] = torch.from_numpy(res["beta"]).to(dev)
    k_learned = f.eval(torch.from_numpy(pts).to(dev)).cpu().numpy().reshape(idx.shape)
    k_oracle = oracle.evaluate(ref, pts).reshape(idx.shape)
    K = grid.reshape(-1)[idx]
    l1_learned = np.abs(k_learned - K).sum(axis=1) / K.sum(axis=1)
    l1_oracle = np.abs(k_oracle - K).sum(axis=1) / K.sum(axis=1)
    assert np.all(np.abs(l1_learned - l1_oracle) <= L1_RTOL * l1_oracle), np.abs(l1_learned / l1_oracle - 1).max()
    lo = np.log10(k_oracle)
    d = np.abs(np.log10(k_learned) - lo) / np.maximum(1.0, np.abs(lo))
    assert d.max() <= LOG10_RTOL, d.max()
    mean_cold, mean_warm = it(info_cold).mean(), it(res["info"]).mean()
    print(f"precision {precision}: {N_HELD} held-out patches, active-set iterations cold {mean_cold:.2f} -> "
          f"learned {mean_warm:.2f} (max {it(info_cold).max():.0f} -> {it(res['info']).max():.0f}), "
          f"solve {ms_cold:.2f} ms -> {res['solve_ms']:.2f} ms, batched inference {res['predict_ms']:.2f} ms, "
          f"plain refits {res['refit']}; sampled L1 vs oracle max rel diff "
          f"{np.abs(l1_learned / l1_oracle - 1).max():.2e}, log10 {d.max():.2e}")
    assert mean_warm <= 0.85 * mean_cold
    assert it(res["info"]).max() < it(info_cold).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_layered_3d_learned_seed(precision):
    # The 3-D network (PAM_NN_LAYERED3D) trained on the level-0 fits of 8
    # seeded layered fields seeds the level-0 active set of a new field:
    # fewer steps on average, every subdomain certified, and the same
    # minimiser (fp64: coefficients within 1e-9; fp32 form: the surrogate
    # per cell within its log10 tolerance).
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam, warmstart as ws
    dev = torch.device("cuda:0")
    shape, n_sub = (30, 110, 85), (3, 11, 17)
    fit = pam.Fitter(shape, n_sub, 1, (4, 4, 2), device=dev, precision=precision, k_top=30, levels=3)
    lw = ws.LayeredWarmStart(dev, batch=256, seed=0)
    train = [torch.from_numpy(fields.layered_field(shape, seed=200 + i)).to(dev) for i in range(8)]
    hist = lw.train(fit, train, epochs=8)
    assert hist[-1][1] < 0.7 * hist[0][1], hist
    Kd = torch.from_numpy(fields.layered_field(shape, seed=5)).to(dev)
    it = lambda: fit.model.info.cpu().numpy()[:, pam.INFO_ITERS] % 100
    flags = lambda: fit.model.info.cpu().numpy()[:, pam.INFO_FLAGS]
    assert fit.fit(Kd, levels=0, check=False) == 0
    it_cold, beta_cold = it(), fit.model.beta.cpu().numpy().copy()
    pts = fields.cell_centred_points(shape, [n / max(shape) for n in shape])
    X = torch.from_numpy(pts).to(dev)
    k_cold = fit.eval(X).cpu().numpy()
    lw.seed(fit, Kd)
    assert fit.fit(Kd, levels=0, check=False, warm_start=True) == 0
    it_warm = it()
    assert np.all((flags() & pam.FLAG_NOT_CERTIFIED) == 0)
    # the same seeded fit with the inference on a side stream, joined by an
    # event before the level-0 solve (pam_params.warm_start_event): the same
    # bits, although model.beta holds NaN when the fit is enqueued
    b_seq, i_seq = fit.model.beta.cpu().numpy().copy(), fit.model.info.cpu().numpy().copy()
    fit.model.beta.fill_(float("nan"))
    side, ev = torch.cuda.Stream(device=dev), torch.cuda.Event()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        torch.cuda._sleep(20_000_000)  # the seed lands well after the fit is enqueued
        lw.seed(fit, Kd)
        ev.record(side)
    assert fit.fit(Kd, levels=0, check=False, warm_start=True, warm_start_event=ev) == 0
    np.testing.assert_array_equal(fit.model.beta.cpu().numpy(), b_seq)
    np.testing.assert_array_equal(fit.model.info.cpu().numpy(), i_seq)
    print(f"precision {precision}: level-0 active-set steps cold {it_cold.mean():.2f} -> learned "
          f"{it_warm.mean():.2f} (max {it_cold.max()} -> {it_warm.max()})")
    assert it_warm.mean() <= 0.8 * it_cold.mean()
    if precision == 0:
        b = fit.model.beta.cpu().numpy()
        scale = np.maximum(1.0, np.abs(beta_cold).max(axis=1, keepdims=True))
        assert np.all(np.abs(b - beta_cold) <= 1e-9 * scale)
    else:
        k_warm = fit.eval(X).cpu().numpy()
        d = np.abs(np.log10(k_warm) - np.log10(k_cold)) / np.maximum(1.0, np.abs(np.log10(k_cold)))
        assert d.max() <= 1e-3, d.max()


def test_layered_3d_benchmark_configuration_matches_the_oracle():
    # The 60 x 220 x 85 layered workload as the benchmark times it: mixed
    # form, the 3-D network's seed written on a side stream and joined
    # before the level-0 solve, the fit over 3 levels + evaluation + errors
    # captured in one CUDA graph and replayed. Against the oracle on 24
    # evenly spaced subdomains: L1 within 1 %, and log10 K* per cell within
    # 1e-3 (relative) where the refinement made the oracle's decisions (at
    # least 75 % of the sampled subdomains); every subdomain certified.
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam, warmstart as ws
    dev = torch.device("cuda:0")
    shape, n_sub, params = (60, 220, 85), (6, 22, 17), dict(k_top=30, levels=3)
    fit = pam.Fitter(shape, n_sub, 1, (4, 4, 2), device=dev, precision=pam.PAM_PREC_MIXED, **params)
    lw = ws.LayeredWarmStart(dev, batch=256, seed=0)
    lw.train(fit, [torch.from_numpy(fields.layered_field(shape, seed=5100 + i)).to(dev) for i in range(8)])
    K = fields.layered_field(shape, seed=5)
    Kd = torch.from_numpy(K).to(dev)
    which = list(range(0, 2244, 97))
    boxes = oracle.partition(shape, n_sub, 1)
    h = 1.0 / 220
    pts, kt, sl = [], [], []
    for s in which:
        b = boxes[s]
        ax = [(np.arange(b[a], b[3 + a]) + 0.5) * h for a in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        sl.append(slice(sum(len(p) for p in pts), sum(len(p) for p in pts) + X.size))
        pts.append(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1))
        kt.append(K[b[2]:b[5], b[1]:b[4], b[0]:b[3]].ravel())
    pts, kt = np.concatenate(pts), np.concatenate(kt)
    ptsd = torch.from_numpy(pts).to(dev)
    out = torch.empty(len(pts), dtype=torch.float64, device=dev)
    err = torch.zeros(4, dtype=torch.float64, device=dev)
    side, ev = torch.cuda.Stream(device=dev), torch.cuda.Event()

    def step():
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            lw.seed(fit, Kd)
            ev.record(side)
        fit.fit(Kd, warm_start=True, deferred=True, warm_start_event=ev)
        fit.eval(ptsd, out=out)
        fit.errors_device(Kd, err)

    s0 = torch.cuda.Stream(device=dev)
    s0.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s0):
        step()  # eager, on a side stream, before capture
    torch.cuda.current_stream().wait_stream(s0)
    torch.cuda.synchronize()
    assert fit.status() == 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    fit.model.beta.zero_()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert fit.status() == 0
    got = fit.host_model()
    assert np.count_nonzero(got["info"][:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED) == 0
    km = out.cpu().numpy()
    ref = oracle.fit_all(K, shape, n_sub, 1, (4, 4, 2), oracle.default_params(**params), which=which)
    ko = oracle.evaluate(ref, pts)
    same = 0
    for s, q in zip(which, sl):
        m = ref["M"][s]
        if got["M"][s] == m and np.array_equal(got["c"][s, :m], ref["c"][s, :m]):
            same += 1
            lo = np.log10(ko[q])
        else:  # the oracle's fit of the GPU's own refined dictionary of s
            lo = np.log10(oracle_on_gpu_dictionary(shape, ref, got, s, K, pts[q]))
        d = np.abs(np.log10(km[q]) - lo) / np.maximum(1.0, np.abs(lo))
        assert d.max() <= 1e-3, (s, d.max())
    assert same >= 0.75 * len(which), same
    l1m, l1o = np.abs(kt - km).sum(), np.abs(kt - ko).sum()
    assert abs(l1m - l1o) <= 0.01 * l1o, (l1m, l1o)
    # the replayed step's error reduction is that of the model it left
    e = fit.errors(Kd)
    np.testing.assert_allclose(err.cpu().numpy(), [e["l1"], e["l2"], e["l1_log"], e["max_log10"]], rtol=0,
                               atol=0)
    del g
