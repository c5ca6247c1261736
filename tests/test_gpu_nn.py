"""The learned warm start's network on the GPU (bf16 tensor-core passes with
fp32 accumulation) against the FP64 network oracle: forward outputs, the
loss, and every parameter gradient of the hand-written backward pass."""
import numpy as np
import pytest

from oracle import nn as onn

pytestmark = pytest.mark.gpu

OUT_RTOL = 3e-2      # ||out_gpu - out_ref|| / ||out_ref||: bf16 activations through 6 layers
GRAD_RTOL = 0.12     # per layer tensor, relative 2-norm (bf16 dz at every layer; the first
                     # layer's weight gradient sums ~1e4-1e5 cancelling bf16 products)
GRAD_COS = 0.99      # per layer tensor, cosine similarity (a transposed operand gives ~0)
LOSS_RTOL = 2e-2


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam
    return torch, pam, torch.device("cuda:0")


def _data(B, seed, arch=0):
    A = onn.ARCHS[arch]
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(B, A["h0"], A["h0"], A["c0"]))
    support = (rng.uniform(size=(B, A["n_out"])) < 0.3).astype(np.float64)
    beta = rng.standard_normal((B, A["n_out"])) * 3 * support
    return x, support, beta


@pytest.mark.parametrize("arch", [0, 1])
def test_layout_matches_the_oracle(env, arch):
    torch, pam, dev = env
    lay, total = onn.layout(arch)
    n, _ = pam.pam_nn_sizes(32, arch=arch)
    assert n == total
    off = pam.pam_nn_layer_offsets(arch=arch)
    np.testing.assert_array_equal(off, np.array(lay))
    A = onn.ARCHS[arch]
    assert pam.pam_nn_geometry(arch) == (A["h0"], A["c0"], A["n_out"])


@pytest.mark.parametrize("arch,B", [(0, 32), (0, 96), (1, 64)])
def test_forward_loss_and_gradients(env, arch, B):
    torch, pam, dev = env
    n_out = onn.ARCHS[arch]["n_out"]
    p = onn.init_params(11, arch)
    p[onn.layout(arch)[0][5][1]:] += 0.05  # output biases
    x, s, b = _data(B, 12, arch)
    ref_out, _ = onn.forward(p, x, arch)
    ref_loss, ref_g = onn.gradients(p, x, s, b, arch)
    n, ws_bytes = pam.pam_nn_sizes(B, arch=arch)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    P = torch.from_numpy(p.astype(np.float32)).to(dev)
    X = torch.from_numpy(x.astype(np.float32)).to(dev)
    out = torch.zeros((B, 2 * n_out), dtype=torch.float32, device=dev)
    pam.pam_nn_forward(P, X, out, ws, arch=arch)
    o = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(o - ref_out) <= OUT_RTOL * np.linalg.norm(ref_out)
    g = torch.zeros(n, dtype=torch.float32, device=dev)
    loss = torch.zeros(2, dtype=torch.float32, device=dev)
    pam.pam_nn_gradients(P, X, torch.from_numpy(s.astype(np.float32)).to(dev),
                         torch.from_numpy(b.astype(np.float32)).to(dev), g, loss, ws, arch=arch)
    np.testing.assert_allclose(loss.cpu().numpy(), ref_loss, rtol=LOSS_RTOL)
    gg = g.cpu().numpy().astype(np.float64)
    errs = []
    for l, (wo, bo, rows, cols) in enumerate(onn.layout(arch)[0]):
        for kind, lo, hi in (("W", wo, wo + rows * cols), ("b", bo, bo + rows)):
            a, r = gg[lo:hi], ref_g[lo:hi]
            nr = np.linalg.norm(r)
            if nr == 0:
                assert np.abs(a).max() == 0
                continue
            errs.append((l, kind, np.linalg.norm(a - r) / nr, a @ r / (np.linalg.norm(a) * nr)))
    print("per-layer gradient (rel error, cosine):", [(l, k, round(e, 4), round(c, 5)) for l, k, e, c in errs])
    for l, k, e, c in errs:
        assert e <= GRAD_RTOL and c >= GRAD_COS, (l, k, e, c)


def test_adamw_step(env):
    torch, pam, dev = env
    rng = np.random.default_rng(13)
    n = 1000
    p0 = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    P = torch.from_numpy(p0.copy()).to(dev)
    m = torch.zeros(n, device=dev)
    v = torch.zeros(n, device=dev)
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 0.01
    for t in (1, 2):
        pam.pam_nn_adamw(P, torch.from_numpy(g).to(dev), m, v, lr, b1, b2, eps, wd, t)
    # reference: the same two AdamW steps in float64
    pr, mr, vr = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in (1, 2):
        mr = b1 * mr + (1 - b1) * g
        vr = b2 * vr + (1 - b2) * g.astype(np.float64) ** 2
        pr = pr - lr * ((mr / (1 - b1 ** t)) / (np.sqrt(vr / (1 - b2 ** t)) + eps) + wd * pr)
    np.testing.assert_allclose(P.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
