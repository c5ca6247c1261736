"""Pins of the FP64 network oracle (oracle/nn.py): its forward pass against
PyTorch's CPU convolution and linear routines, its loss against PyTorch's
BCE-with-logits and MSE, and its hand-written backward pass against central
finite differences."""
import numpy as np
import pytest

from oracle import nn

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _torch_forward(p, x, arch):
    A = nn.ARCHS[arch]
    lay, _ = nn.layout(arch)
    B = x.shape[0]
    a = torch.from_numpy(x.reshape(B, A["h0"], A["h0"], A["c0"])).permute(0, 3, 1, 2)  # NCHW
    for l, (hin, cin, hout, cout, stride, kpad) in enumerate(A["conv"]):
        wo, bo, rows, cols = lay[l]
        W = p[wo:wo + rows * cols].reshape(rows, cols)[:, :9 * cin]
        Wt = torch.from_numpy(W.reshape(cout, 3, 3, cin).transpose(0, 3, 1, 2).copy())
        a = F.relu(F.conv2d(a, Wt, torch.from_numpy(p[bo:bo + rows]), stride=stride, padding=1))
    h = a.permute(0, 2, 3, 1).reshape(B, -1)  # NHWC flatten
    wo, bo, rows, cols = lay[4]
    h = F.relu(F.linear(h, torch.from_numpy(p[wo:wo + rows * cols].reshape(rows, cols)),
                        torch.from_numpy(p[bo:bo + rows])))
    wo, bo, rows, cols = lay[5]
    return F.linear(h, torch.from_numpy(p[wo:wo + rows * cols].reshape(rows, cols)),
                    torch.from_numpy(p[bo:bo + rows])).numpy()


def _data(B, seed, arch=0):
    A = nn.ARCHS[arch]
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(B, A["h0"], A["h0"], A["c0"]))
    support = (rng.uniform(size=(B, A["n_out"])) < 0.3).astype(np.float64)
    beta = rng.standard_normal((B, A["n_out"])) * 3 * support
    return x, support, beta


@pytest.mark.parametrize("arch", [0, 1])
def test_forward_matches_torch_convolutions(arch):
    p = nn.init_params(1, arch)
    p[np.arange(p.size) % 7 == 0] += 0.01  # nonzero biases too
    x, _, _ = _data(3, 2, arch)
    out, _ = nn.forward(p, x, arch)
    np.testing.assert_allclose(out, _torch_forward(p, x, arch), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("arch", [0, 1])
def test_loss_matches_torch(arch):
    p = nn.init_params(3, arch)
    x, s, b = _data(4, 4, arch)
    out, _ = nn.forward(p, x, arch)
    loss, _ = nn.loss_and_grad_out(out, s, b)
    n_out = nn.ARCHS[arch]["n_out"]
    o = torch.from_numpy(out)
    bce = F.binary_cross_entropy_with_logits(o[:, :n_out], torch.from_numpy(s)).item()
    mse = F.mse_loss(o[:, n_out:], torch.from_numpy(b / nn.BETA_SCALE)).item()
    assert loss[0] == pytest.approx(bce, rel=1e-12)
    assert loss[1] == pytest.approx(mse, rel=1e-12)


@pytest.mark.parametrize("arch", [0, 1])
def test_backward_matches_finite_differences(arch):
    p = nn.init_params(5, arch)
    x, s, b = _data(2, 6, arch)
    loss, g = nn.gradients(p, x, s, b, arch)
    lay, total = nn.layout(arch)
    rng = np.random.default_rng(7)
    idx = []
    for wo, bo, rows, cols in lay:
        idx += list(rng.integers(wo, wo + rows * cols, size=6)) + list(rng.integers(bo, bo + rows, size=2))
    f = lambda q: sum(nn.loss_and_grad_out(nn.forward(q, x, arch)[0], s, b)[0])
    eps = 1e-6
    for i in idx:
        e = np.zeros(total); e[i] = eps
        fd = (f(p + e) - f(p - e)) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10), i
