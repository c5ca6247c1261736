"""Pins of the FP64 network oracle (oracle/nn.py): its forward pass against
PyTorch's CPU convolution and linear routines, its loss against PyTorch's
BCE-with-logits and MSE, and its hand-written backward pass against central
finite differences."""
import numpy as np
import pytest

from oracle import nn

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _torch_forward(p, x):
    lay, _ = nn.layout()
    B = x.shape[0]
    a = torch.from_numpy(x.reshape(B, 1, 32, 32))
    for l, (hin, cin, hout, cout, stride, kpad) in enumerate(nn.CONV):
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


def _data(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(B, 32, 32))
    support = (rng.uniform(size=(B, 256)) < 0.3).astype(np.float64)
    beta = rng.standard_normal((B, 256)) * 3 * support
    return x, support, beta


def test_forward_matches_torch_convolutions():
    p = nn.init_params(1)
    p[np.arange(p.size) % 7 == 0] += 0.01  # nonzero biases too
    x, _, _ = _data(3, 2)
    out, _ = nn.forward(p, x)
    np.testing.assert_allclose(out, _torch_forward(p, x), rtol=1e-10, atol=1e-12)


def test_loss_matches_torch():
    p = nn.init_params(3)
    x, s, b = _data(4, 4)
    out, _ = nn.forward(p, x)
    loss, _ = nn.loss_and_grad_out(out, s, b)
    o = torch.from_numpy(out)
    bce = F.binary_cross_entropy_with_logits(o[:, :256], torch.from_numpy(s)).item()
    mse = F.mse_loss(o[:, 256:], torch.from_numpy(b / nn.BETA_SCALE)).item()
    assert loss[0] == pytest.approx(bce, rel=1e-12)
    assert loss[1] == pytest.approx(mse, rel=1e-12)


def test_backward_matches_finite_differences():
    p = nn.init_params(5)
    x, s, b = _data(2, 6)
    loss, g = nn.gradients(p, x, s, b)
    lay, total = nn.layout()
    rng = np.random.default_rng(7)
    idx = []
    for wo, bo, rows, cols in lay:
        idx += list(rng.integers(wo, wo + rows * cols, size=6)) + list(rng.integers(bo, bo + rows, size=2))
    f = lambda q: sum(nn.loss_and_grad_out(nn.forward(q, x)[0], s, b)[0])
    eps = 1e-6
    for i in idx:
        e = np.zeros(total); e[i] = eps
        fd = (f(p + e) - f(p - e)) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10), i
