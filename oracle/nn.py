"""FP64 CPU oracle of the learned warm-start network -- test infrastructure only.

Same architectures, parameter layouts and loss as the CUDA network (see the
pam_nn_* entry points of the C ABI), written with numpy in float64, forward
and backward by hand (no automatic differentiation). Two architectures:

  arch 0 (patch 2-D): x [B,32,32,1] (log10 K / 3)
    -> conv3x3 s2 pad1 (1->32) -> ReLU -> conv3x3 s2 (32->64) -> ReLU
    -> conv3x3 s2 (64->128) -> ReLU -> conv3x3 s1 (128->128) -> ReLU
    -> flatten (NHWC, 2048) -> dense 256 -> ReLU -> dense 512
    out = [256 support logits | 256 beta / 4]
  arch 1 (layered 3-D): x [B,16,16,8] (z layers as channels)
    -> conv3x3 s2 (8->32) -> ReLU -> conv3x3 s2 (32->64) -> ReLU
    -> conv3x3 s1 (64->64) -> ReLU -> conv3x3 s1 (64->64) -> ReLU
    -> flatten (1024) -> dense 128 -> ReLU -> dense 64
    out = [32 support logits | 32 beta / 4]
  loss = mean BCE-with-logits(logits, support) + mean (out_beta - beta / 4)^2

Parameters are one flat float array; layer l has W [rows][cols] at
offsets[l][0] and b [rows] at offsets[l][1]; a convolution's columns are
(ky*3 + kx)*cin + c, zero-padded up to a multiple of 32.
"""
from __future__ import annotations

import numpy as np

ARCHS = {
    0: dict(h0=32, c0=1,
            conv=[(32, 1, 16, 32, 2, 32), (16, 32, 8, 64, 2, 288), (8, 64, 4, 128, 2, 576),
                  (4, 128, 4, 128, 1, 1152)],  # hin, cin, hout, cout, stride, kpad
            dense=[(2048, 256), (256, 512)], n_out=256),
    1: dict(h0=16, c0=8,
            conv=[(16, 8, 8, 32, 2, 96), (8, 32, 4, 64, 2, 288), (4, 64, 4, 64, 1, 576),
                  (4, 64, 4, 64, 1, 576)],
            dense=[(1024, 128), (128, 64)], n_out=32),
}
CONV = ARCHS[0]["conv"]
DENSE = ARCHS[0]["dense"]
N_OUT = ARCHS[0]["n_out"]
BETA_SCALE = 4.0


def layout(arch=0):
    """Per layer (w_offset, b_offset, rows, cols) and the total size."""
    A = ARCHS[arch]
    out, off = [], 0
    for l in range(6):
        rows = A["conv"][l][3] if l < 4 else A["dense"][l - 4][1]
        cols = A["conv"][l][5] if l < 4 else A["dense"][l - 4][0]
        out.append((off, off + rows * cols, rows, cols))
        off += rows * cols + rows
    return out, off


def init_params(seed=0, arch=0):
    """He-normal weights (padding columns zero), zero biases."""
    A = ARCHS[arch]
    rng = np.random.default_rng(seed)
    lay, total = layout(arch)
    p = np.zeros(total)
    for l, (wo, bo, rows, cols) in enumerate(lay):
        fan_in = 9 * A["conv"][l][1] if l < 4 else cols
        used = fan_in if l < 4 else cols
        w = np.zeros((rows, cols))
        w[:, :used] = rng.standard_normal((rows, used)) * np.sqrt(2.0 / fan_in)
        if l == 5:
            w *= 0.1
        p[wo:wo + rows * cols] = w.reshape(-1)
    return p


def _im2col(x, stride, kpad):
    """x [B,h,h,c] -> cols [B*ho*ho, kpad], column (ky*3+kx)*c + ch."""
    B, h, _, c = x.shape
    ho = (h + 2 - 3) // stride + 1
    xp = np.zeros((B, h + 2, h + 2, c))
    xp[:, 1:h + 1, 1:h + 1, :] = x
    cols = np.zeros((B, ho, ho, kpad))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + stride * (ho - 1) + 1:stride, kx:kx + stride * (ho - 1) + 1:stride, :]
            t = ky * 3 + kx
            cols[..., t * c:(t + 1) * c] = patch
    return cols.reshape(B * ho * ho, kpad), ho


def _col2im(dcols, B, h, c, stride, kpad):
    ho = (h + 2 - 3) // stride + 1
    dc = dcols.reshape(B, ho, ho, kpad)
    dxp = np.zeros((B, h + 2, h + 2, c))
    for ky in range(3):
        for kx in range(3):
            t = ky * 3 + kx
            dxp[:, ky:ky + stride * (ho - 1) + 1:stride, kx:kx + stride * (ho - 1) + 1:stride, :] += \
                dc[..., t * c:(t + 1) * c]
    return dxp[:, 1:h + 1, 1:h + 1, :]


def _wb(p, l, arch=0):
    lay, _ = layout(arch)
    wo, bo, rows, cols = lay[l]
    return p[wo:wo + rows * cols].reshape(rows, cols), p[bo:bo + rows]


def forward(p, x, arch=0):
    """x [B,h0,h0,c0] (or [B,32,32] for arch 0) -> (out [B,2 n_out], cache)."""
    A = ARCHS[arch]
    B = x.shape[0]
    a = x.reshape(B, A["h0"], A["h0"], A["c0"]).astype(np.float64)
    cache = []
    for l, (hin, cin, hout, cout, stride, kpad) in enumerate(A["conv"]):
        cols, ho = _im2col(a, stride, kpad)
        W, b = _wb(p, l, arch)
        z = cols @ W.T + b
        y = np.maximum(z, 0.0)
        cache.append((cols, z))
        a = y.reshape(B, ho, ho, cout)
    h = a.reshape(B, -1)
    W4, b4 = _wb(p, 4, arch)
    z4 = h @ W4.T + b4
    y4 = np.maximum(z4, 0.0)
    W5, b5 = _wb(p, 5, arch)
    out = y4 @ W5.T + b5
    cache.append((h, z4))
    cache.append((y4, out))
    return out, cache


def loss_and_grad_out(out, support, beta):
    """(loss [bce, mse], dL/dout); n_out = out.shape[1] / 2."""
    n_out = out.shape[1] // 2
    n = support.size
    z = out[:, :n_out]
    bce = np.logaddexp(0.0, z) - support * z
    d = out[:, n_out:] - beta / BETA_SCALE
    dout = np.zeros_like(out)
    dout[:, :n_out] = (1.0 / (1.0 + np.exp(-z)) - support) / n
    dout[:, n_out:] = 2.0 * d / n
    return np.array([bce.sum() / n, (d * d).sum() / n]), dout


def gradients(p, x, support, beta, arch=0):
    """(loss [2], grads like p): forward, loss, and the backward pass by hand."""
    A = ARCHS[arch]
    B = x.shape[0]
    lay, total = layout(arch)
    g = np.zeros(total)
    out, cache = forward(p, x, arch)
    loss, dout = loss_and_grad_out(out, support, beta)
    y4, _ = cache[5]
    h, z4 = cache[4]
    W5, _ = _wb(p, 5, arch)
    wo, bo, rows, cols = lay[5]
    g[wo:wo + rows * cols] = (dout.T @ y4).reshape(-1)
    g[bo:bo + rows] = dout.sum(0)
    dy4 = dout @ W5
    dz4 = dy4 * (z4 > 0)
    W4, _ = _wb(p, 4, arch)
    wo, bo, rows, cols = lay[4]
    g[wo:wo + rows * cols] = (dz4.T @ h).reshape(-1)
    g[bo:bo + rows] = dz4.sum(0)
    dh = dz4 @ W4
    last = A["conv"][3]
    da = dh.reshape(B, last[2], last[2], last[3])
    for l in range(3, -1, -1):
        hin, cin, hout, cout, stride, kpad = A["conv"][l]
        cols_l, z = cache[l]
        dz = da.reshape(-1, cout) * (z > 0)
        W, _ = _wb(p, l, arch)
        wo, bo, rows, cols = lay[l]
        g[wo:wo + rows * cols] = (dz.T @ cols_l).reshape(-1)
        g[bo:bo + rows] = dz.sum(0)
        if l > 0:
            da = _col2im(dz @ W, B, hin, cin, stride, kpad)
    return loss, g
