"""Learned warm start of the per-patch Elastic Net solve.

A batch of 32 x 32 patches (each its own subdomain, 16 x 16 dictionary with
width = 2 cells, no refinement) is tiled into one grid and fitted in one
call of the C ABI. The plain fit labels the training patches with their
selected support and coefficients; the network (pam_nn_* kernels, bf16
tensor cores) learns to predict both from log10 K; on new patches its
prediction seeds the active-set solve (pam_params.warm_start). A patch whose
warm-started solve is not certified within the learned iteration budget is
refitted plainly from zero. Every numerical step runs in libpam; this module
only moves arrays and drives the loop.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import pam

PATCH = 32
G = 16
N_OUT = G * G
BETA_SCALE = 4.0


def tile(patches):
    """(P, 32, 32) patches -> (grid K of shape (T*32, T*32), T) with patch
    p = px + T*py at block (py, px); P must be a square T*T."""
    P = patches.shape[0]
    T = int(round(np.sqrt(P)))
    assert T * T == P, "the number of patches must be a square"
    grid = patches.reshape(T, T, PATCH, PATCH).transpose(0, 2, 1, 3).reshape(T * PATCH, T * PATCH)
    return np.ascontiguousarray(grid), T


def network_input(patches):
    """log10 K / 3 clipped to [-1, 1], float32 (P, 32, 32)."""
    return np.clip(np.log10(patches) / 3.0, -1.0, 1.0).astype(np.float32)


class PatchFit:
    """Fit of a square batch of patches through the C ABI (one subdomain each)."""

    def __init__(self, n_patches, device, precision=pam.PAM_PREC_FP64, max_iters=0):
        T = int(round(np.sqrt(n_patches)))
        assert T * T == n_patches
        self.T = T
        self.device = device
        self.precision = precision
        self.max_iters = max_iters
        self.fitter = pam.Fitter((T * PATCH, T * PATCH), (T, T), 0, (G, G), device=device, precision=precision,
                                 k_top=1, levels=0, max_iters=max_iters)

    def device_field(self, patches):
        """The tiled field of the patches on the device."""
        import torch
        grid, _ = tile(patches)
        return torch.from_numpy(grid).to(self.device)

    def fit(self, patches, beta0=None, Kd=None, seeded=False):
        """Solve every patch; beta0 [P, 256] (numpy or tensor) seeds the solve,
        or seeded=True: the model's coefficients were seeded on the device
        (pam_nn_seed). Kd: the tiled field already on the device.
        Returns (beta [P,256] numpy, info [P,8] numpy, solve ms)."""
        if Kd is None:
            Kd = self.device_field(patches)
        f = self.fitter
        warm = seeded or beta0 is not None
        p = pam.make_params(k_top=1, levels=0, max_iters=self.max_iters, precision=self.precision,
                            warm_start=1 if warm else 0)
        if beta0 is not None and not seeded:
            import torch
            b0 = torch.as_tensor(beta0, dtype=torch.float64).to(self.device)
            f.model.beta.zero_()
            f.model.beta[:, :N_OUT] = b0
        L = pam.lib()
        L.pam_timing_reset()
        L.pam_timing_enable(1)
        code = pam.pam_fit_subdomains(f.problem, p, f.plan, Kd, f.model, f.workspace, check=False)
        L.pam_timing_enable(0)
        tot, cnt = C.c_double(0), C.c_int(0)
        L.pam_timing_read(3, C.byref(tot), C.byref(cnt))  # PAM_PHASE_SOLVE
        L.pam_timing_reset()
        if code not in (0, 5):
            raise pam.PamError(code, "pam_fit_subdomains")
        beta = f.model.beta[:, :N_OUT].cpu().numpy().copy()
        info = f.model.info.cpu().numpy().copy()
        return beta, info, tot.value


def label(patches, device, batch=4096, precision=pam.PAM_PREC_FP64, max_iters=400):
    """Plain fit of every patch (batches of `batch`): beta [P,256] and support.
    A few patches need a few hundred safeguarded active-set steps, hence
    the larger iteration budget."""
    P = patches.shape[0]
    assert P % batch == 0
    fit = PatchFit(batch, device, precision, max_iters=max_iters)
    betas = []
    for i in range(0, P, batch):
        b, info, _ = fit.fit(patches[i:i + batch])
        if np.any(info[:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED):
            raise RuntimeError("a label fit was not certified")
        betas.append(b)
    beta = np.concatenate(betas)
    return beta, (beta != 0).astype(np.float32)


# input channels of the four convolutions, per architecture
_CIN = {0: [1, 32, 64, 128], 1: [8, 32, 64, 64]}


def init_params(n, offsets, seed=0, arch=0):
    """He-normal weights on the used columns, zero biases and padding."""
    rng = np.random.default_rng(seed)
    p = np.zeros(n, dtype=np.float32)
    cin = _CIN[arch]
    for l in range(6):
        wo, bo, rows, cols = (int(v) for v in offsets[l])
        used = 9 * cin[l] if l < 4 else cols
        w = np.zeros((rows, cols), dtype=np.float32)
        w[:, :used] = rng.standard_normal((rows, used)) * np.sqrt(2.0 / used)
        if l == 5:
            w *= 0.1
        p[wo:wo + rows * cols] = w.reshape(-1)
    return p


class Network:
    """The warm-start network: fp32 master weights on the device, AdamW state."""

    def __init__(self, device, batch=256, seed=0, arch=0):
        import torch
        self.device = device
        self.batch = batch
        self.arch = arch
        n, ws = pam.pam_nn_sizes(batch, arch=arch)
        self.n = n
        self.h0, self.c0, self.n_out = pam.pam_nn_geometry(arch)
        self.offsets = pam.pam_nn_layer_offsets(arch=arch)
        self.params = torch.from_numpy(init_params(n, self.offsets, seed, arch)).to(device)
        self.m = torch.zeros(n, device=device)
        self.v = torch.zeros(n, device=device)
        self.grads = torch.zeros(n, device=device)
        self.loss = torch.zeros(2, device=device)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=device)
        self.step = 0

    def _dev(self, a):
        import torch
        return torch.as_tensor(a, dtype=torch.float32).to(self.device).contiguous()

    def train(self, x, support, beta, epochs=8, lr=2e-3, weight_decay=1e-4, seed=0, log=None):
        """AdamW on (x [P,h,h,c] f32, support, beta [P,n_out]) with a cosine
        learning-rate schedule; returns the per-epoch mean losses. Inputs may
        be numpy arrays or device tensors."""
        import torch
        P = x.shape[0]
        X = self._dev(x).reshape(P, self.h0, self.h0, self.c0)
        Sp, Bt = self._dev(support), self._dev(beta)
        rng = np.random.default_rng(seed)
        steps_per_epoch = P // self.batch
        total = epochs * steps_per_epoch
        history = []
        for ep in range(epochs):
            perm = torch.from_numpy(rng.permutation(P)).to(self.device)
            acc = torch.zeros(2, device=self.device)
            for i in range(steps_per_epoch):
                idx = perm[i * self.batch:(i + 1) * self.batch]
                xb, sb, bb = X[idx].contiguous(), Sp[idx].contiguous(), Bt[idx].contiguous()
                pam.pam_nn_gradients(self.params, xb, sb, bb, self.grads, self.loss, self.ws, arch=self.arch)
                self.step += 1
                frac = (ep * steps_per_epoch + i) / max(total - 1, 1)
                lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * frac))
                pam.pam_nn_adamw(self.params, self.grads, self.m, self.v, lr_t, 0.9, 0.999, 1e-8,
                                 weight_decay, self.step)
                acc += self.loss
            history.append((acc / steps_per_epoch).cpu().numpy().tolist())
            if log:
                log(f"epoch {ep}: bce {history[-1][0]:.4f} mse {history[-1][1]:.4f}")
        return history

    def mean_loss(self, x, support, beta):
        """Mean (BCE, MSE) of the current weights over (x, support, beta),
        in passes of the training batch size (a ragged tail is dropped);
        the weights are not changed."""
        import torch
        P = x.shape[0] // self.batch * self.batch
        X = self._dev(x[:P]).reshape(P, self.h0, self.h0, self.c0)
        Sp, Bt = self._dev(support[:P]), self._dev(beta[:P])
        grads = torch.zeros(self.n, device=self.device)
        acc = torch.zeros(2, device=self.device)
        for i in range(0, P, self.batch):
            sl = slice(i, i + self.batch)
            pam.pam_nn_gradients(self.params, X[sl].contiguous(), Sp[sl].contiguous(), Bt[sl].contiguous(),
                                 grads, self.loss, self.ws, arch=self.arch)
            acc += self.loss
        return (acc / (P // self.batch)).cpu().numpy().tolist()

    def forward_device(self, X, out=None, ws=None):
        """Device forward of X [rows,h,h,c] (rows a multiple of 32) into out
        [rows, 2 n_out]; one call, with a workspace sized for the rows."""
        import torch
        rows = X.shape[0]
        if out is None:
            out = torch.empty((rows, 2 * self.n_out), dtype=torch.float32, device=self.device)
        if ws is None:
            ws = torch.empty(pam.pam_nn_sizes(rows, arch=self.arch)[1], dtype=torch.uint8, device=self.device)
        pam.pam_nn_forward(self.params, X, out, ws, arch=self.arch)
        return out

    def predict(self, x, batched=False):
        """x [P,h,h,c] -> (support logits [P,n_out], beta [P,n_out]) numpy.
        batched: one forward pass over all P rows (padded to a multiple of
        32) instead of passes of the training batch size."""
        import torch
        P = x.shape[0]
        X = self._dev(x).reshape(P, self.h0, self.h0, self.c0)
        if batched:
            rows = -(-P // 32) * 32
            if rows > P:
                X = torch.cat([X, torch.zeros((rows - P, self.h0, self.h0, self.c0), device=self.device)])
            o = self.forward_device(X.contiguous())[:P].cpu().numpy()
            return o[:, :self.n_out], o[:, self.n_out:] * BETA_SCALE
        out = torch.zeros((P, 2 * self.n_out), dtype=torch.float32, device=self.device)
        for i in range(0, P, self.batch):
            xb = X[i:i + self.batch]
            if xb.shape[0] < self.batch:
                pad = torch.zeros((self.batch - xb.shape[0], self.h0, self.h0, self.c0), device=self.device)
                xb = torch.cat([xb, pad])
            ob = torch.zeros((self.batch, 2 * self.n_out), dtype=torch.float32, device=self.device)
            pam.pam_nn_forward(self.params, xb.contiguous(), ob, self.ws, arch=self.arch)
            out[i:i + self.batch] = ob[:min(self.batch, P - i)]
        o = out.cpu().numpy()
        return o[:, :self.n_out], o[:, self.n_out:] * BETA_SCALE


# Seed threshold on the predicted coefficients (log-space units). Measured on
# held-out patches: the coefficients the network predicts large are reliable,
# the small ones are better left for the active-set iterations to add; a
# seed of {|beta_hat| > 3} cut the mean iterations from 9.8 to 6.8 and the
# worst case from 74 to 14, more than the support logits did (70 % accurate).
SEED_THRESHOLD = 3.0


def warm_start_coefficients(logits, beta, threshold=SEED_THRESHOLD):
    """The warm start handed to the solve: the predicted coefficients whose
    magnitude exceeds `threshold` (their signs seed the active set)."""
    del logits  # the support logits are trained jointly but seed worse
    return np.where(np.abs(beta) > threshold, beta, 0.0).astype(np.float64)


def learned_fit(net, patches, device, precision=pam.PAM_PREC_FP64, budget=48):
    """Fit with the network's warm start; patches not certified within
    `budget` active-set iterations are refitted plainly from zero. Inputs,
    inference (one batched forward pass over all the patches) and the seed
    (the predicted coefficients above SEED_THRESHOLD, pam_nn_seed) stay on
    the device. Returns dict(beta, info, solve_ms, refit, predict_ms)."""
    import torch
    fit = PatchFit(patches.shape[0], device, precision, max_iters=budget)
    Kd = fit.device_field(patches)
    f = fit.fitter
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows = -(-patches.shape[0] // 32) * 32
    X = torch.empty((rows, net.h0, net.h0, net.c0), dtype=torch.float32, device=device)
    pam.pam_nn_inputs(f.problem, f.plan, Kd, X, arch=net.arch)
    out = net.forward_device(X)
    f.model.beta.zero_()
    pam.pam_nn_seed(f.plan, out, SEED_THRESHOLD, f.model, arch=net.arch)
    torch.cuda.synchronize()
    t_pred = (time.perf_counter() - t0) * 1e3
    beta, info, ms = fit.fit(patches, Kd=Kd, seeded=True)
    miss = np.nonzero(info[:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED)[0]
    refit_ms = 0.0
    if len(miss):
        # plain refit of the missed patches only (padded to a square batch)
        T = int(np.ceil(np.sqrt(len(miss))))
        sel = np.concatenate([miss, np.repeat(miss[-1:], T * T - len(miss))])
        plain = PatchFit(T * T, device, precision)
        b2, info2, refit_ms = plain.fit(patches[sel])
        beta[miss] = b2[:len(miss)]
        info[miss] = info2[:len(miss)]
    return dict(beta=beta, info=info, solve_ms=ms + refit_ms, refit=len(miss), predict_ms=t_pred)


# --------------------------------------------------------------------------
# Layered 3-D decompositions: the network (PAM_NN_LAYERED3D) reads each
# subdomain's patch (up to 16 x 16 x 8 cells, z layers as channels) and
# predicts the coefficients of its 32-centre initial lattice; the level-0
# solve starts from them. Inputs, inference and seeding all run on the
# device (pam_nn_layered_inputs, pam_nn_forward, pam_nn_seed).
# --------------------------------------------------------------------------
SEED_THRESHOLD_3D = 1.0


class LayeredWarmStart:
    """Learned warm start of a 3-D decomposition's level-0 solves."""

    def __init__(self, device, batch=256, seed=0, threshold=SEED_THRESHOLD_3D):
        self.net = Network(device, batch=batch, seed=seed, arch=pam.PAM_NN_LAYERED3D)
        self.device = device
        self.threshold = threshold
        self._buf = {}

    def _rows(self, fitter):
        return (fitter.plan.n_subdomains + 31) // 32 * 32

    def inputs(self, fitter, Kd):
        """[rows,16,16,8] device tensor of the patches (rows = S rounded up to 32)."""
        import torch
        rows = self._rows(fitter)
        key = ("x", rows)
        if key not in self._buf:
            self._buf[key] = torch.empty((rows, 16, 16, 8), dtype=torch.float32, device=self.device)
        x = self._buf[key]
        pam.pam_nn_layered_inputs(fitter.problem, fitter.plan, Kd, x)
        return x

    def labels(self, fitter, Kd):
        """Level-0 fit of every subdomain: (inputs [S,16,16,8] device,
        support [S,32], beta [S,32]) as device tensors."""
        S = fitter.plan.n_subdomains
        code = fitter.fit(Kd, levels=0, check=False)
        if code not in (0, 5):
            raise pam.PamError(code, "label fit")
        n_out = self.net.n_out
        beta = fitter.model.beta[:, :n_out].float().clone()
        return self.inputs(fitter, Kd)[:S].clone(), (beta != 0).float(), beta

    def train(self, fitter, fields, epochs=8, lr=2e-3, log=None):
        """Label each field (device tensors of the decomposition's shape) with
        its level-0 fits and train the network on all of them."""
        import torch
        xs, ss, bs = [], [], []
        for Kd in fields:
            x, s, b = self.labels(fitter, Kd)
            xs.append(x); ss.append(s); bs.append(b)
        X, Sp, B = torch.cat(xs), torch.cat(ss), torch.cat(bs)
        P = (X.shape[0] // self.net.batch) * self.net.batch
        return self.net.train(X[:P], Sp[:P], B[:P], epochs=epochs, lr=lr, log=log)

    def seed(self, fitter, Kd):
        """Network inference on the patches of Kd and seeding of model.beta;
        the next fitter.fit(Kd, warm_start=True) starts from it."""
        import torch
        x = self.inputs(fitter, Kd)
        rows = x.shape[0]
        key = ("out", rows)
        if key not in self._buf:
            self._buf[key] = torch.empty((rows, 2 * self.net.n_out), dtype=torch.float32, device=self.device)
            self._buf[("ws", rows)] = torch.empty(pam.pam_nn_sizes(rows, arch=self.net.arch)[1],
                                                  dtype=torch.uint8, device=self.device)
        out = self.net.forward_device(x, self._buf[key], self._buf[("ws", rows)])
        pam.pam_nn_seed(fitter.plan, out, self.threshold, fitter.model, arch=self.net.arch)
