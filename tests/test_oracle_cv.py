"""Pins of the oracle's per-subdomain cross-validation of the Elastic Net
weights (oracle.cv_lambda), against closed forms it does not use.

With lambda1 = 0 the Elastic Net is ridge regression with penalty
alpha = N_train lambda2_hat. When every fold has the same size, alpha is the
same for all folds and the held-out residuals have the block form of the
PRESS identity: r_F = (I - H_FF)^{-1} (y_F - (H y)_F), with the full-data
hat matrix H = W (W^T W + alpha I)^{-1} W^T. Leave-one-out is the case of
folds of one cell. A lambda1 above every |b_j| zeroes the coefficients, so
the cross-validation error is the mean of y^2.
"""
import numpy as np
import pytest

import oracle

N_CELLS = (12, 9)   # 108 cells: folds of equal size for k = 2, 3, 4, 108


def _model_and_field(g=(3, 3)):
    x = (np.arange(N_CELLS[0]) + 0.5) / 12.0
    y = (np.arange(N_CELLS[1]) + 0.5) / 12.0
    X, Y = np.meshgrid(x, y, indexing="ij")
    K = np.exp(np.sin(4.0 * X) + 0.7 * np.cos(5.0 * Y) + 0.3 * X * Y)
    K = np.ascontiguousarray(K.T)  # numpy layout [ny, nx] (x fastest in memory)
    model = oracle.fit_all(K, N_CELLS, (1, 1), 0, g, oracle.default_params(levels=0))
    return model, K


def _design(model, K):
    b = model["boxes"][0]
    x, yv, _ = oracle.box_cells(N_CELLS, b[6:9], b[9:12], K)
    M = int(model["M"][0])
    return oracle.assemble(2, x, model["c"][0, :M]), yv


@pytest.mark.parametrize("k", [2, 3, 4, 108])
def test_ridge_cv_matches_the_block_press_identity(k):
    model, K = _model_and_field()
    W, y = _design(model, K)
    N, M = W.shape
    l2h = 3e-4
    alpha = (N - N // k) * l2h
    H = W @ np.linalg.solve(W.T @ W + alpha * np.eye(M), W.T)
    e = y - H @ y
    fold = np.arange(N) % k
    total = 0.0
    for f in range(k):
        F = np.flatnonzero(fold == f)
        rF = np.linalg.solve(np.eye(F.size) - H[np.ix_(F, F)], e[F])
        total += rF @ rF
    got = oracle.cv_lambda(model, K, [(0.0, l2h)], k)
    np.testing.assert_allclose(got["cv"][0, 0], total / N, rtol=1e-8)


def test_large_lambda1_gives_the_mean_square_of_y():
    model, K = _model_and_field()
    W, y = _design(model, K)
    big = 10.0 * np.abs(W.T @ y).max()  # lambda1 = N_train * big > every |b_j|
    got = oracle.cv_lambda(model, K, [(big, 1e-6), (4.59e-4, 4.64e-6)], 3)
    np.testing.assert_allclose(got["cv"][0, 0], np.mean(y * y), rtol=1e-12)
    assert got["choice"][0] == 1 and got["cv"][0, 1] < got["cv"][0, 0]


def test_single_pair_refit_equals_the_level0_fit():
    model, K = _model_and_field()
    p = oracle.default_params(levels=0)
    got = oracle.cv_lambda(model, K, [(p["lambda1_hat"], p["lambda2_hat"])], 4)
    assert got["choice"][0] == 0 and got["certified"][0]
    M = int(model["M"][0])
    scale = np.abs(model["beta"][0, :M]).max()
    np.testing.assert_allclose(got["beta"][0, :M], model["beta"][0, :M], rtol=0, atol=1e-9 * scale)


def test_choice_is_the_first_least_cv_and_ties_take_the_lower_index():
    model, K = _model_and_field()
    pair = (4.59e-4, 4.64e-6)
    got = oracle.cv_lambda(model, K, [(1e-2, 1e-4), pair, pair, (1e-7, 1e-9)], 3)
    cv = got["cv"][0]
    assert cv[1] == cv[2]
    assert got["choice"][0] == int(np.argmin(cv))
    assert got["choice"][0] != 2
