"""Pins of the oracle's glued evaluation (oracle.glue_weights,
oracle.evaluate_glued) against what the construction fixes, independently
of the code under test:

- the weights form a partition of unity on the domain (any number of
  subdomains, ragged cores, 1-3 D);
- a model whose coefficients are one constant c_i per subdomain has
  u_i = c_i exactly (Shepard rows sum to one), so across an interface the
  glued log-field is the smoothstep blend of the two constants, and at a
  2-D corner the product of the two 1-D blends;
- farther than the band from every interface it equals the piecewise
  evaluation; as the band shrinks the glued field converges to it;
- it is continuous across interfaces where the piecewise field jumps.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields


def _smooth(t):
    t = min(max(t, 0.0), 1.0)
    return 3 * t * t - 2 * t * t * t


@pytest.mark.parametrize("n_cells,n_sub,band", [
    ((50,), (7,), 2.5), ((37, 23), (4, 3), 1.5), ((24, 30, 12), (3, 5, 2), 1.0), ((64, 64), (8, 8), 4.0)])
def test_weights_are_a_partition_of_unity(n_cells, n_sub, band):
    rng = np.random.default_rng(3)
    h = 1.0 / max(n_cells)
    pts = rng.random((4000, len(n_cells))) * (np.asarray(n_cells) * h)
    psi = oracle.glue_weights(n_cells, n_sub, pts, band)
    np.testing.assert_allclose(psi.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert (psi >= 0).all() and (psi <= 1).all()
    # at most 2^dim subdomains overlap anywhere
    assert (psi > 0).sum(axis=1).max() <= 2 ** len(n_cells)


def _constant_model(n_cells, n_sub, g, consts):
    boxes = oracle.partition(n_cells, n_sub, 0)
    S = boxes.shape[0]
    m = int(np.prod(g))
    c = np.zeros((S, m, 4))
    for s in range(S):
        c[s] = oracle.initial_dictionary(n_cells, boxes[s, 0:3], boxes[s, 3:6], g)
    beta = np.repeat(np.asarray(consts, dtype=np.float64)[:, None], m, axis=1)
    return dict(boxes=boxes, M=np.full(S, m, dtype=np.int32), c=c, beta=beta, m_cap=m,
                n_cells=tuple(n_cells), n_sub=tuple(n_sub))


def test_constant_pieces_blend_by_the_smoothstep_across_an_interface():
    n_cells, n_sub, band = (40, 20), (2, 1), 3.0
    model = _constant_model(n_cells, n_sub, (3, 3), [0.7, -1.9])
    h = 1.0 / 40
    xI, delta = 20 * h, band * h
    xs = np.linspace(xI - 1.5 * delta, xI + 1.5 * delta, 301)
    pts = np.stack([xs, np.full_like(xs, 0.37 * 20 * h)], axis=1)
    got = oracle.evaluate_glued(model, pts, band, log_space=True)
    want = np.array([0.7 + (-1.9 - 0.7) * _smooth((x - xI + delta) / (2 * delta)) for x in xs])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_constant_pieces_at_a_corner_blend_as_a_product():
    n_cells, n_sub, band = (30, 30), (2, 2), 2.0
    cs = [1.0, 2.5, -0.5, 4.0]  # subdomain index = ix + 2 iy
    model = _constant_model(n_cells, n_sub, (2, 2), cs)
    h = 1.0 / 30
    xI, delta = 15 * h, band * h
    rng = np.random.default_rng(5)
    pts = xI + (rng.random((500, 2)) * 2 - 1) * 1.2 * delta
    got = oracle.evaluate_glued(model, pts, band, log_space=True)
    for (x, y), v in zip(pts, got):
        px = _smooth((x - xI + delta) / (2 * delta))
        py = _smooth((y - xI + delta) / (2 * delta))
        want = (cs[0] * (1 - px) * (1 - py) + cs[1] * px * (1 - py) + cs[2] * (1 - px) * py + cs[3] * px * py)
        assert abs(v - want) <= 1e-13


def _fitted_model():
    K = fields.voronoi_field(n=64, n_sites=10, seed=4)
    model = oracle.fit_all(K, (64, 64), (4, 4), 2, (4, 4), oracle.default_params(levels=1, k_top=8))
    return model


def test_equals_the_piecewise_field_away_from_the_bands():
    model = _fitted_model()
    band = 1.5
    h = 1.0 / 64
    rng = np.random.default_rng(6)
    pts = rng.random((3000, 2))
    d = np.abs(((pts / h) + 8) % 16 - 8)  # distance in cells to the nearest core face (cores of 16)
    far = np.all(d > band + 1e-9, axis=1)
    got = oracle.evaluate_glued(model, pts[far], band, log_space=True)
    want = oracle.evaluate(model, pts[far], log_space=True)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_continuous_across_interfaces_where_the_piecewise_field_jumps():
    model = _fitted_model()
    h = 1.0 / 64
    ys = (np.arange(64) + 0.5) * h
    xI = 16 * h
    jumps_pw, jumps_gl = [], []
    for eps in (1e-3 * h, 1e-6 * h):
        left = np.stack([np.full_like(ys, xI - eps), ys], axis=1)
        right = np.stack([np.full_like(ys, xI + eps), ys], axis=1)
        jumps_gl.append(np.abs(oracle.evaluate_glued(model, left, 1.0, True)
                               - oracle.evaluate_glued(model, right, 1.0, True)).max())
        jumps_pw.append(np.abs(oracle.evaluate(model, left, True) - oracle.evaluate(model, right, True)).max())
    assert jumps_pw[1] > 1e-3          # the piecewise surrogate jumps
    assert jumps_gl[0] < 1e-2 * jumps_pw[1]
    assert jumps_gl[1] < 1e-3 * jumps_gl[0] + 1e-12  # shrinks with eps (Lipschitz)


def test_small_band_converges_to_the_piecewise_field():
    model = _fitted_model()
    rng = np.random.default_rng(8)
    pts = rng.random((2000, 2))
    pw = oracle.evaluate(model, pts, log_space=True)
    errs = [np.abs(oracle.evaluate_glued(model, pts, b, True) - pw).mean() for b in (2.0, 0.5, 0.125)]
    assert errs[0] > errs[1] > errs[2] > 0
