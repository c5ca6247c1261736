"""Pins of the oracle's fit on general meshes given as cells
(oracle.partition_cells, oracle.fit_cells, oracle.errors_cells,
oracle.residual_cells, oracle.mark_cells), each against something other
than the code under test:

- a structured grid handed over as a cell list (centroids, |T| = h^d, global
  order) reproduces the grid path (oracle.fit_all, pinned in
  test_oracle_pins.py) bit for bit, and its errors agree with oracle.errors;
- the patch lists of a shuffled grid are exactly the cells of the patch
  boxes (brute force by cell index, not by coordinates);
- every element lies in exactly one core;
- the measure weights: splitting an element into two halves (same point and
  value, half the measure each) leaves the errors unchanged, and the
  indicators sum to the squared L2 error (Eq. (4) and Eq. (12) with a
  measure per element);
- the per-element marking equals the sort-based definition on planted ties;
- on a triangle mesh and a graded tensor mesh every subdomain certifies, a
  constant field's error is linear in lambda (the Shepard basis reproduces
  constants), and a 1-D step's error does not increase with the levels.
"""
import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields


def _shape_points(shape):
    h = fields.cell_size(shape)
    return fields.cell_centred_points(shape, [n * h for n in shape])


@pytest.mark.parametrize("K,geo,params", [
    (fields.voronoi_field(64, n_sites=10, seed=4), ((64, 64), (4, 4), 2, (4, 4)), dict(levels=2, k_top=8)),
    (fields.voronoi_field(37, n_sites=7, seed=8)[:23, :], ((37, 23), (4, 3), 3, (3, 5)), dict(levels=2, k_top=4)),
    (fields.layered_field((16, 20, 9), seed=31), ((16, 20, 9), (2, 2, 2), 1, (3, 3, 2)), dict(levels=2, k_top=5)),
    (fields.step_field_1d(200, 77), ((200,), (4,), 3, (4,)), dict(levels=3, k_top=3)),
])
def test_grid_as_cells_reproduces_the_grid_path(K, geo, params):
    p = oracle.default_params(**params)
    a = oracle.fit_all(K, *geo, p)
    x, vol, k = fields.grid_as_cells(K, geo[0])
    b = oracle.fit_cells(x, vol, k, *geo, p)
    for key in ("M", "c", "beta"):
        np.testing.assert_array_equal(a[key], b[key])
    ea, eb = oracle.errors(a, K), oracle.errors_cells(b, x, vol, k)
    for key in ("l1", "l2", "l1_log", "max_log10"):
        assert eb[key] == pytest.approx(ea[key], rel=1e-12, abs=1e-15), key


@pytest.mark.parametrize("shape,n_sub,overlap", [((24, 17), (3, 2), 2), ((10, 12, 7), (2, 3, 2), 1), ((50,), (6,), 4)])
def test_patch_lists_of_a_shuffled_grid_are_the_patch_boxes(shape, n_sub, overlap):
    x = _shape_points(shape)
    perm = np.random.default_rng(1).permutation(x.shape[0])
    boxes, start, cells = oracle.partition_cells(shape, n_sub, overlap, x[perm])
    np.testing.assert_array_equal(boxes, oracle.partition(shape, n_sub, overlap))
    dim = len(shape)
    idx = np.stack(np.unravel_index(np.arange(x.shape[0]), tuple(reversed(shape))), 1)[:, ::-1]  # (i, j, k)
    for s in range(boxes.shape[0]):
        lo, hi = boxes[s, 6:6 + dim], boxes[s, 9:9 + dim]
        want = np.flatnonzero(np.all((idx >= lo) & (idx < hi), axis=1))
        got = np.sort(perm[cells[start[s]:start[s + 1]]])
        np.testing.assert_array_equal(got, want)
        assert np.all(np.diff(cells[start[s]:start[s + 1]]) > 0)  # ascending local order


def test_every_element_lies_in_exactly_one_core():
    x, _ = fields.triangle_mesh(40, seed=5)
    boxes, start, cells = oracle.partition_cells((40, 40), (3, 4), 0, x)
    counts = np.bincount(cells, minlength=x.shape[0])
    assert counts.min() == 1 and counts.max() == 1
    # with an overlap the cores still own each element once (Step 4 owner rule)
    K = fields.voronoi_at(x, 6, 5)
    m = oracle.fit_cells(x, np.full(x.shape[0], 0.5 / 1600), K, (40, 40), (3, 4), 2, (3, 3),
                         oracle.default_params(levels=0))
    _, own = oracle.evaluate(m, x, return_owner=True)
    b = m["boxes"]
    h = 1.0 / 40
    for s in range(b.shape[0]):
        sel = own == s
        assert np.all(x[sel] >= b[s, 0:2] * h) and np.all(x[sel] < b[s, 3:5] * h + 1e-15)


def test_splitting_an_element_in_two_halves_keeps_the_errors():
    x, vol = fields.triangle_mesh(32, seed=6)
    K = fields.voronoi_at(x, 8, 6)
    m = oracle.fit_cells(x, vol, K, (32, 32), (2, 2), 1, (4, 4), oracle.default_params(levels=1, k_top=6))
    e = oracle.errors_cells(m, x, vol, K)
    sel = np.arange(0, x.shape[0], 3)
    x2 = np.concatenate([x, x[sel]])
    v2 = vol.copy()
    v2[sel] *= 0.5
    v2 = np.concatenate([v2, vol[sel] * 0.5])
    k2 = np.concatenate([K, K[sel]])
    e2 = oracle.errors_cells(m, x2, v2, k2)
    for key in ("l1", "l2", "l1_log", "max_log10"):
        assert e2[key] == pytest.approx(e[key], rel=1e-12), key
    # dropping the weights would change them
    e3 = oracle.errors_cells(m, x2, np.ones_like(v2), k2)
    assert abs(e3["l1"] - e["l1"]) > 1e-6 * e["l1"]


def test_indicators_sum_to_the_squared_l2_error():
    # one subdomain: sum_T R_T = sum_T |T| (K* - K_T)^2 = l2^2 sum |T| K_T^2
    x, vol = fields.graded_mesh((30, 24), seed=7)
    K = fields.voronoi_at(x, 5, 7)
    m = oracle.fit_cells(x, vol, K, (30, 24), (1, 1), 0, (5, 4), oracle.default_params(levels=0))
    c = m["c"][0, :m["M"][0]]
    W = oracle.assemble(2, np.concatenate([x, np.zeros((x.shape[0], 1))], 1), c)
    R = oracle.residual_cells(W, m["beta"][0, :m["M"][0]], K, vol)
    e = oracle.errors_cells(m, x, vol, K)
    assert R.sum() == pytest.approx(e["l2"] ** 2 * np.sum(vol * K * K), rel=1e-11)
    # a constant measure gives the grid indicator
    R1 = oracle.residual_cells(W, m["beta"][0, :m["M"][0]], K, np.full_like(vol, 0.3))
    np.testing.assert_allclose(R1, oracle.residual(W, m["beta"][0, :m["M"][0]], K, 0.3), rtol=0, atol=0)


def test_marking_with_a_threshold_per_element():
    rng = np.random.default_rng(9)
    for _ in range(20):
        n = 300
        R = rng.choice([0.5, 1.0, 2.0, 3.0], size=n) * 10.0 ** rng.integers(-3, 1, size=n)
        eps = rng.choice([0.0, 1e-3, 0.6, 5.0], size=n)
        k = int(rng.integers(1, 40))
        got = oracle.mark_cells(R, eps, k)
        r32, e32 = R.astype(np.float32), eps.astype(np.float32)
        cand = np.flatnonzero(r32 >= e32)
        order = sorted(cand, key=lambda j: (-float(r32[j]), j))
        np.testing.assert_array_equal(got, np.array(order[:k], dtype=np.int32))
    # equal thresholds: the grid marking
    R = rng.random(200)
    np.testing.assert_array_equal(oracle.mark_cells(R, np.full(200, 0.3), 25), oracle.mark(R, 0.3, 25))


@pytest.mark.parametrize("mesh", ["triangles", "graded2d", "graded3d"])
def test_general_meshes_certify_and_reproduce_constants(mesh):
    if mesh == "triangles":
        shape = (48, 40)
        x, vol = fields.triangle_mesh(48, seed=13, ny=40)
        geo = (shape, (3, 2), 2, (4, 4))
    elif mesh == "graded2d":
        shape = (40, 40)
        x, vol = fields.graded_mesh(shape, seed=14)
        geo = (shape, (2, 2), 1, (4, 4))
    else:
        shape = (12, 14, 8)
        x, vol = fields.graded_mesh(shape, seed=15)
        geo = (shape, (2, 2, 1), 1, (3, 3, 2))
    K = np.full(x.shape[0], 2.5)
    errs = []
    for scale in (0.1, 0.01, 0.001):  # the linear regime
        m = oracle.fit_cells(x, vol, K, *geo, oracle.default_params(levels=0, lambda1_hat=4.59e-4 * scale,
                                                                     lambda2_hat=4.64e-6 * scale))
        assert m["failed"] == 0
        errs.append(oracle.errors_cells(m, x, vol, K)["l1_log"])
    # linear in lambda (the shrinkage of an exactly representable constant)
    assert errs[0] > 0
    assert errs[1] / errs[0] == pytest.approx(0.1, rel=0.1)
    assert errs[2] / errs[1] == pytest.approx(0.1, rel=0.1)
    if mesh == "triangles":
        Kv = fields.voronoi_at(x, 8, 16)
        m = oracle.fit_cells(x, vol, Kv, *geo, oracle.default_params(levels=2, k_top=6))
        assert m["failed"] == 0 and m["M"].max() > 16


def test_step_error_does_not_increase_with_levels_on_a_graded_1d_mesh():
    x, vol = fields.graded_mesh((120,), seed=17)
    K = np.where(x[:, 0] < 0.41, 1e-3, 1.0)
    prev = np.inf
    for lv in range(4):
        m = oracle.fit_cells(x, vol, K, (120,), (1,), 0, (4,), oracle.default_params(levels=lv, k_top=2))
        e = oracle.errors_cells(m, x, vol, K)["l1"]
        assert e <= prev * (1 + 1e-9)
        prev = e
    assert prev < 0.5 * oracle.errors_cells(
        oracle.fit_cells(x, vol, K, (120,), (1,), 0, (4,), oracle.default_params(levels=0, k_top=2)), x, vol, K)["l1"]


def test_a_hole_that_empties_a_patch():
    # reading: no elements -> beta = 0 (the limit of the minimisers as
    # lambda -> 0+ with G = 0, b = 0), stopped at once, K* = 1 in its core;
    # the other subdomains are fitted exactly as without it
    h = 1 / 64
    x, vol = fields.triangle_mesh(64, seed=61)
    x, vol = fields.cut_box(x, vol, (14.5 * h, 30.5 * h), (33.5 * h, 49.5 * h))
    K = fields.voronoi_at(x, 10, 61)
    geo = ((64, 64), (4, 4), 1, (4, 4))
    p = oracle.default_params(levels=2, k_top=6)
    m = oracle.fit_cells(x, vol, K, *geo, p)
    sizes = np.diff(m["patch_start"])
    assert sizes[9] == 0 and (np.delete(sizes, 9) > 0).all()
    assert m["failed"] == 0
    assert m["M"][9] == 16 and not m["beta"][9].any() and m["info"][9, 2] == 0
    np.testing.assert_array_equal(m["c"][9, :16], oracle.initial_dictionary((64, 64), m["boxes"][9, 0:3],
                                                                            m["boxes"][9, 3:6], (4, 4)))
    assert oracle.evaluate(m, np.array([[24.0 * h, 40.0 * h]]))[0] == 1.0
    others = [s for s in range(16) if s != 9]
    m2 = oracle.fit_cells(x, vol, K, *geo, p, which=others)
    for key in ("M", "c", "beta"):
        np.testing.assert_array_equal(m[key][others], m2[key][others])
    e = oracle.errors_cells(m, x, vol, K)
    assert np.isfinite(e["l1"]) and e["l1"] < 1
