"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a closed
form (Theorem 1), an invariant (partition of unity, convex-combination
bounds), a special case that reduces to a textbook or library routine
(ridge solve, zero-solution threshold, numpy products, scikit-learn's Elastic
Net), brute force on tiny inputs (sign-pattern enumeration, sorting), or a
number the paper prints (tests/golden/*.txt, each with its citation).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2605_16564_gb300 import fields

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Step 1 ---

@pytest.mark.parametrize("n_cells,n_sub,overlap", [
    ((256, 256), (8, 8), 2), ((60, 220, 85), (6, 22, 17), 1), ((37, 23), (4, 3), 3),
    ((50,), (7,), 2), ((64, 64), (1, 1), 0)])
def test_partition_owns_every_cell_once(n_cells, n_sub, overlap):
    boxes = oracle.partition(n_cells, n_sub, overlap)
    dim = len(n_cells)
    cover = np.zeros(tuple(reversed(n_cells)), dtype=np.int32)
    for bx in boxes:
        lo, hi, plo, phi = bx[0:3], bx[3:6], bx[6:9], bx[9:12]
        sl = tuple(slice(lo[a], hi[a]) for a in reversed(range(dim)))
        cover[sl] += 1
        for a in range(dim):
            assert plo[a] == max(lo[a] - overlap, 0)
            assert phi[a] == min(hi[a] + overlap, n_cells[a])
    assert cover.min() == 1 and cover.max() == 1


def test_partition_patch_sizes_of_the_workloads():
    # 256^2 in 8x8 cores of 32^2 grown by 2 cells: 36^2, 34x36, 34^2.
    b = oracle.partition((256, 256), (8, 8), 2)
    n = np.prod(b[:, 9:12] - b[:, 6:9], axis=1)
    assert set(n.tolist()) == {1156, 1224, 1296} and n.sum() == 80656
    # 60x220x85 in 6x22x17 cores of 10x10x5 grown by 1 cell.
    b = oracle.partition((60, 220, 85), (6, 22, 17), 1)
    n = np.prod(b[:, 9:12] - b[:, 6:9], axis=1)
    assert n.max() == 12 * 12 * 7 and n.sum() == 2145780
    assert np.prod(b[:, 3:6] - b[:, 0:3], axis=1).sum() == 60 * 220 * 85


def test_owner_lookup_brute_force():
    n_cells, n_sub = (37, 23), (4, 3)
    boxes = oracle.partition(n_cells, n_sub, 0)
    h = 1.0 / 37
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 1, size=(4000, 2)) * np.array([37 * h, 23 * h])
    # points exactly on interior and outer faces
    faces = np.array([[b[0] * h, (b[1] + 0.5) * h] for b in boxes] +
                     [[37 * h, 23 * h], [0.0, 0.0], [37 * h, 0.3]])
    pts = np.concatenate([pts, faces])
    model = dict(n_cells=n_cells, n_sub=n_sub, m_cap=1, M=np.ones(len(boxes), np.int32),
                 c=np.tile(np.array([0.5, 0.5, 0, 1.0]), (len(boxes), 1, 1)),
                 beta=np.zeros((len(boxes), 1)))
    _, own = oracle.evaluate(model, pts, log_space=True, return_owner=True)
    for p, s in zip(pts, own):
        u = p * 37.0
        i = np.minimum(np.floor(u).astype(int), np.array(n_cells) - 1)
        b = boxes[s]
        assert all(b[a] <= i[a] < b[3 + a] for a in range(2)), (p, s)
        # exactly one core box contains the cell index
        assert sum(all(bb[a] <= i[a] < bb[3 + a] for a in range(2)) for bb in boxes) == 1
    out = oracle.evaluate(model, np.array([[-1e-3, 0.5], [0.5, 23 * h + 1e-9]]), log_space=True)
    assert np.isnan(out).all()


def test_initial_dictionary_lattice_and_table1_widths():
    c = oracle.initial_dictionary((64, 64), (0, 0, 0), (64, 64, 1), (16, 16))
    assert c.shape == (256, 4)
    np.testing.assert_allclose(c[:16, 0], (np.arange(16) + 0.5) / 16, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c[::16, 1], (np.arange(16) + 0.5) / 16, rtol=0, atol=1e-15)
    assert np.all(c[:, 3] == 1.0 / 16)
    for g, sig, digits in _golden_rows("table1_dictionaries.txt"):
        g, sig, digits = int(g), float(sig), int(digits)
        c = oracle.initial_dictionary((32, 32), (0, 0, 0), (32, 32, 1), (g, g))
        assert len(c) == g * g
        assert float(f"{c[0, 3]:.{digits}g}") == pytest.approx(sig, rel=1e-12)


# ------------------------------------------------------- Step 2: assembly ---

def _random_problem(rng, n=200, m=30, dim=2, spread=0.2):
    x = np.zeros((n, 3)); x[:, :dim] = rng.uniform(0, 1, size=(n, dim))
    c = np.zeros((m, 4)); c[:, :dim] = rng.uniform(0, 1, size=(m, dim))
    c[:, 3] = rng.uniform(0.3, 1.0, size=m) * spread
    return x, c


def test_shepard_rows_are_a_partition_of_unity():
    rng = np.random.default_rng(1)
    for dim in (1, 2, 3):
        x, c = _random_problem(rng, dim=dim, m=57)
        W = oracle.assemble(dim, x, c)
        assert (W >= 0).all()
        assert np.abs(W.sum(axis=1) - 1).max() <= 57 * 2.0 ** -52


def test_shepard_matches_raw_gaussian_quotient():
    # Eq. (6) and Eq. (10) evaluated literally, where no Gaussian underflows.
    rng = np.random.default_rng(2)
    x, c = _random_problem(rng, spread=1.0)
    W = oracle.assemble(2, x, c)
    d2 = ((x[:, None, :2] - c[None, :, :2]) ** 2).sum(-1)
    phi = np.exp(-d2 / (2 * c[None, :, 3] ** 2))
    np.testing.assert_allclose(W, phi / phi.sum(1, keepdims=True), rtol=1e-13, atol=0)


def test_shepard_is_finite_where_every_gaussian_underflows():
    c = np.array([[0.0, 0, 0, 1e-3], [1.0, 0, 0, 1e-3]])
    x = np.array([[0.3, 0, 0], [0.9, 0, 0]])
    W = oracle.assemble(1, x, c)
    assert np.isfinite(W).all()
    np.testing.assert_array_equal(W, [[1.0, 0.0], [0.0, 1.0]])


def _single_model(c, beta, n_cells=(64, 64)):
    m = len(c)
    return dict(n_cells=n_cells, n_sub=(1,) * len(n_cells), m_cap=m,
                M=np.array([m], np.int32), c=np.asarray(c, float)[None],
                beta=np.asarray(beta, float)[None])


def test_constant_coefficients_reproduce_constants_exactly_and_bounds():
    # Partition of unity (section 3.2): beta = c * 1 gives the constant c;
    # any beta gives a convex combination inside [min beta, max beta].
    rows = np.array([[float(v) for v in r] for r in _golden_rows("shepard_example.txt")])
    c = np.zeros((3, 4)); c[:, :2] = rows[:, :2]; c[:, 3] = rows[:, 2]
    pts = fields.cell_centred_points((101, 101), (1.0, 1.0))
    for const in (-2.5, 0.0, 3.75):
        v = oracle.evaluate(_single_model(c, [const] * 3), pts, log_space=True)
        assert np.abs(v - const).max() <= 4 * np.finfo(float).eps * max(1, abs(const))
    beta = np.array([1.0, -0.5, 2.0])
    v = oracle.evaluate(_single_model(c, beta), pts, log_space=True)
    assert v.min() >= beta.min() - 1e-15 and v.max() <= beta.max() + 1e-15
    K = oracle.evaluate(_single_model(c, beta), pts)
    np.testing.assert_allclose(K, np.exp(v), rtol=1e-15)


def _theorem1_model(c_, sigma, b_, v):
    """Two-centre Shepard RBF of Theorem 1: c1 = c v, c2 = gamma c v,
    gamma = -1 - 2 b / (c |v|^2), equal widths, beta = (1, 0)."""
    v = np.asarray(v, float)
    gamma = -1.0 - 2.0 * b_ / (c_ * v.dot(v))
    cc = np.zeros((2, 4))
    cc[0, :len(v)] = c_ * v
    cc[1, :len(v)] = gamma * c_ * v
    cc[:, 3] = sigma
    return cc


@pytest.mark.parametrize("c_,sigma,b_,theta", [
    (0.05, 0.02, 0.0, 0.3), (0.1, 0.05, -0.02, 1.1), (0.2, 0.03, 0.05, 2.0)])
def test_theorem1_two_centre_shepard_is_logistic(c_, sigma, b_, theta):
    # Theorem 1 (section 4.1): K*(x) = 1 / (1 + exp(-2 (b + c) y / sigma^2)),
    # y = <v, x> + b, for points around the hyperplane (the domain is shifted
    # so that it contains them; the identity holds for every x).
    v = np.array([math.cos(theta), math.sin(theta)])
    cc = _theorem1_model(c_, sigma, b_, v)
    shift = np.array([0.5, 0.5])
    cc[:, :2] += shift  # translate the whole configuration into [0,1]^2
    rng = np.random.default_rng(3)
    x = shift + rng.uniform(-0.2, 0.2, size=(500, 2))
    val = oracle.evaluate(_single_model(cc, [1.0, 0.0], n_cells=(10, 10)), x, log_space=True)
    y = (x - shift) @ v + b_
    expect = 1.0 / (1.0 + np.exp(-2.0 * (b_ + c_) * y / sigma ** 2))
    # the exponent carries an absolute rounding error of about eps times
    # |x - c|^2 / sigma^2 (<= ~400 here), hence the 1e-13 allowance
    np.testing.assert_allclose(val, expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("c_,sigma,b_", [
    (0.05, 0.01, 0.0), (0.1, 0.02, 0.0), (0.03, 0.004, 0.0), (0.08, 0.015, 0.01)])
def test_theorem1_l1_error_closed_form(c_, sigma, b_):
    # Eq. (13)/(15): int |H(y) - K*(y)| dy = ln 2 * sigma^2 / (c + b), the
    # integral taken numerically through the oracle's evaluation along the
    # normal line (composite Simpson on each side of the kink at y = 0).
    v = np.array([1.0])
    cc = _theorem1_model(c_, sigma, b_, v)
    x0 = 0.5
    cc[:, 0] += x0 + b_  # the interface <v, x> + b = 0 moves to x = x0
    rate = 2.0 * (b_ + c_) / sigma ** 2
    Y = 40.0 / rate
    assert Y < 0.45
    n = 4000
    model = _single_model(cc, [1.0, 0.0], n_cells=(16,))
    total = 0.0
    for side in (-1.0, 1.0):
        ys = np.linspace(0.0, Y, 2 * n + 1) * side
        Kst = oracle.evaluate(model, (x0 + ys)[:, None], log_space=True)
        H = np.where(ys > 0, 1.0, np.where(ys < 0, 0.0, 0.5))
        f = np.abs(H - Kst)
        f[0] = 0.5  # the one-sided limit at the kink, |H - K*| -> 1/2
        hh = Y / (2 * n)
        total += hh / 3.0 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    expect = math.log(2.0) * sigma ** 2 / (c_ + b_)
    assert total == pytest.approx(expect, rel=1e-9)


# ----------------------------------------------------------- Step 2: Gram ---

def test_gram_against_library_product():
    rng = np.random.default_rng(4)
    x, c = _random_problem(rng, n=300, m=41)
    W = oracle.assemble(2, x, c)
    y = rng.standard_normal(300)
    G, b = oracle.gram(W, y)
    np.testing.assert_allclose(G, W.T @ W, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(b, W.T @ y, rtol=1e-12, atol=1e-13)
    assert np.array_equal(G, G.T)
    np.testing.assert_allclose(np.diag(G), (W * W).sum(0), rtol=1e-13)


# ---------------------------------------------------- Step 2: Elastic Net ---

def _enet_problem(seed, n=60, m=6, dim=1):
    rng = np.random.default_rng(seed)
    x, c = _random_problem(rng, n=n, m=m, dim=dim, spread=0.3)
    W = oracle.assemble(dim, x, c)
    y = rng.standard_normal(n) * 2 + np.sin(6 * x[:, 0])
    G, b = oracle.gram(W, y)
    return W, y, G, b


def _brute_force_enet(G, b, lam1, lam2):
    """Enumerate all 3^M sign patterns; keep the one satisfying the KKT
    conditions of Eq. (2) (unique by strict convexity)."""
    import itertools
    m = len(b)
    hits = []
    for pat in itertools.product((-1, 0, 1), repeat=m):
        s = np.array(pat, float)
        S = np.nonzero(s)[0]
        beta = np.zeros(m)
        if len(S):
            A = G[np.ix_(S, S)] + lam2 * np.eye(len(S))
            beta[S] = np.linalg.solve(A, b[S] - lam1 * s[S])
            if np.any(np.sign(beta[S]) != s[S]):
                continue
        g = b - G @ beta
        off = np.setdiff1d(np.arange(m), S)
        if np.all(np.abs(g[off]) <= lam1 * (1 + 1e-12)):
            hits.append(beta)
    return hits


@pytest.mark.parametrize("seed,m,lam1", [(0, 5, 0.3), (1, 6, 1.0), (2, 7, 0.05), (3, 6, 3.0),
                                          (4, 7, 0.6)])
def test_enet_matches_brute_force_support_enumeration(seed, m, lam1):
    W, y, G, b = _enet_problem(seed, m=m)
    lam2 = 0.01
    hits = _brute_force_enet(G, b, lam1, lam2)
    assert len(hits) == 1
    beta, info = oracle.enet(G, b, lam1, lam2)
    assert info["certified"]
    np.testing.assert_array_equal(beta != 0, hits[0] != 0)
    np.testing.assert_allclose(beta, hits[0], rtol=1e-10, atol=1e-12)


def test_enet_zero_solution_threshold():
    # KKT at beta = 0: the minimiser is 0 iff lambda1 >= max_j |b_j|.
    W, y, G, b = _enet_problem(5, m=20, n=100)
    lam = np.abs(b).max()
    beta, info = oracle.enet(G, b, lam, 0.1)
    assert info["certified"] and np.all(beta == 0.0)
    beta, _ = oracle.enet(G, b, lam * (1 - 1e-6), 0.1)
    assert np.count_nonzero(beta) == 1 and np.argmax(np.abs(beta)) == np.argmax(np.abs(b))


def test_enet_without_l1_is_the_ridge_solve():
    W, y, G, b = _enet_problem(6, m=25, n=120)
    lam2 = 0.05
    beta, info = oracle.enet(G, b, 0.0, lam2)
    assert info["certified"]
    ridge = np.linalg.solve(G + lam2 * np.eye(len(b)), b)
    np.testing.assert_allclose(beta, ridge, rtol=1e-9, atol=1e-11)


def test_enet_diagonal_design_is_the_soft_threshold():
    d = np.array([2.0, 0.5, 3.0, 1.0, 4.0])
    G = np.diag(d)
    b = np.array([1.5, -0.2, -4.0, 0.9, 0.05])
    lam1, lam2 = 0.8, 0.1
    beta, _ = oracle.enet(G, b, lam1, lam2)
    expect = np.sign(b) * np.maximum(np.abs(b) - lam1, 0) / (d + lam2)
    np.testing.assert_allclose(beta, expect, rtol=1e-15, atol=0)


def test_enet_matches_scikit_learn():
    sk = pytest.importorskip("sklearn.linear_model")
    W, y, G, b = _enet_problem(7, m=30, n=150)
    n = len(y)
    lam1, lam2 = 0.2, 0.03
    # scikit-learn minimises 1/(2n)|y - Xw|^2 + a r |w|_1 + a (1-r)/2 |w|^2,
    # i.e. Eq. (2) divided by n with a r = lam1 / n and a (1 - r) = lam2 / n.
    a = (lam1 + lam2) / n
    r = lam1 / (lam1 + lam2)
    model = sk.ElasticNet(alpha=a, l1_ratio=r, fit_intercept=False, tol=1e-14,
                          max_iter=1000000, selection="cyclic").fit(W, y)
    beta, _ = oracle.enet(G, b, lam1, lam2)
    np.testing.assert_allclose(beta, model.coef_, rtol=1e-6, atol=1e-8)
    np.testing.assert_array_equal(beta != 0, model.coef_ != 0)


def test_enet_is_a_minimum_of_the_objective():
    W, y, G, b = _enet_problem(8, m=40, n=200, dim=2)
    lam1, lam2 = 0.5, 0.02
    beta, info = oracle.enet(G, b, lam1, lam2)
    yty = y @ y
    f0 = oracle.enet_objective(G, b, yty, lam1, lam2, beta)
    direct = 0.5 * np.sum((y - W @ beta) ** 2) + lam1 * np.abs(beta).sum() + 0.5 * lam2 * beta @ beta
    assert f0 == pytest.approx(direct, rel=1e-12)
    rng = np.random.default_rng(9)
    for _ in range(200):
        d = rng.standard_normal(len(beta)) * 10.0 ** rng.uniform(-6, -1)
        assert oracle.enet_objective(G, b, yty, lam1, lam2, beta + d) >= f0 - 1e-10 * abs(f0)


def test_enet_warm_start_reaches_the_same_minimiser():
    W, y, G, b = _enet_problem(10, m=40, n=200, dim=2)
    beta0, _ = oracle.enet(G, b, 0.4, 0.02)
    rng = np.random.default_rng(11)
    beta1, info = oracle.enet(G, b, 0.4, 0.02, beta0=rng.standard_normal(40))
    assert info["certified"]
    np.testing.assert_allclose(beta1, beta0, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- Step 3 ---

def test_residual_indicators_sum_to_the_squared_l2_error():
    # Eq. (4) is the elementwise L2 error of K*: on one subdomain without
    # overlap, sum_T R_T / sum_T |T| K_T^2 equals the squared relative L2
    # error of Eq. (12) computed through the independent evaluation path.
    K = fields.voronoi_field(24, n_sites=6, seed=12)
    n_cells = (24, 24)
    x, y, kv = oracle.box_cells(n_cells, (0, 0, 0), (24, 24, 1), K)
    c = oracle.initial_dictionary(n_cells, (0, 0, 0), (24, 24, 1), (6, 6))
    W = oracle.assemble(2, x, c)
    G, b = oracle.gram(W, y)
    beta, _ = oracle.enet(G, b, 24 * 24 * 4.59e-4, 24 * 24 * 4.64e-6)
    vol = (1 / 24) ** 2
    R = oracle.residual(W, beta, kv, vol)
    model = _single_model(c, beta, n_cells)
    err = oracle.errors(model, K)
    assert R.sum() / (vol * (kv ** 2).sum()) == pytest.approx(err["l2"] ** 2, rel=1e-11)
    assert np.all(R >= 0)


# Gauss-Legendre indicators (quad = 1), the first "next" row: pinned by the
# rule's exactness on cubics, a constant surrogate, a brute-force fine
# subdivision and the L2 identity above under the same rule.

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_gauss_legendre_nodes_integrate_cubics_exactly(dim):
    rng = np.random.default_rng(31)
    h = 0.37
    x0 = rng.uniform(-1, 1, size=dim)
    pts = oracle.gl_points(x0, h)
    assert pts.shape == (2 ** dim, dim)
    # the cell average of prod_a x_a^p_a, exactly, for every degree <= 3
    def exact(p):
        v = 1.0
        for a in range(dim):
            lo, hi = x0[a] - h / 2, x0[a] + h / 2
            v *= (hi ** (p[a] + 1) - lo ** (p[a] + 1)) / ((p[a] + 1) * h)
        return v
    for p in np.ndindex(*([4] * dim)):
        q = np.prod(pts ** np.array(p), axis=1).mean()
        assert q == pytest.approx(exact(p), rel=1e-12, abs=1e-14), p
    # ... and not for degree 4 (it is not the midpoint rule in disguise)
    p4 = [4] + [0] * (dim - 1)
    assert abs(np.prod(pts ** np.array(p4), axis=1).mean() - exact(p4)) > 1e-6


def test_gauss_legendre_residual_of_a_constant_surrogate():
    # W rows sum to one, so beta = b for every centre gives K* = e^b at every
    # node: R_T = |T| (e^b - K_T)^2 for each rule.
    rng = np.random.default_rng(32)
    x, c = _random_problem(rng, n=40, m=9, dim=2, spread=0.5)
    kv = rng.uniform(0.5, 2.0, size=40)
    beta = np.full(9, 0.3)
    vol, h = 0.01, 0.1
    R = oracle.residual_gl(x, c, beta, kv, vol, h, 2)
    np.testing.assert_allclose(R, vol * (np.exp(0.3) - kv) ** 2, rtol=1e-12)


def test_gauss_legendre_residual_against_fine_subdivision():
    # a smooth surrogate (wide Gaussians): the two-point rule matches a 64 x 64
    # midpoint subdivision of each cell far better than the one-point rule
    n_cells = (12, 12)
    h = 1 / 12
    c = oracle.initial_dictionary(n_cells, (0, 0, 0), (12, 12, 1), (3, 3))
    rng = np.random.default_rng(33)
    beta = rng.normal(size=c.shape[0])
    x, _, _ = oracle.box_cells(n_cells, (0, 0, 0), (12, 12, 1), np.ones((12, 12)))
    kv = np.full(x.shape[0], 1.7)
    vol = h * h
    R_gl = oracle.residual_gl(x, c, beta, kv, vol, h, 2)
    R_mid = oracle.residual(oracle.assemble(2, x, c), beta, kv, vol)
    f = (np.arange(64) + 0.5) / 64 - 0.5
    R_ref = np.zeros(x.shape[0])
    for j in range(x.shape[0]):
        sub = np.zeros((64 * 64, 3))
        sub[:, 0] = x[j, 0] + np.repeat(f, 64) * h
        sub[:, 1] = x[j, 1] + np.tile(f, 64) * h
        t = oracle.assemble(2, sub, c) @ beta
        R_ref[j] = vol * np.mean((np.exp(t) - kv[j]) ** 2)
    e_gl = np.abs(R_gl - R_ref) / R_ref
    e_mid = np.abs(R_mid - R_ref) / R_ref
    assert e_gl.max() <= 1e-3
    assert np.median(e_gl) < 0.05 * np.median(e_mid)


def test_gauss_legendre_indicators_sum_to_the_squared_l2_error():
    # the L2 identity of the midpoint test, with both sides on the same
    # two-point rule (the errors through the independent evaluation path)
    K = fields.voronoi_field(24, n_sites=6, seed=12)
    n_cells = (24, 24)
    x, y, kv = oracle.box_cells(n_cells, (0, 0, 0), (24, 24, 1), K)
    c = oracle.initial_dictionary(n_cells, (0, 0, 0), (24, 24, 1), (6, 6))
    W = oracle.assemble(2, x, c)
    G, b = oracle.gram(W, y)
    beta, _ = oracle.enet(G, b, 24 * 24 * 4.59e-4, 24 * 24 * 4.64e-6)
    vol = (1 / 24) ** 2
    R = oracle.residual_gl(x, c, beta, kv, vol, 1 / 24, 2)
    model = _single_model(c, beta, n_cells)
    err = oracle.errors(model, K, quad=1)
    assert R.sum() / (vol * (kv ** 2).sum()) == pytest.approx(err["l2"] ** 2, rel=1e-11)


def test_algorithm1_with_gauss_legendre_indicators_certifies():
    K = fields.voronoi_field(64, n_sites=8, seed=34)
    params = oracle.default_params(k_top=5, levels=2, quad=1)
    ref = oracle.fit_all(K, (64, 64), (2, 2), 1, (4, 4), params)
    assert ref["failed"] == 0
    assert np.all(ref["M"] == 16 + 2 * 3 * 5)


def test_mark_matches_sorting():
    rng = np.random.default_rng(13)
    for trial in range(20):
        n = int(rng.integers(1, 300))
        R = rng.exponential(size=n) * 10.0 ** rng.uniform(-3, 3)
        if trial % 3 == 0:  # planted exact ties
            R[rng.integers(0, n, size=n // 2)] = R[0]
        eps = np.quantile(R, rng.uniform(0, 1))
        k = int(rng.integers(0, 60))
        keys = R.astype(np.float32)
        cand = [j for j in range(n) if keys[j] >= np.float32(eps)]
        order = sorted(cand, key=lambda j: (-keys[j], j))[:k]
        np.testing.assert_array_equal(oracle.mark(R, eps, k), order)


def test_mark_is_empty_below_tolerance():
    R = np.array([1e-9, 2e-9, 5e-10])
    assert len(oracle.mark(R, 1e-8, 5)) == 0


def test_enrichment_counts_of_table2():
    # Table 2: +3 x 204 centres per round on a 32 x 32 grid in 2-D.
    rows = [(int(r), int(m)) for r, m in _golden_rows("table2_center_counts.txt")]
    n_cells = (32, 32)
    x, _, _ = oracle.box_cells(n_cells, (0, 0, 0), (32, 32, 1), np.ones((32, 32)))
    c = oracle.initial_dictionary(n_cells, (0, 0, 0), (32, 32, 1), (32, 32))
    rng = np.random.default_rng(14)
    assert len(c) == rows[0][1]
    for r, m_expected in rows[1:]:
        R = rng.exponential(size=len(x))
        mk = oracle.mark(R, -np.inf, 204)
        c = oracle.enrich(2, c, mk, x, (0, 0), (1, 1), 0.5, 10 ** 6)
        assert len(c) == m_expected, r


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_enrichment_geometry(dim):
    rng = np.random.default_rng(15 + dim)
    m = 12
    c = np.zeros((m, 4)); c[:, :dim] = rng.uniform(0.2, 0.8, size=(m, dim))
    c[:, 3] = rng.uniform(0.05, 0.1, size=m)
    x = np.zeros((40, 3)); x[:, :dim] = rng.uniform(0.3, 0.7, size=(40, dim))
    marked = np.array([3, 17, 0, 39], np.int32)
    eta = 0.5
    out = oracle.enrich(dim, c, marked, x, [0.0] * dim, [1.0] * dim, eta, 1000)
    assert len(out) == m + len(marked) * (dim + 1)
    np.testing.assert_array_equal(out[:m], c)
    for t, j in enumerate(marked):
        d2 = ((c[:, :dim] - x[j, :dim]) ** 2).sum(1)
        p = int(np.argmin(d2))
        new = out[m + t * (dim + 1): m + (t + 1) * (dim + 1)]
        assert np.all(new[:, 3] == eta * c[p, 3])  # width ratio exactly eta
        off = new[:, :dim] - x[j, :dim]
        np.testing.assert_allclose(np.linalg.norm(off, axis=1), eta * c[p, 3], rtol=1e-14)
        np.testing.assert_allclose(off.sum(0), 0.0, atol=1e-15)  # simplex centred on x_T
        if dim > 1:  # distinct directions, equal pairwise angles
            u = off / np.linalg.norm(off, axis=1, keepdims=True)
            gram = u @ u.T
            np.testing.assert_allclose(gram[~np.eye(dim + 1, dtype=bool)], -1.0 / dim, atol=1e-14)


def test_enrichment_clips_to_the_patch_and_respects_the_cap():
    c = np.array([[0.0, 0.0, 0, 0.2]])
    x = np.array([[0.01, 0.01, 0]])
    out = oracle.enrich(2, c, np.array([0], np.int32), x, (0.0, 0.0), (1.0, 1.0), 0.5, 1000)
    assert np.all(out[1:, :2] >= 0.0) and np.all(out[1:, :2] <= 1.0)
    capped = oracle.enrich(2, c, np.array([0, 0], np.int32), np.vstack([x, x]), (0, 0), (1, 1), 0.5, 3)
    assert len(capped) == 3


# ------------------------------------------------- Algorithm 1 end to end ---

def test_algorithm1_count_rule_without_tolerance():
    K = fields.voronoi_field(16, n_sites=5, seed=16)
    p = oracle.default_params(k_top=20, levels=3, eps_tol_rel=-1.0)
    mdl = oracle.fit_all(K, (16, 16), (1, 1), 0, (8, 8), p)
    assert mdl["M"][0] == 64 + 3 * 20 * 3
    assert mdl["info"][0, 2] == 3 and mdl["info"][0, 3] == 1


def test_algorithm1_step_function_error_decreases_with_refinement():
    # Examples 1-3 (section 3.5): a 1-D step captured better as centres are
    # added where the residual is largest.
    n = 256
    K = fields.step_field_1d(n, n // 2)
    errs = []
    for levels in range(4):
        p = oracle.default_params(k_top=2, levels=levels)
        mdl = oracle.fit_all(K, (n,), (1,), 0, (2,), p)
        assert mdl["failed"] == 0
        errs.append(oracle.errors(mdl, K)["l1"])
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.6 * errs[0], errs


def test_constant_field_error_vanishes_linearly_with_lambda():
    K = np.full((20, 20), 7.0)
    errs = []
    for scale in (1.0, 0.1, 0.01):
        p = oracle.default_params(k_top=5, levels=0, lambda1_hat=4.59e-4 * scale,
                                  lambda2_hat=4.64e-6 * scale)
        mdl = oracle.fit_all(K, (20, 20), (1, 1), 0, (5, 5), p)
        errs.append(oracle.errors(mdl, K)["l1_log"])
    assert errs[0] > 0
    # linear in lambda: a factor 10 less weight gives ~10x less error (a
    # quadratic or square-root law would give 0.01 or 0.32)
    assert errs[1] / errs[0] == pytest.approx(0.1, rel=0.1)
    assert errs[2] / errs[1] == pytest.approx(0.1, rel=0.1)


def test_algorithm1_certifies_every_subdomain_of_a_batched_case():
    K = fields.voronoi_field(64, n_sites=10, seed=17)
    p = oracle.default_params(k_top=10, levels=2)
    mdl = oracle.fit_all(K, (64, 64), (4, 4), 2, (4, 4), p)
    assert mdl["failed"] == 0
    assert np.all(mdl["info"][:, 3] == 1)
    assert np.all(mdl["M"] >= 16) and np.all(mdl["M"] <= 16 + 2 * 3 * 10)
    lam = [float(v) for _, v in _golden_rows("example2_lambdas.txt")]
    assert lam == [p["lambda1_hat"], p["lambda2_hat"]]


def test_results_do_not_depend_on_the_thread_count():
    # the OpenMP loops run subdomains and points independently: one thread
    # and all threads give the same bits (the host timing table uses both)
    K = fields.voronoi_field(64, n_sites=10, seed=18)
    p = oracle.default_params(k_top=10, levels=2)
    pts = np.random.default_rng(18).uniform(0, 1, size=(2000, 2))
    n_all = oracle.threads()
    try:
        oracle.threads(1)
        a = oracle.fit_all(K, (64, 64), (4, 4), 2, (4, 4), p)
        ea = oracle.evaluate(a, pts)
    finally:
        oracle.threads(n_all)
    b = oracle.fit_all(K, (64, 64), (4, 4), 2, (4, 4), p)
    for key in ("M", "c", "beta", "info"):
        np.testing.assert_array_equal(a[key], b[key])
    np.testing.assert_array_equal(ea, oracle.evaluate(b, pts))


@pytest.mark.parametrize("quad", [0, 1])
def test_error_measures_of_piecewise_constant_surrogates_in_closed_form(quad):
    # A surrogate with every coefficient of subdomain s equal to c_s is ln K* = c_s
    # on s's core (Shepard weights sum to one), whatever the centres. On a
    # hand-built K the four measures of the error reduction then have closed
    # forms over the cells each core owns: L1 = sum|K - e^c| / sum|K|,
    # L2 = sqrt(sum (K - e^c)^2 / sum K^2), the log-L1 = sum|ln K - c| / sum|ln K|
    # and the maximum of |ln K - c| / ln 10 over all cells. Every node of the
    # Gauss-Legendre rule sees the same constant, so quad = 1 gives the same
    # values. A dropped /ln 10, a maximum over one subdomain's cells only, or the
    # log-L1 normalised by sum|K| fails here.
    n_cells, n_sub = (12, 10), (3, 2)
    rng = np.random.default_rng(99)
    K = 10.0 ** rng.choice([-2.0, -0.5, 0.0, 1.0, 3.0], size=n_cells[::-1])  # K[j, i]
    boxes = oracle.partition(n_cells, n_sub, 0)
    S, m_cap = boxes.shape[0], 5
    c_s = np.log(np.array([0.3, 2.0, 7.0, 0.05, 40.0, 1.0]))
    cen = np.zeros((S, m_cap, 4))
    beta = np.zeros((S, m_cap))
    M = np.full(S, m_cap, dtype=np.int32)
    for s in range(S):
        cen[s, :, 0] = rng.uniform(0, 1, m_cap)
        cen[s, :, 1] = rng.uniform(0, 10 / 12, m_cap)
        cen[s, :, 3] = rng.uniform(0.05, 0.3, m_cap)
        beta[s, :] = c_s[s]
    model = dict(boxes=boxes, M=M, c=cen, beta=beta, m_cap=m_cap, n_cells=n_cells, n_sub=n_sub)
    lnKs = np.zeros(n_cells[::-1])
    for s in range(S):
        i0, j0, _, i1, j1, _ = boxes[s, :6]  # core box lo/hi (x, y, z)
        lnKs[j0:j1, i0:i1] = c_s[s]
    Ks = np.exp(lnKs)
    lk = np.log(K)
    want = dict(l1=np.abs(K - Ks).sum() / np.abs(K).sum(),
                l2=np.sqrt(((K - Ks) ** 2).sum() / (K ** 2).sum()),
                l1_log=np.abs(lk - lnKs).sum() / np.abs(lk).sum(),
                max_log10=np.abs(lk - lnKs).max() / np.log(10.0))
    got = oracle.errors(model, K, quad=quad)
    for key, v in want.items():
        assert got[key] == pytest.approx(v, rel=1e-13, abs=0), key
    # the maximum sits in one subdomain: it is not the first one's
    owner_max = np.unravel_index(np.argmax(np.abs(lk - lnKs)), lk.shape)
    assert not (owner_max[0] < boxes[0, 4] and owner_max[1] < boxes[0, 3])
