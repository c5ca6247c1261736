"""FP64 CPU oracle for the PAM fitting path -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never imports, links or calls anything here, and the two
share no code.

The arithmetic lives in ``pam_oracle.c`` (plain C, binary64, no fused
multiply-add); this module compiles it with gcc on first use and wraps each
function with numpy marshalling. Which paper passage each function follows is
stated beside it in the C source. ``cv_lambda`` composes those primitives in
a plain Python loop (its residual dot products in numpy).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pam_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpam_oracle.so")
_lock = threading.Lock()
_lib = None

NINFO = 8  # per-subdomain diagnostics, see orc_fit_subdomain


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            L.orc_partition.argtypes = [C.c_int, i32p, i32p, C.c_int, i32p]
            L.orc_partition.restype = C.c_int
            L.orc_box_cells.argtypes = [C.c_int, i32p, i32p, i32p, f64p, f64p, f64p, f64p]
            L.orc_box_cells.restype = C.c_int64
            L.orc_initial_dictionary.argtypes = [C.c_int, i32p, i32p, i32p, i32p, f64p]
            L.orc_initial_dictionary.restype = C.c_int
            L.orc_assemble.argtypes = [C.c_int, C.c_int64, f64p, C.c_int, f64p, f64p]
            L.orc_assemble.restype = None
            L.orc_gram.argtypes = [C.c_int64, C.c_int, f64p, f64p, f64p, f64p]
            L.orc_gram.restype = None
            L.orc_enet.argtypes = [C.c_int, f64p, f64p, C.c_double, C.c_double, f64p,
                                   C.c_int, f64p]
            L.orc_enet.restype = C.c_int
            L.orc_enet_objective.argtypes = [C.c_int, f64p, f64p, C.c_double, C.c_double,
                                             C.c_double, f64p]
            L.orc_enet_objective.restype = C.c_double
            L.orc_residual.argtypes = [C.c_int64, C.c_int, f64p, f64p, f64p, C.c_double, f64p]
            L.orc_residual.restype = None
            L.orc_mark.argtypes = [C.c_int64, f64p, C.c_double, C.c_int, i32p]
            L.orc_mark.restype = C.c_int
            L.orc_enrich.argtypes = [C.c_int, C.c_int, f64p, C.c_int, i32p, f64p, f64p,
                                     f64p, C.c_double, C.c_int]
            L.orc_enrich.restype = C.c_int
            L.orc_fit_all.argtypes = [C.c_int, i32p, f64p, C.c_int, i32p, i32p,
                                      C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                      f64p, f64p, f64p]
            L.orc_fit_all.restype = C.c_int
            L.orc_eval.argtypes = [C.c_int, i32p, i32p, C.c_int, i32p, f64p, f64p,
                                   C.c_int64, f64p, C.c_int, f64p, C.c_void_p]
            L.orc_eval.restype = None
            L.orc_errors.argtypes = [C.c_int, i32p, i32p, C.c_int, i32p, f64p, f64p,
                                     f64p, C.c_int, f64p]
            L.orc_errors.restype = None
            L.orc_gl_points.argtypes = [C.c_int, f64p, C.c_double, f64p]
            L.orc_gl_points.restype = None
            L.orc_residual_gl.argtypes = [C.c_int, C.c_int64, f64p, C.c_int, f64p, f64p, f64p, C.c_double,
                                          C.c_double, f64p]
            L.orc_residual_gl.restype = None
            L.orc_residual_cells.argtypes = [C.c_int64, C.c_int, f64p, f64p, f64p, f64p, f64p]
            L.orc_residual_cells.restype = None
            L.orc_mark_cells.argtypes = [C.c_int64, f64p, f64p, C.c_int, i32p]
            L.orc_mark_cells.restype = C.c_int
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            L.orc_fit_cells_all.argtypes = [C.c_int, i32p, f64p, f64p, f64p, C.c_int, i32p, i64p, i32p, i32p,
                                            C.c_void_p, C.c_int, C.c_void_p, C.c_int, f64p, f64p, f64p]
            L.orc_fit_cells_all.restype = C.c_int
            L.orc_threads.argtypes = [C.c_int]
            L.orc_threads.restype = C.c_int
            _lib = L
    return _lib


def threads(n=0):
    """OpenMP threads of the oracle's loops (n > 0 sets them); returns the
    count in effect. Timing only: the results do not depend on it."""
    return int(lib().orc_threads(int(n)))


class _Params(C.Structure):
    _fields_ = [("lambda1_hat", C.c_double), ("lambda2_hat", C.c_double),
                ("eps_tol_rel", C.c_double), ("eta", C.c_double),
                ("k_top", C.c_int), ("m_max", C.c_int), ("levels", C.c_int),
                ("max_sweeps", C.c_int), ("quad", C.c_int)]


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _pad3(v, fill):
    v = list(v)
    return _i32(v + [fill] * (3 - len(v)))


# --------------------------------------------------------------------------
# Step 1
# --------------------------------------------------------------------------

def partition(n_cells, n_sub, overlap=0):
    """Core/patch boxes, int32 [S, 12] (core_lo, core_hi, patch_lo, patch_hi)."""
    dim = len(n_cells)
    S = int(np.prod(n_sub))
    boxes = np.zeros((S, 12), dtype=np.int32)
    lib().orc_partition(dim, _pad3(n_cells, 1), _pad3(n_sub, 1), int(overlap), boxes)
    return boxes


def box_cells(n_cells, lo, hi, K):
    """(x [N,3], y = ln K [N], K [N]) of the cells of box [lo, hi), x fastest."""
    dim = len(n_cells)
    lo, hi = _pad3(list(lo)[:3], 0), _pad3(list(hi)[:3], 1)
    N = int(np.prod(hi - lo))
    x = np.zeros((N, 3)); y = np.zeros(N); kv = np.zeros(N)
    lib().orc_box_cells(dim, _pad3(n_cells, 1), lo, hi, _f64(K).reshape(-1), x, y, kv)
    return x, y, kv


def initial_dictionary(n_cells, core_lo, core_hi, g):
    """Uniform cell-centred lattice over the core box: [M, 4] = (c, sigma)."""
    dim = len(n_cells)
    M = int(np.prod(g))
    c = np.zeros((M, 4))
    lib().orc_initial_dictionary(dim, _pad3(n_cells, 1), _pad3(list(core_lo)[:3], 0),
                                 _pad3(list(core_hi)[:3], 1), _pad3(g, 1), c)
    return c


# --------------------------------------------------------------------------
# Step 2
# --------------------------------------------------------------------------

def assemble(dim, x, c):
    """Shepard-normalised feature matrix W [N, M] (x: [N,3] or [N,dim])."""
    x = _f64(x)
    if x.shape[1] != 3:
        x = _f64(np.concatenate([x, np.zeros((x.shape[0], 3 - x.shape[1]))], axis=1))
    c = _f64(c)
    W = np.zeros((x.shape[0], c.shape[0]))
    lib().orc_assemble(dim, x.shape[0], x, c.shape[0], c, W)
    return W


def gram(W, y):
    W = _f64(W); y = _f64(y)
    n, m = W.shape
    G = np.zeros((m, m)); b = np.zeros(m)
    lib().orc_gram(n, m, W, y, G, b)
    return G, b


def enet(G, b, lam1, lam2, beta0=None, max_sweeps=200000):
    """Elastic Net minimiser of Eq. (2) given G = W^T W, b = W^T y.

    Returns (beta, info) with info = dict(sweeps, attempts, margin,
    certified, support).
    """
    G = _f64(G); b = _f64(b)
    m = b.shape[0]
    beta = np.zeros(m) if beta0 is None else _f64(beta0).copy()
    info = np.zeros(5)
    lib().orc_enet(m, G, b, float(lam1), float(lam2), beta, int(max_sweeps), info)
    return beta, dict(sweeps=int(info[0]), attempts=int(info[1]), margin=float(info[2]),
                      certified=bool(info[3]), support=int(info[4]))


def enet_objective(G, b, yty, lam1, lam2, beta):
    return lib().orc_enet_objective(b.shape[0], _f64(G), _f64(b), float(yty), float(lam1),
                                    float(lam2), _f64(beta))


# --------------------------------------------------------------------------
# Step 3
# --------------------------------------------------------------------------

def residual(W, beta, kv, vol):
    W = _f64(W)
    R = np.zeros(W.shape[0])
    lib().orc_residual(W.shape[0], W.shape[1], W, _f64(beta), _f64(kv), float(vol), R)
    return R


def mark(R, eps_tol, k_top):
    R = _f64(R)
    out = np.zeros(max(int(k_top), 1), dtype=np.int32)
    n = lib().orc_mark(R.shape[0], R, float(eps_tol), int(k_top), out)
    return out[:n].copy()


def residual_cells(W, beta, kv, vol):
    """R_T = |T| (exp(W beta)_T - K_T)^2 with a measure per cell."""
    W = _f64(W)
    R = np.zeros(W.shape[0])
    lib().orc_residual_cells(W.shape[0], W.shape[1], W, _f64(beta), _f64(kv), _f64(vol), R)
    return R


def mark_cells(R, eps_cell, k_top):
    """Marking with a threshold per cell."""
    R = _f64(R)
    out = np.zeros(max(int(k_top), 1), dtype=np.int32)
    n = lib().orc_mark_cells(R.shape[0], R, _f64(eps_cell), int(k_top), out)
    return out[:n].copy()


def enrich(dim, c, marked, x, ext_lo, ext_hi, eta, m_limit):
    """Append the new centres of the marked cells; returns the grown [M', 4]."""
    c = _f64(c)
    m = c.shape[0]
    cap = max(int(m_limit), m)
    buf = np.zeros((cap, 4))
    buf[:m] = c
    x = _f64(x)
    if x.shape[1] != 3:
        x = _f64(np.concatenate([x, np.zeros((x.shape[0], 3 - x.shape[1]))], axis=1))
    lo = _f64(list(ext_lo) + [0.0] * (3 - len(ext_lo)))
    hi = _f64(list(ext_hi) + [0.0] * (3 - len(ext_hi)))
    mk = _i32(marked)
    mm = lib().orc_enrich(dim, m, buf, mk.shape[0], mk, x, lo, hi, float(eta), cap)
    return buf[:mm].copy()


# --------------------------------------------------------------------------
# Algorithm 1 on all subdomains, and Step 4
# --------------------------------------------------------------------------

def default_params(**kw):
    p = dict(lambda1_hat=4.59e-4, lambda2_hat=4.64e-6, eps_tol_rel=1e-3, eta=0.5,
             k_top=37, m_max=1 << 30, levels=3, max_sweeps=200000, quad=0)
    p.update(kw)
    return p


def m_capacity(g, dim, k_top, levels, m_max):
    m0 = int(np.prod(g))
    return int(min(m0 + levels * (dim + 1) * k_top, m0 + m_max))


def fit_all(K, n_cells, n_sub, overlap, g, params, which=None, m_cap=None):
    """Algorithm 1 on every subdomain (or the subset ``which``).

    Returns dict(boxes, M, c [S, m_cap, 4], beta [S, m_cap], info [S, NINFO],
    m_cap, failed). Subdomains not in ``which`` are left empty (M = 0).
    """
    dim = len(n_cells)
    boxes = partition(n_cells, n_sub, overlap)
    S = boxes.shape[0]
    P = _Params(**{k: params[k] for k, _ in _Params._fields_})
    if m_cap is None:
        m_cap = m_capacity(g, dim, params["k_top"], params["levels"], params["m_max"])
    c = np.zeros((S, m_cap, 4)); beta = np.zeros((S, m_cap)); info = np.zeros((S, NINFO))
    wh = None if which is None else _i32(which)
    failed = lib().orc_fit_all(dim, _pad3(n_cells, 1), _f64(K).reshape(-1), S, boxes,
                               _pad3(g, 1), C.byref(P), int(m_cap),
                               None if wh is None else wh.ctypes.data, 0 if wh is None else wh.shape[0],
                               c, beta, info)
    M = info[:, 0].astype(np.int32)
    return dict(boxes=boxes, M=M, c=c, beta=beta, info=info, m_cap=int(m_cap), failed=int(failed),
                n_cells=tuple(n_cells), n_sub=tuple(n_sub))


def evaluate(model, pts, log_space=False, return_owner=False):
    """K*(x) (or its log) at points [n, dim] from a fitted model (Step 4)."""
    n_cells, n_sub = model["n_cells"], model["n_sub"]
    dim = len(n_cells)
    pts = _f64(pts).reshape(-1, dim)
    out = np.zeros(pts.shape[0])
    own = np.zeros(pts.shape[0], dtype=np.int32)
    lib().orc_eval(dim, _pad3(n_cells, 1), _pad3(n_sub, 1), int(model["m_cap"]), _i32(model["M"]),
                   _f64(model["c"]), _f64(model["beta"]), pts.shape[0], pts, int(bool(log_space)),
                   out, own.ctypes.data)
    return (out, own) if return_owner else out


def errors(model, K, quad=0):
    """dict(l1, l2, l1_log, max_log10) of the reconstruction over the source cells
    (quad 0: midpoint rule, 1: 2^dim-point Gauss-Legendre rule per cell)."""
    n_cells, n_sub = model["n_cells"], model["n_sub"]
    dim = len(n_cells)
    err = np.zeros(4)
    lib().orc_errors(dim, _pad3(n_cells, 1), _pad3(n_sub, 1), int(model["m_cap"]), _i32(model["M"]),
                     _f64(model["c"]), _f64(model["beta"]), _f64(K).reshape(-1), int(quad), err)
    return dict(l1=err[0], l2=err[1], l1_log=err[2], max_log10=err[3])


def gl_points(x, h):
    """The 2^dim Gauss-Legendre nodes of the cell of side h centred at x [dim]."""
    x = _f64(x).reshape(-1)
    dim = x.shape[0]
    pts = np.zeros(((1 << dim), dim))
    lib().orc_gl_points(dim, x, float(h), pts)
    return pts


def residual_gl(x, c, beta, kv, vol, h, dim):
    """Eq. (4) with the Gauss-Legendre rule for cells x [n, 3] (padded), dictionary c [m, 4]."""
    x = _f64(x).reshape(-1, 3)
    n, m = x.shape[0], int(c.shape[0])
    R = np.zeros(n)
    lib().orc_residual_gl(dim, n, x, m, _f64(c), _f64(beta), _f64(kv), float(vol), float(h), R)
    return R


# --------------------------------------------------------------------------
# Per-subdomain choice of the Elastic Net weights (section 5, Experiment 1.2:
# lambda is chosen independently on each subdomain; the rule is not stated).
# Reading: k-fold cross-validation over a caller-given grid of
# (lambda1_hat, lambda2_hat) pairs on the subdomain's final dictionary.
# --------------------------------------------------------------------------

def cv_lambda(model, K, grid, n_folds, which=None):
    """For each subdomain: cell t of the patch (local row-major index) is in
    fold t mod n_folds; for every grid pair and fold the Elastic Net (Eq. (2),
    lambda_k = N_train lambda_k_hat) is solved on the other folds' cells and
    its squared log-residuals y_t - (W beta)_t on the held-out cells summed;
    cv = that sum over all folds / N. choice = first grid index of least cv;
    the coefficients are then refit on all N cells with the chosen pair.

    Returns dict(cv [S, n_grid], choice [S], beta [S, m_cap], certified [S]).
    Subdomains not in ``which`` are skipped (cv NaN, choice -1).
    """
    n_cells = tuple(model["n_cells"])
    dim = len(n_cells)
    boxes = model["boxes"]
    S, mc = boxes.shape[0], int(model["m_cap"])
    grid = np.asarray(grid, dtype=np.float64).reshape(-1, 2)
    cv = np.full((S, grid.shape[0]), np.nan)
    choice = np.full(S, -1, dtype=np.int32)
    beta = np.zeros((S, mc))
    certified = np.zeros(S, dtype=bool)
    for s in (range(S) if which is None else which):
        x, y, _ = box_cells(n_cells, boxes[s, 6:9], boxes[s, 9:12], K)
        M = int(model["M"][s])
        W = assemble(dim, x, model["c"][s, :M])
        N = y.shape[0]
        fold = np.arange(N) % n_folds
        for gi, (l1h, l2h) in enumerate(grid):
            total = 0.0
            for f in range(n_folds):
                train = fold != f
                n_tr = int(train.sum())
                G, b = gram(W[train], y[train])
                bf, _ = enet(G, b, n_tr * l1h, n_tr * l2h)
                r = y[~train] - W[~train] @ bf
                total += float(r @ r)
            cv[s, gi] = total / N
        choice[s] = int(np.argmin(cv[s]))
        l1h, l2h = grid[choice[s]]
        G, b = gram(W, y)
        bs, inf = enet(G, b, N * l1h, N * l2h)
        beta[s, :M] = bs
        certified[s] = inf["certified"]
    return dict(cv=cv, choice=choice, beta=beta, certified=certified)


# --------------------------------------------------------------------------
# Interface gluing (Step 4 remark: the piecewise K* is discontinuous across
# subdomain interfaces; a gluing or averaging across neighbours makes it
# continuous; the paper leaves the procedure open). Reading: the local
# log-surrogates u_i = sum_m beta_m w_m are blended with a tensor-product
# partition of unity that ramps across each interior core face over a band
# of half-width delta = band * h:
#   psi_i(x) = prod_a phi_lo(x_a) phi_hi(x_a),
#   phi_lo = r((x_a - lo_a + delta) / (2 delta)) (1 on the outer face),
#   phi_hi = r((hi_a + delta - x_a) / (2 delta)) (1 on the outer face),
#   r(t) = t^2 (3 - 2 t) on [0, 1] (clamped), so r(t) + r(1 - t) = 1,
#   ln K*(x) = sum_i psi_i u_i / sum_i psi_i.
# --------------------------------------------------------------------------

def _smoothstep(t):
    t = np.clip(t, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def glue_weights(n_cells, n_sub, pts, band):
    """psi_i(x) of every subdomain at points [n, dim]: [n, S] (brute force
    over all subdomains; points outside the domain get 0)."""
    n_cells = tuple(n_cells)
    dim = len(n_cells)
    pts = _f64(pts).reshape(-1, dim)
    h = 1.0 / max(n_cells)
    delta = band * h
    boxes = partition(n_cells, n_sub, 0)
    psi = np.ones((pts.shape[0], boxes.shape[0]))
    for s in range(boxes.shape[0]):
        for a in range(dim):
            lo, hi = boxes[s, a], boxes[s, 3 + a]
            xa = pts[:, a]
            if lo > 0:
                psi[:, s] *= _smoothstep((xa - lo * h + delta) / (2.0 * delta))
            if hi < n_cells[a]:
                psi[:, s] *= _smoothstep((hi * h + delta - xa) / (2.0 * delta))
    inside = np.all((pts >= 0.0) & (pts <= np.asarray(n_cells) * h), axis=1)
    psi[~inside] = 0.0
    return psi


def evaluate_glued(model, pts, band, log_space=False):
    """Glued K*(x) (or its log) at points [n, dim]; NaN outside the domain."""
    n_cells, n_sub = tuple(model["n_cells"]), tuple(model["n_sub"])
    dim = len(n_cells)
    pts = _f64(pts).reshape(-1, dim)
    psi = glue_weights(n_cells, n_sub, pts, band)
    num = np.zeros(pts.shape[0])
    for s in range(psi.shape[1]):
        sel = np.flatnonzero(psi[:, s] > 0.0)
        if sel.size == 0:
            continue
        M = int(model["M"][s])
        u = assemble(dim, pts[sel], model["c"][s, :M]) @ model["beta"][s, :M]
        num[sel] += psi[sel, s] * u
    den = psi.sum(axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = np.where(den > 0.0, num / den, np.nan)
    return v if log_space else np.exp(v)


# --------------------------------------------------------------------------
# General (unstructured) meshes given as cells (section 2: elements T of a
# shape-regular partition, e.g. intervals, triangles or quadrilaterals, each
# with a sampling point x_T in T, its value K_T and its measure |T|).
# Reading: the subdomains are the boxes of the lattice decomposition of the
# problem (cores [floor(j n / p) h, floor((j+1) n / p) h) per axis, h =
# 1 / max n); an element belongs to the core holding its sampling point (the
# owner rule of Step 4, so every element is in exactly one core and each
# subdomain is a union of elements), and to the patch of every subdomain
# whose core grown by `overlap` h holds its point (closed at the outer face
# of the domain). A patch's local order is ascending element index.
# --------------------------------------------------------------------------

def partition_cells(n_cells, n_sub, overlap, x):
    """(boxes [S, 12], patch_start int64 [S+1], patch_cells int32 [...]) for
    elements with sampling points x [n, dim] (brute force over subdomains)."""
    n_cells = tuple(n_cells)
    dim = len(n_cells)
    x = _f64(x).reshape(-1, dim)
    nmax = max(n_cells)
    u = x * float(nmax)
    boxes = partition(n_cells, n_sub, overlap)
    lists = []
    for s in range(boxes.shape[0]):
        ok = np.ones(x.shape[0], dtype=bool)
        for a in range(dim):
            lo, hi = boxes[s, 6 + a], boxes[s, 9 + a]
            upper = (u[:, a] <= hi) if hi == n_cells[a] else (u[:, a] < hi)
            ok &= (u[:, a] >= lo) & upper
        lists.append(np.flatnonzero(ok).astype(np.int32))
    start = np.zeros(len(lists) + 1, dtype=np.int64)
    start[1:] = np.cumsum([len(v) for v in lists])
    cells = np.concatenate(lists) if lists else np.zeros(0, dtype=np.int32)
    return boxes, start, _i32(cells)


def fit_cells(x, vol, K, n_cells, n_sub, overlap, g, params, which=None, m_cap=None):
    """Algorithm 1 on every subdomain of a mesh given as cells (the subset
    ``which`` if given). Returns the model dict of fit_all plus the patch
    lists (patch_start, patch_cells)."""
    n_cells = tuple(n_cells)
    dim = len(n_cells)
    x = _f64(x).reshape(-1, dim)
    boxes, start, cells = partition_cells(n_cells, n_sub, overlap, x)
    S = boxes.shape[0]
    P = _Params(**{k: params[k] for k, _ in _Params._fields_})
    P.quad = 0
    if m_cap is None:
        m_cap = m_capacity(g, dim, params["k_top"], params["levels"], params["m_max"])
    c = np.zeros((S, m_cap, 4)); beta = np.zeros((S, m_cap)); info = np.zeros((S, NINFO))
    wh = None if which is None else _i32(which)
    failed = lib().orc_fit_cells_all(dim, _pad3(n_cells, 1), x, _f64(K).reshape(-1), _f64(vol).reshape(-1), S,
                                     boxes, start, cells if cells.size else np.zeros(1, dtype=np.int32),
                                     _pad3(g, 1), C.byref(P), int(m_cap),
                                     None if wh is None else wh.ctypes.data, 0 if wh is None else wh.shape[0],
                                     c, beta, info)
    M = info[:, 0].astype(np.int32)
    return dict(boxes=boxes, M=M, c=c, beta=beta, info=info, m_cap=int(m_cap), failed=int(failed),
                n_cells=n_cells, n_sub=tuple(n_sub), patch_start=start, patch_cells=cells)


def errors_cells(model, x, vol, K):
    """Relative errors over the elements, each measured with its owner's
    surrogate at its sampling point (midpoint rule, weight |T|):
    l1 = sum |T| |K_T - K*| / sum |T| |K_T|, l2 = (sum |T| (K_T - K*)^2 /
    sum |T| K_T^2)^(1/2) (Eq. (12)), l1_log = sum |T| |ln K_T - ln K*| /
    sum |T| |ln K_T|, max_log10 = max |log10 K_T - log10 K*|."""
    dim = len(model["n_cells"])
    x = _f64(x).reshape(-1, dim)
    v = evaluate(model, x, log_space=True)
    K = _f64(K).reshape(-1)
    vol = _f64(vol).reshape(-1)
    lk = np.log(K)
    ks = np.exp(v)
    l1 = np.sum(vol * np.abs(K - ks)) / np.sum(vol * np.abs(K))
    l2 = np.sqrt(np.sum(vol * (K - ks) ** 2) / np.sum(vol * K * K))
    bl = np.sum(vol * np.abs(lk))
    l1l = np.sum(vol * np.abs(lk - v)) / bl if bl > 0 else np.sum(vol * np.abs(lk - v))
    return dict(l1=float(l1), l2=float(l2), l1_log=float(l1l),
                max_log10=float(np.max(np.abs(lk - v)) / np.log(10.0)))
