"""Seeded synthetic cellwise-constant coefficient fields and target point sets.

This module only draws inputs: positive cell values K_T on a structured grid
and the points a surrogate is evaluated at. It holds none of the fitting
method's arithmetic (no basis functions, no regression, no refinement), so
both the CPU oracle tests and the CUDA path can take their inputs from it.

Grid convention (shared by every consumer of these arrays):
  * ``shape`` is (n_x, n_y, n_z) with unused trailing axes absent, e.g.
    (64, 64) for a 2-D grid;
  * the value array is C-ordered with the x index fastest, i.e. a 3-D field
    has numpy shape (n_z, n_y, n_x) and a 2-D field (n_y, n_x);
  * cells are isotropic squares/cubes of side h = 1 / max(shape), so a square
    grid covers exactly the unit square, and the centroid of cell (i, j, k)
    is ((i+1/2) h, (j+1/2) h, (k+1/2) h).

The fields stand in for the paper's permeability data (Case 1/2 of the
numerical experiments and the SPE10 slice), which are not available here:
they reproduce the kind of structure (sharp discs, Voronoi patches, thin
high-contrast channels, layered lognormal media) at the sizes of the
workloads, not the paper's actual values.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "cell_size", "numpy_shape", "disc_field", "voronoi_field", "channel_field",
    "layered_field", "patch_batch", "cell_centred_points", "step_field_1d",
    "grid_as_cells", "triangle_mesh", "graded_mesh", "voronoi_at", "cut_box",
]


def cell_size(shape) -> float:
    """Side h of the isotropic cells of a grid with ``shape`` = (n_x, ...)."""
    return 1.0 / float(max(shape))


def numpy_shape(shape):
    """numpy array shape for a grid (x fastest): (n_x,n_y,n_z) -> (n_z,n_y,n_x)."""
    return tuple(reversed(tuple(int(s) for s in shape)))


def _centroids(shape):
    """Per-axis centroid coordinate arrays broadcast to the field shape."""
    h = cell_size(shape)
    axes = [(np.arange(n) + 0.5) * h for n in shape]
    grids = np.meshgrid(*reversed(axes), indexing="ij")  # (z, y, x) order
    return list(reversed(grids))  # x, y, z


def disc_field(n: int = 64, radius: float = 0.3, centre=(0.5, 0.5),
               k_in: float = 1.0, k_out: float = 1e-3) -> np.ndarray:
    """2-D n x n field: k_in inside a disc, k_out outside (by cell centroid)."""
    x, y = _centroids((n, n))
    inside = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 < radius * radius
    return np.where(inside, k_in, k_out).astype(np.float64)


def voronoi_field(n: int = 256, n_sites: int = 32, seed: int = 2,
                  log10_range=(-3.0, 3.0)) -> np.ndarray:
    """2-D n x n Voronoi field.

    ``n_sites`` sites are drawn uniformly in the unit square and each site
    draws one log10 k uniformly from ``log10_range``; every cell takes the
    value of its nearest site (ties go to the lower site index).
    """
    rng = np.random.default_rng(seed)
    sites = rng.uniform(0.0, 1.0, size=(n_sites, 2))
    logk = rng.uniform(log10_range[0], log10_range[1], size=n_sites)
    x, y = _centroids((n, n))
    d2 = (x[..., None] - sites[:, 0]) ** 2 + (y[..., None] - sites[:, 1]) ** 2
    owner = np.argmin(d2, axis=-1)  # first minimum = lower index
    return (10.0 ** logk[owner]).astype(np.float64)


def channel_field(n: int = 1024, n_channels: int = 12, seed: int = 3,
                  contrast_log10: float = 3.0, noise_log10: float = 0.5,
                  width_cells=(8, 24)) -> np.ndarray:
    """2-D n x n channelised field.

    Each channel follows a sinusoidal centreline y = y0 + A sin(2 pi x / L + phi)
    with y0 ~ U[0,1], A ~ U[0.02,0.1], L ~ U[0.25,1], phi ~ U[0, 2 pi) and a
    width drawn uniformly from the integer range ``width_cells`` (in cells).
    log10 k = contrast * 1[in a channel] + noise * xi with xi ~ N(0,1) per cell,
    so k spans about six orders of magnitude for the defaults.
    """
    rng = np.random.default_rng(seed)
    h = cell_size((n, n))
    x, y = _centroids((n, n))
    inside = np.zeros((n, n), dtype=bool)
    for _ in range(n_channels):
        y0 = rng.uniform(0.0, 1.0)
        amp = rng.uniform(0.02, 0.1)
        wavelength = rng.uniform(0.25, 1.0)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        width = int(rng.integers(width_cells[0], width_cells[1] + 1)) * h
        centre = y0 + amp * np.sin(2.0 * np.pi * x / wavelength + phase)
        inside |= np.abs(y - centre) <= 0.5 * width
    xi = rng.standard_normal((n, n))
    logk = contrast_log10 * inside + noise_log10 * xi
    return (10.0 ** logk).astype(np.float64)


def layered_field(shape=(60, 220, 85), seed: int = 5, k_channel: float = 1e4,
                  k_background: float = 1.0, width_cells=(2, 6)) -> np.ndarray:
    """3-D layered field of grid ``shape`` = (n_x, n_y, n_z).

    Even z-layers are lognormal: log10 k ~ N(0,1) independently per cell.
    Odd z-layers are binary channel layers: 2-4 sinusoidal channels running
    along the y axis, each x = x0 + A sin(2 pi y / L + phi) with x0 ~ U[0, X],
    A ~ U[0.02, 0.1] X, L ~ U[0.25, 1] Y (X, Y the layer extents) and a width
    of 2-6 cells; k = ``k_channel`` in a channel and ``k_background`` outside
    (a contrast of 1e4 for the defaults).
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    h = cell_size(shape)
    X, Y = nx * h, ny * h
    xs = (np.arange(nx) + 0.5) * h
    ys = (np.arange(ny) + 0.5) * h
    xg, yg = np.meshgrid(xs, ys, indexing="xy")  # (ny, nx)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for k in range(nz):
        if k % 2 == 0:
            out[k] = 10.0 ** rng.standard_normal((ny, nx))
        else:
            inside = np.zeros((ny, nx), dtype=bool)
            for _ in range(int(rng.integers(2, 5))):
                x0 = rng.uniform(0.0, X)
                amp = rng.uniform(0.02, 0.1) * X
                wavelength = rng.uniform(0.25, 1.0) * Y
                phase = rng.uniform(0.0, 2.0 * np.pi)
                width = int(rng.integers(width_cells[0], width_cells[1] + 1)) * h
                centre = x0 + amp * np.sin(2.0 * np.pi * yg / wavelength + phase)
                inside |= np.abs(xg - centre) <= 0.5 * width
            out[k] = np.where(inside, k_channel, k_background)
    return out


def patch_batch(n_patches: int, size: int = 32, seed: int = 4) -> np.ndarray:
    """Batch of ``n_patches`` 2-D size x size fields, shape (P, size, size).

    A mixture, one third each (patch p takes kind p % 3): Voronoi patches
    with 8-32 sites and per-site log10 k ~ U[-3,3]; channel patches with 1-4
    sinusoidal channels of width 2-8 cells (channel log10 k ~ U[0,3],
    background ~ U[-3,0]); disc patches with a radius ~ U[0.15,0.45]
    (inside and outside log10 k each ~ U[-3,3]). log10 k is clipped to [-3,3].
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / size
    c = (np.arange(size) + 0.5) * h
    x, y = np.meshgrid(c, c, indexing="xy")
    out = np.empty((n_patches, size, size), dtype=np.float64)
    for p in range(n_patches):
        kind = p % 3
        if kind == 0:
            ns = int(rng.integers(8, 33))
            sites = rng.uniform(0.0, 1.0, size=(ns, 2))
            lk = rng.uniform(-3.0, 3.0, size=ns)
            d2 = (x[..., None] - sites[:, 0]) ** 2 + (y[..., None] - sites[:, 1]) ** 2
            logk = lk[np.argmin(d2, axis=-1)]
        elif kind == 1:
            inside = np.zeros((size, size), dtype=bool)
            for _ in range(int(rng.integers(1, 5))):
                y0 = rng.uniform(0.0, 1.0)
                amp = rng.uniform(0.02, 0.1)
                wavelength = rng.uniform(0.25, 1.0)
                phase = rng.uniform(0.0, 2.0 * np.pi)
                width = int(rng.integers(2, 9)) * h
                centre = y0 + amp * np.sin(2.0 * np.pi * x / wavelength + phase)
                inside |= np.abs(y - centre) <= 0.5 * width
            logk = np.where(inside, rng.uniform(0.0, 3.0), rng.uniform(-3.0, 0.0))
        else:
            r = rng.uniform(0.15, 0.45)
            cx, cy = rng.uniform(0.2, 0.8, size=2)
            inside = (x - cx) ** 2 + (y - cy) ** 2 < r * r
            logk = np.where(inside, rng.uniform(-3.0, 3.0), rng.uniform(-3.0, 3.0))
        out[p] = 10.0 ** np.clip(logk, -3.0, 3.0)
    return out


def step_field_1d(n: int, x0_cells: int, k_left: float = 1e-4,
                  k_right: float = 1e-1) -> np.ndarray:
    """1-D field of n cells: k_left on cells [0, x0_cells), k_right after."""
    out = np.full(n, k_left, dtype=np.float64)
    out[x0_cells:] = k_right
    return out


def cell_centred_points(counts, extent) -> np.ndarray:
    """Centres of a counts[0] x counts[1] x ... mesh over [0, extent[a]].

    Returns an (n, d) float64 array, x fastest, used as a non-matching target
    mesh (e.g. a 97 x 97 mesh over the unit square, or the 2x refined mesh of
    a 3-D grid).
    """
    axes = [(np.arange(c) + 0.5) * (e / c) for c, e in zip(counts, extent)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    cols = [g.reshape(-1) for g in reversed(grids)]
    return np.stack(cols, axis=1).astype(np.float64)


# --------------------------------------------------------------------------
# General meshes given as cells: per element its sampling point x_T (the
# centroid), its measure |T| and its value K_T, in a flat element order.
# --------------------------------------------------------------------------

def grid_as_cells(K: np.ndarray, shape):
    """The cells of a structured grid field as a cell list in global order
    (x fastest): (x [n, dim] centroids, vol [n] = h^dim, K [n])."""
    dim = len(shape)
    h = cell_size(shape)
    axes = [(np.arange(n) + 0.5) * h for n in shape]  # (i + 1/2) h, as the grid path forms them
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    x = np.stack([g.reshape(-1) for g in reversed(grids)], axis=1)
    vol = np.full(x.shape[0], h ** dim)
    return x, vol, np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(-1))


def voronoi_at(points: np.ndarray, n_sites: int = 32, seed: int = 2, log10_range=(-3.0, 3.0)) -> np.ndarray:
    """The Voronoi field of voronoi_field (same sites and values for the same
    seed) evaluated at arbitrary 2-D points [n, 2]."""
    rng = np.random.default_rng(seed)
    sites = rng.uniform(0.0, 1.0, size=(n_sites, 2))
    logk = rng.uniform(log10_range[0], log10_range[1], size=n_sites)
    p = np.asarray(points, dtype=np.float64)
    d2 = (p[:, 0:1] - sites[:, 0]) ** 2 + (p[:, 1:2] - sites[:, 1]) ** 2
    return (10.0 ** logk[np.argmin(d2, axis=1)]).astype(np.float64)


def triangle_mesh(n: int, seed: int = 11, ny: int | None = None):
    """Unstructured 2-D triangle mesh of the rectangle [0, n h] x [0, ny h]
    (h = 1 / max(n, ny)): every grid square is cut along one of its two
    diagonals, chosen at random per square, into two triangles of area h^2/2.
    Returns (x [2 n ny, 2] triangle centroids, vol [2 n ny]) in square order
    (x fastest), the two triangles of a square consecutive."""
    ny = n if ny is None else ny
    h = 1.0 / max(n, ny)
    rng = np.random.default_rng(seed)
    diag = rng.integers(0, 2, size=(ny, n))
    i = np.arange(n)[None, :].repeat(ny, 0)
    j = np.arange(ny)[:, None].repeat(n, 1)
    # diagonal 0 joins (i, j)-(i+1, j+1): centroids (i+2/3, j+1/3), (i+1/3, j+2/3)
    # diagonal 1 joins (i+1, j)-(i, j+1): centroids (i+1/3, j+1/3), (i+2/3, j+2/3)
    a = np.where(diag == 0, 2.0, 1.0) / 3.0
    b = np.where(diag == 0, 1.0, 2.0) / 3.0
    t0 = np.stack([(i + a) * h, (j + 1.0 / 3.0) * h], -1)
    t1 = np.stack([(i + b) * h, (j + 2.0 / 3.0) * h], -1)
    x = np.stack([t0, t1], axis=2).reshape(-1, 2)
    vol = np.full(x.shape[0], 0.5 * h * h)
    return x, vol


def graded_mesh(shape, seed: int = 12, ratio: float = 3.0):
    """Non-uniform tensor mesh of the box [0, n_a h]: along each axis the n_a
    cell widths are drawn from a seeded log-uniform law spanning ``ratio``
    and rescaled to the axis length. Returns (x [n, dim] cell centroids,
    vol [n] cell volumes) in x-fastest order."""
    rng = np.random.default_rng(seed)
    h = cell_size(shape)
    edges = []
    for n in shape:
        w = np.exp(rng.uniform(0.0, np.log(ratio), size=n))
        w *= n * h / w.sum()
        e = np.concatenate([[0.0], np.cumsum(w)])
        e[-1] = n * h
        edges.append(e)
    mids = [0.5 * (e[1:] + e[:-1]) for e in edges]
    widths = [e[1:] - e[:-1] for e in edges]
    grids = np.meshgrid(*reversed(mids), indexing="ij")
    wgrid = np.meshgrid(*reversed(widths), indexing="ij")
    x = np.stack([g.reshape(-1) for g in reversed(grids)], axis=1)
    vol = np.prod(np.stack([g.reshape(-1) for g in wgrid], axis=1), axis=1)
    return x, vol


def cut_box(x: np.ndarray, vol: np.ndarray, lo, hi):
    """The mesh (x, vol) without the elements whose sampling point lies in the
    open box (lo, hi): a domain with a rectangular hole."""
    x = np.asarray(x)
    inside = np.all((x > np.asarray(lo)) & (x < np.asarray(hi)), axis=1)
    return np.ascontiguousarray(x[~inside]), np.ascontiguousarray(np.asarray(vol)[~inside])
