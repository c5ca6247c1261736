"""The seeded input generators against the workload recipes they stand for:
shapes and layout, value distributions and structure, measures of the
meshes, and bit-for-bit determinism per seed."""
import numpy as np
import pytest

from paper_2605_16564_gb300 import fields


def test_disc_field_is_the_disc_by_centroid():
    K = fields.disc_field(64)
    assert K.shape == (64, 64)
    x, y = np.meshgrid((np.arange(64) + 0.5) / 64, (np.arange(64) + 0.5) / 64, indexing="xy")
    np.testing.assert_array_equal(K, np.where((x - 0.5) ** 2 + (y - 0.5) ** 2 < 0.09, 1.0, 1e-3))


def test_voronoi_field_is_piecewise_constant_over_its_sites():
    K = fields.voronoi_field(256, n_sites=32, seed=2)
    assert K.shape == (256, 256)
    lk = np.log10(np.unique(K))
    assert 2 <= lk.size <= 32 and lk.min() >= -3 and lk.max() <= 3
    # the same sites at the cell centroids through voronoi_at
    pts = fields.cell_centred_points((256, 256), (1.0, 1.0))
    np.testing.assert_array_equal(fields.voronoi_at(pts, 32, 2), K.reshape(-1))


def test_channel_field_has_two_modes_six_decades_apart():
    K = fields.channel_field(1024, seed=3)
    assert K.shape == (1024, 1024)
    lk = np.log10(K)
    inside = lk > 1.5
    frac = inside.mean()
    assert 0.05 < frac < 0.6  # 12 channels of 8-24 cells across 1024 rows
    # background: 0.5 xi; channels: 3 + 0.5 xi (xi ~ N(0,1))
    assert abs(lk[~inside].mean()) < 0.05 and abs(lk[inside].mean() - 3.0) < 0.05
    assert lk.min() < -1.5 and lk.max() > 4.5


def test_layered_field_alternates_lognormal_and_binary_channel_layers():
    shape = (60, 220, 85)
    K = fields.layered_field(shape, seed=5)
    assert K.shape == (85, 220, 60)
    even = np.log10(K[0::2])
    assert abs(even.mean()) < 0.01 and abs(even.std() - 1.0) < 0.01
    odd = K[1::2]
    assert set(np.unique(odd)) == {1.0, 1e4}
    share = (odd == 1e4).mean(axis=(1, 2))
    assert share.min() > 0 and share.max() < 0.5
    # channels run along y: neighbouring rows (y) of a channel layer agree far
    # more often than neighbouring columns (x)
    along_y = (odd[:, 1:, :] == odd[:, :-1, :]).mean()
    along_x = (odd[:, :, 1:] == odd[:, :, :-1]).mean()
    assert along_y > along_x
    assert fields.layered_field(shape, seed=5).tobytes() == K.tobytes()


def test_patch_batch_mixes_three_kinds_clipped_to_six_decades():
    P = fields.patch_batch(300, seed=4)
    assert P.shape == (300, 32, 32)
    lk = np.log10(P)
    assert lk.min() >= -3 - 1e-12 and lk.max() <= 3 + 1e-12
    n_levels = np.array([np.unique(p).size for p in P])
    # discs: two values; channels: two values; Voronoi: up to 32 values
    assert np.all(n_levels[1::3] <= 2) and np.all(n_levels[2::3] <= 2)
    assert np.median(n_levels[0::3]) > 4
    np.testing.assert_array_equal(P, fields.patch_batch(300, seed=4))
    assert not np.array_equal(P, fields.patch_batch(300, seed=5))


@pytest.mark.parametrize("n,ny", [(16, None), (24, 10)])
def test_triangle_mesh_tiles_the_rectangle(n, ny):
    x, vol = fields.triangle_mesh(n, seed=3, ny=ny)
    ny = n if ny is None else ny
    h = 1.0 / max(n, ny)
    assert x.shape == (2 * n * ny, 2) and vol.shape == (2 * n * ny,)
    assert vol.sum() == pytest.approx(n * ny * h * h, rel=1e-14)
    # the two triangles of a square share it: their centroids average to its centre
    sq = x.reshape(ny, n, 2, 2).mean(axis=2)
    i, j = np.meshgrid(np.arange(n), np.arange(ny), indexing="xy")
    np.testing.assert_allclose(sq[..., 0], (i + 0.5) * h, rtol=0, atol=1e-15)
    np.testing.assert_allclose(sq[..., 1], (j + 0.5) * h, rtol=0, atol=1e-15)


@pytest.mark.parametrize("shape", [(40, 30), (12, 14, 8), (100,)])
def test_graded_mesh_measures_sum_to_the_box(shape):
    x, vol = fields.graded_mesh(shape, seed=9)
    h = fields.cell_size(shape)
    assert x.shape == (int(np.prod(shape)), len(shape))
    assert vol.sum() == pytest.approx(np.prod([n * h for n in shape]), rel=1e-12)
    assert vol.min() > 0
    for a, n in enumerate(shape):
        assert x[:, a].min() > 0 and x[:, a].max() < n * h


def test_grid_as_cells_orders_x_fastest():
    K = np.arange(6 * 4, dtype=float).reshape(4, 6) + 1.0  # numpy (n_y, n_x)
    x, vol, k = fields.grid_as_cells(K, (6, 4))
    h = 1.0 / 6
    np.testing.assert_array_equal(k, K.reshape(-1))
    np.testing.assert_allclose(x[7], [1.5 * h, 1.5 * h])
    assert np.all(vol == h * h)
