"""Host-side logic of the learned warm start's driver on CPU: the tiling of
a patch batch into one grid (patch p = px + T py at block (py, px), one
subdomain each), the network input and the seed's threshold."""
import numpy as np
import pytest

from paper_2605_16564_gb300 import fields, warmstart as ws


def test_tile_puts_patch_p_at_its_block():
    P = fields.patch_batch(9, seed=6)
    grid, T = ws.tile(P)
    assert T == 3 and grid.shape == (96, 96) and grid.flags["C_CONTIGUOUS"]
    for p in range(9):
        px, py = p % T, p // T
        np.testing.assert_array_equal(grid[py * 32:(py + 1) * 32, px * 32:(px + 1) * 32], P[p])
    with pytest.raises(AssertionError):
        ws.tile(P[:8])  # not a square number of patches


def test_tiled_patches_are_the_subdomains_of_the_grid():
    # the partition of the T x T tiling without overlap has the patches as
    # its subdomains, in the same order (subdomain s = px + T py)
    import oracle
    T = 4
    boxes = oracle.partition((T * 32, T * 32), (T, T), 0)
    for s in range(T * T):
        assert tuple(boxes[s, 0:2]) == ((s % T) * 32, (s // T) * 32)
        assert tuple(boxes[s, 3:5]) == ((s % T) * 32 + 32, (s // T) * 32 + 32)


def test_network_input_is_clipped_log10_over_three():
    P = np.array([[[1e-4, 1e-3], [1.0, 1e4]]])
    x = ws.network_input(P)
    assert x.dtype == np.float32
    np.testing.assert_allclose(x, [[[-1.0, -1.0], [0.0, 1.0]]], rtol=0, atol=1e-7)


def test_seed_keeps_the_large_predicted_coefficients():
    beta = np.array([[0.5, -3.5, 3.0, 4.0, -2.9]], dtype=np.float32)
    got = ws.warm_start_coefficients(np.zeros_like(beta), beta)
    np.testing.assert_array_equal(got, [[0.0, -3.5, 0.0, 4.0, 0.0]])
    assert got.dtype == np.float64
