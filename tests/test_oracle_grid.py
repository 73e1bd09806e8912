"""Pins of the grid-epilogue oracle (Gaussian smoothing, Sec. III-B; max-union
of several humans, Sec. IV-B) against closed forms and brute force."""
import math

import numpy as np
import pytest

from oracle import grid_ops as G


@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.7, 3.0])
def test_taps_are_the_normalised_truncated_gaussian(sigma):
    R, w = G.gaussian_taps(sigma)
    assert R == math.ceil(3 * sigma)
    assert w.shape == (2 * R + 1,)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w[::-1], rtol=0, atol=0)
    # successive ratios of exp(-i^2 / 2 sigma^2): w_{i+1} / w_i = exp(-(2i + 1) / (2 sigma^2))
    for i in range(R):
        assert w[R + i + 1] / w[R + i] == pytest.approx(math.exp(-(2 * i + 1) / (2 * sigma * sigma)), rel=1e-13)


def test_sigma_zero_is_normalisation_only():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 50, size=(3, 7, 5))
    assert np.array_equal(G.smooth(c, 400, 0.0), c / 400.0)


def test_impulse_gives_the_outer_product_of_the_taps():
    """A lone cell of mass N (away from the edges) spreads as w_y[i] * w_x[j];
    a non-square grid and an off-centre cell catch a transposed axis."""
    sigma = 1.3
    R, w = G.gaussian_taps(sigma)
    c = np.zeros((2, 17, 23), np.int64)
    c[1, 6, 14] = 1000
    s = G.smooth(c, 1000, sigma, pad=0)
    want = np.zeros((17, 23))
    want[6 - R:6 + R + 1, 14 - R:14 + R + 1] = np.outer(w, w)
    assert np.allclose(s[1], want, rtol=0, atol=1e-15)
    assert np.all(s[0] == 0)
    assert s[1].sum() == pytest.approx(1.0, abs=1e-14)


def test_mass_past_the_edge_is_dropped_unless_padded():
    sigma = 1.0
    R, w = G.gaussian_taps(sigma)
    c = np.zeros((1, 9, 9), np.int64)
    c[0, 0, 0] = 10
    inside = G.smooth(c, 10, sigma, pad=0)[0].sum()
    assert inside == pytest.approx(w[R:].sum() ** 2, rel=1e-13)
    assert G.smooth(c, 10, sigma)[0].sum() == pytest.approx(1.0, rel=1e-13)


def test_separable_blur_equals_direct_2d_convolution():
    """Brute force: every output cell as a double sum over the 2-D kernel."""
    sigma = 0.8
    R, w = G.gaussian_taps(sigma)
    rng = np.random.default_rng(11)
    c = rng.integers(0, 9, size=(1, 6, 8))
    s = G.smooth(c, 37, sigma, pad=R)[0]
    H, W = 6, 8
    for y in range(H + 2 * R):
        for x in range(W + 2 * R):
            acc = 0.0
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    yy, xx = y - R + dy, x - R + dx
                    if 0 <= yy < H and 0 <= xx < W:
                        acc += w[dy + R] * w[dx + R] * c[0, yy, xx] / 37.0
            assert s[y, x] == pytest.approx(acc, rel=1e-12, abs=1e-17)


def test_union_places_takes_max_and_respects_horizons():
    rng = np.random.default_rng(5)
    sigma = 0.9
    R, _ = G.gaussian_taps(sigma)
    a = rng.integers(0, 30, size=(4, 5, 6))
    b = rng.integers(0, 30, size=(2, 5, 6))
    H, W, T = 20, 24, 4
    out = G.union([dict(counts=a, n=500, offset=(3, 7)), dict(counts=b, n=300, offset=(9, 4))], T, H, W, sigma)
    sa = G.smooth(a, 500, sigma)  # window + R on each side
    sb = G.smooth(b, 300, sigma)
    pa = np.zeros((T, H, W))
    pa[:, 7 - R:7 + 5 + R, 3 - R:3 + 6 + R] = sa
    pb = np.zeros((T, H, W))
    pb[:2, 4 - R:4 + 5 + R, 9 - R:9 + 6 + R] = sb
    assert np.array_equal(out, np.maximum(pa, pb))
    # one human alone, offset 0, no blur: the normalised counts
    one = G.union([dict(counts=a, n=500, offset=(0, 0))], 4, 5, 6, 0.0)
    assert np.array_equal(one, a / 500.0)
    # identical humans: the same grid
    two = G.union([dict(counts=a, n=500, offset=(0, 0))] * 2, 4, 5, 6, sigma)
    assert np.array_equal(two, G.union([dict(counts=a, n=500, offset=(0, 0))], 4, 5, 6, sigma))


def test_window_offset_is_the_fp32_cell_minus_half_width():
    grid = (0.0, 0.0, 0.05, 400, 400)
    assert G.window_offset((5.025, 3.025), grid, 121, 121) == (100 - 60, 60 - 60)
    assert G.window_offset((0.0, 0.0), grid, 11, 5) == (-5, -2)
    # just left of a cell edge: FP32 (x - x0) * (1/res) rounds to the cell below
    assert G.window_offset((np.float32(0.1) - np.float32(1e-6), 0.0), grid, 1, 1) == (1, 0)
