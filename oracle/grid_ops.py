"""FP64 oracle of the grid epilogue -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module. It shares
no code with the CUDA library.

Two steps after emplacement, written out plainly with numpy in FP64:

* :func:`smooth` -- the Gaussian convolution of Sec. III-B, read as a blur of
  each step's normalised occupancy grid (counts / N) by the truncated,
  normalised, separable Gaussian of width ``sigma`` cells: each particle's
  unit mass is spread around its cell instead of sitting in it. Zero padding:
  mass blurred past the edge of the grid is dropped.
* :func:`union` -- the multi-human prediction of Sec. IV-B: every human's
  (smoothed) grid is placed at its cell offset on one shared grid and the
  shared grid takes the pointwise maximum.

The window offset of a human whose output window is centred on its cell
(the serving layout) is the FP32 cell of z0 (the binning of Algorithm 1's
emplacement) minus the window's half width.
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_taps(sigma):
    """Weights w_{-R..R} of the truncated Gaussian exp(-i^2 / (2 sigma^2)),
    R = ceil(3 sigma), normalised to sum 1; sigma = 0 gives the identity."""
    if sigma <= 0.0:
        return 0, np.ones(1)
    R = int(math.ceil(3.0 * sigma))
    i = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-(i * i) / (2.0 * sigma * sigma))
    return R, w / w.sum()


def smooth(counts, n_particles, sigma, pad=None):
    """counts [T][H][W] (integers) -> blurred probabilities [T][H + 2P][W + 2P]
    (FP64) on the window extended by P = pad (default R) cells on every side,
    so that the mass blurred past the window is kept."""
    R, w = gaussian_taps(sigma)
    P = R if pad is None else pad
    c = np.asarray(counts, np.float64) / float(n_particles)
    T, H, W = c.shape
    src = np.zeros((T, H + 2 * P, W + 2 * P))
    src[:, P:P + H, P:P + W] = c
    # horizontal pass, then vertical: one term per tap, added in tap order
    tmp = np.zeros_like(src)
    for k in range(-R, R + 1):
        lo, hi = max(0, -k), min(W + 2 * P, W + 2 * P - k)
        tmp[:, :, lo:hi] += w[k + R] * src[:, :, lo + k:hi + k]
    out = np.zeros_like(src)
    for k in range(-R, R + 1):
        lo, hi = max(0, -k), min(H + 2 * P, H + 2 * P - k)
        out[:, lo:hi, :] += w[k + R] * tmp[:, lo + k:hi + k, :]
    return out


def window_offset(z0, grid, Wh, Hh):
    """Cell offset (ox, oy) of a window of Wh x Hh cells centred on z0's cell;
    the cell is the FP32 binning of the emplacement step, floor((z -f x0) *f
    inv_res) with inv_res the FP32 value 1/res (numpy float32 arithmetic is
    IEEE single precision, one rounding per operation)."""
    x0, y0, res, _, _ = grid
    inv = np.float32(1.0) / np.float32(res)
    vx = (np.float32(z0[0]) - np.float32(x0)) * inv
    vy = (np.float32(z0[1]) - np.float32(y0)) * inv
    return int(np.floor(vx)) - (Wh - 1) // 2, int(np.floor(vy)) - (Hh - 1) // 2


def union(humans, T, H, W, sigma):
    """Pointwise maximum over humans on a shared grid [T][H][W].

    ``humans`` is a list of dicts with ``counts`` [T_h][H_h][W_h], ``n``
    (particles) and ``offset`` (ox, oy): the human's window cell (x, y) is
    shared cell (x + ox, y + oy). A human contributes to steps t < T_h only;
    cells no human reaches stay 0."""
    R, _ = gaussian_taps(sigma)
    out = np.zeros((T, H, W))
    for hu in humans:
        c = np.asarray(hu["counts"])
        Th, Hh, Wh = c.shape
        ox, oy = hu["offset"]
        s = smooth(c, hu["n"], sigma, pad=R)  # window extended by R cells
        for t in range(min(T, Th)):
            for y in range(Hh + 2 * R):
                Y = y - R + oy
                if not 0 <= Y < H:
                    continue
                for x in range(Wh + 2 * R):
                    X = x - R + ox
                    if 0 <= X < W and s[t, y, x] > out[t, Y, X]:
                        out[t, Y, X] = s[t, y, x]
    return out
