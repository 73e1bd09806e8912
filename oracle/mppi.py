"""FP64 oracle of the MPPI cost rollout -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module. It shares
no code with the CUDA library.

The local planner of Sec. III-C written out plainly (numpy, FP64, vectorised
over the samples only):

* robot model (the unicycle with acceleration of Eq. 8): state
  z = [x, y, v, theta], control u = [a, omega]; explicit Euler over dt:
  x += v cos(theta) dt, y += v sin(theta) dt, v += a dt, theta += omega dt
  (all from the state at the start of the step);
* sample i applies u_ref[t] + delta[t][i] at steps t = 0..T-1 (the
  perturbations are inputs: the caller draws them);
* running cost after step t (state z_{t+1}): (z - g)^T diag(q) (z - g) +
  u^T diag(r) u + step_cost + coll_cost * [p >= coll_threshold], with p the
  predicted occupancy at the robot's cell at prediction step
  (t + 1) * pred_stride - 1 (0 outside the grid or past its horizon); the
  collision cost is the global planner's of the same section;
* terminal cost (z_T - g)^T diag(q_final) (z_T - g);
* the update of the MPPI equation of Sec. III-C with the cost-to-go from
  each step: S_i(t) = sum_{s >= t} running cost_s + terminal, w_i(t) =
  exp(-(S_i(t) - min_i S_i(t)) / tau), u*[t] = u_ref[t] + sum_i w_i(t)
  delta[t][i] / sum_i w_i(t).
"""
from __future__ import annotations

import numpy as np


def rollout(params, z0, u_ref, delta):
    """States [T+1][N][4] and controls [T][N][2] of every sample (FP64)."""
    u_ref = np.asarray(u_ref, np.float64)
    delta = np.asarray(delta, np.float64)
    T, N, _ = delta.shape
    dt = float(params["dt"])
    z = np.zeros((T + 1, N, 4))
    z[0] = np.asarray(z0, np.float64)
    u = u_ref[:, None, :] + delta
    for t in range(T):
        x, y, v, th = z[t, :, 0], z[t, :, 1], z[t, :, 2], z[t, :, 3]
        z[t + 1, :, 0] = x + v * np.cos(th) * dt
        z[t + 1, :, 1] = y + v * np.sin(th) * dt
        z[t + 1, :, 2] = v + u[t, :, 0] * dt
        z[t + 1, :, 3] = th + u[t, :, 1] * dt
    return z, u


def occupancy_at(prob, grid, x, y, k):
    """Grid value at the cell of (x, y) at prediction step k (0 outside).
    The cell is floor((x - x0) / res) in FP64; returns (p, distance of the
    point to the nearest cell edge in cells)."""
    x0, y0, res, W, H = grid
    Tg = prob.shape[0]
    vx = (x - x0) / res
    vy = (y - y0) / res
    cx = np.floor(vx).astype(np.int64)
    cy = np.floor(vy).astype(np.int64)
    edge = np.minimum(np.minimum(vx - cx, cx + 1 - vx), np.minimum(vy - cy, cy + 1 - vy))
    p = np.zeros(x.shape)
    if 0 <= k < Tg:
        inside = (cx >= 0) & (cx < W) & (cy >= 0) & (cy < H)
        p[inside] = prob[k, cy[inside], cx[inside]]
    return p, edge


def costs(params, z, u, prob, grid):
    """Running costs [T][N] and terminal cost [N]; also the smallest distance
    (in cells) of a looked-up position to a cell edge, per sample."""
    T, N = u.shape[0], u.shape[1]
    g = np.asarray(params["goal"], np.float64)
    q = np.asarray(params["q"], np.float64)
    qf = np.asarray(params["q_final"], np.float64)
    r = np.asarray(params["r"], np.float64)
    thr = np.float32(params["coll_threshold"])
    run = np.zeros((T, N))
    edge_min = np.full(N, np.inf)
    for t in range(T):
        e = z[t + 1] - g
        run[t] = (e * e * q).sum(1) + (u[t] * u[t] * r).sum(1) + params["step_cost"]
        k = (t + 1) * int(params["pred_stride"]) - 1
        p, edge = occupancy_at(prob, grid, z[t + 1, :, 0], z[t + 1, :, 1], k)
        run[t] += params["coll_cost"] * (p.astype(np.float32) >= thr)
        if 0 <= k < prob.shape[0]:  # only lookups that read the grid can flip
            edge_min = np.minimum(edge_min, edge)
    eT = z[T] - g
    term = (eT * eT * qf).sum(1)
    return run, term, edge_min


def cost_to_go(run, term):
    """S[t][i] = sum_{s >= t} run[s][i] + term[i]."""
    return np.cumsum(run[::-1], axis=0)[::-1] + term[None, :]


def update(u_ref, delta, S, tau):
    """u*[t] = u_ref[t] + sum_i w_i(t) delta[t][i] / sum_i w_i(t)."""
    w = np.exp(-(S - S.min(axis=1, keepdims=True)) / float(tau))
    num = (w[:, :, None] * np.asarray(delta, np.float64)).sum(1)
    return np.asarray(u_ref, np.float64) + num / w.sum(1)[:, None]


def solve(params, z0, u_ref, delta, prob, grid):
    """(u* [T][2], total cost per sample [N], cost-to-go [T][N], edge_min [N])."""
    z, u = rollout(params, z0, u_ref, delta)
    run, term, edge = costs(params, z, u, np.asarray(prob), grid)
    S = cost_to_go(run, term)
    return update(u_ref, delta, S, params["temperature"]), S[0], S, edge
