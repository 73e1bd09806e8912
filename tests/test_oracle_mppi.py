"""Pins of the MPPI oracle (Sec. III-C local planner, Eq. 8 robot) against
closed forms: straight-line and constant-turn motion, the quadratic costs by
hand, the collision indicator, and the limits of the path-integral update."""
import math

import numpy as np
import pytest

from oracle import mppi as M


def params(**kw):
    p = dict(dt=0.1, pred_stride=5, q=[3.0, 3.0, 10.0, 0.0], q_final=[0.6, 0.6, 2.0, 0.0], r=[2.0, 1.0],
             goal=[4.0, 1.0, 0.5, 0.0], coll_threshold=0.1, coll_cost=1000.0, step_cost=0.1, temperature=2.0)
    p.update(kw)
    return p


EMPTY = (np.zeros((150, 40, 60), np.float32), (0.0, 0.0, 0.1, 60, 40))


def test_straight_line_and_constant_turn():
    p = params()
    T, N = 12, 3
    delta = np.zeros((T, N, 2))
    z, u = M.rollout(p, [1.0, 2.0, 0.8, 0.3], np.zeros((T, 2)), delta)
    t = np.arange(T + 1)
    assert np.allclose(z[:, 0, 0], 1.0 + t * 0.8 * math.cos(0.3) * 0.1, rtol=0, atol=1e-13)
    assert np.allclose(z[:, 0, 1], 2.0 + t * 0.8 * math.sin(0.3) * 0.1, rtol=0, atol=1e-13)
    # constant turn rate and acceleration: theta and v are linear in t; x follows the Euler sum
    u_ref = np.tile([0.5, 0.7], (T, 1))
    z, _ = M.rollout(p, [0.0, 0.0, 1.0, 0.0], u_ref, delta)
    assert np.allclose(z[:, 0, 3], t * 0.07, atol=1e-13)
    assert np.allclose(z[:, 0, 2], 1.0 + t * 0.05, atol=1e-13)
    x = [0.0]
    for s in range(T):
        x.append(x[-1] + (1.0 + 0.05 * s) * math.cos(0.07 * s) * 0.1)
    assert np.allclose(z[:, 0, 0], x, atol=1e-13)


def test_costs_by_hand():
    p = params(step_cost=0.25)
    z0 = [0.0, 0.0, 1.0, 0.0]
    u_ref = np.array([[0.5, -0.2]])
    z, u = M.rollout(p, z0, u_ref, np.zeros((1, 1, 2)))
    run, term, _ = M.costs(p, z, u, *EMPTY)
    # after one step: x = 0.1, y = 0, v = 1.05, theta = -0.02
    e = np.array([0.1 - 4.0, 0.0 - 1.0, 1.05 - 0.5, -0.02])
    want_run = 3 * e[0] ** 2 + 3 * e[1] ** 2 + 10 * e[2] ** 2 + 2 * 0.25 + 1 * 0.04 + 0.25
    assert run[0, 0] == pytest.approx(want_run, rel=1e-14)
    assert term[0] == pytest.approx(0.6 * e[0] ** 2 + 0.6 * e[1] ** 2 + 2 * e[2] ** 2, rel=1e-14)


def test_collision_indicator_reads_the_right_cell_and_step():
    p = params(pred_stride=5, step_cost=0.0, coll_cost=1000.0)
    prob, grid = EMPTY[0].copy(), EMPTY[1]
    # robot from (0.05, 0.05) straight along +x at 1 m/s: after step t it is at x = 0.05 + 0.1 t
    prob[5 * 3 - 1, 0, 3] = 0.2   # step 3 -> x = 0.35 -> cell 3, prediction step 14
    prob[5 * 4 - 1, 0, 4] = 0.05  # below the threshold
    prob[5 * 2 - 1, 0, 3] = 0.9   # right cell, wrong step
    z, u = M.rollout(p, [0.05, 0.05, 1.0, 0.0], np.zeros((6, 2)), np.zeros((6, 1, 2)))
    run, _, _ = M.costs(dict(p, q=[0, 0, 0, 0], r=[0, 0]), z, u, prob, grid)
    assert list(run[:, 0]) == [0.0, 0.0, 1000.0, 0.0, 0.0, 0.0]


def test_update_limits():
    rng = np.random.default_rng(2)
    T, N = 5, 64
    u_ref = rng.normal(size=(T, 2))
    delta = rng.normal(size=(T, N, 2))
    S = rng.uniform(0, 10, size=(T, N))
    # a huge temperature: every sample weighs the same
    assert np.allclose(M.update(u_ref, delta, S, 1e12), u_ref + delta.mean(1), atol=1e-9)
    # a tiny one: the best sample of each step
    best = S.argmin(1)
    assert np.allclose(M.update(u_ref, delta, S, 1e-9), u_ref + delta[np.arange(T), best], atol=1e-12)
    # one sample: its own perturbation; no perturbation: the reference
    assert np.allclose(M.update(u_ref, delta[:, :1], S[:, :1], 1.0), u_ref + delta[:, 0], atol=1e-15)
    assert np.array_equal(M.update(u_ref, np.zeros((T, N, 2)), S, 1.0), u_ref)


def test_cost_to_go_is_the_suffix_sum():
    run = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    S = M.cost_to_go(run, np.array([10.0, 20.0]))
    assert np.array_equal(S, [[19.0, 32.0], [18.0, 30.0], [15.0, 26.0]])
