"""Pins of the oracle's marginal log-likelihood and its analytic gradient.

The loss is pinned by two identities of Bayes' rule (a single hypothesis
gives the plain sum of log pi; in general the log marginal likelihood is the
sum of the log normalisers of the sequential Eq. 3 updates) and by
translation invariance; the analytic gradient is pinned against central
finite differences of the FP64 loss (h = 1e-4) and by the exact zero of
dL/dw1 (w1 shifts every Q of a step by the same amount and cancels in Eq. 2).
"""
import math

import numpy as np
import pytest


def _grid_walk(K, s, ks, z0=(0.0, 0.0)):
    z = np.zeros((len(ks) + 1, 2))
    z[0] = z0
    for t, k in enumerate(ks):
        th = 2 * math.pi * k / K
        z[t + 1] = z[t] + s * np.array([math.cos(th), math.sin(th)])
    return z


def _small_set(orc, seed=0, M=4):
    rng = np.random.default_rng(seed)
    K, v, dt = 12, 1.0, 0.1
    goals = rng.uniform(0, 5, size=(3, 2))
    beta = np.array([0.3, 1.0, 3.0, 8.0])
    m = orc.Model(K, v, dt, goals, beta)
    trajs = []
    for mm in range(M):
        j = int(rng.integers(0, 12))
        trajs.append(orc.simulate(m, j, rng.uniform(0, 5, 2), int(rng.integers(10, 30)), 99, mm))
    offsets = np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32)
    traj = np.concatenate(trajs)
    prior = np.log(np.full(12, 1 / 12))
    return m, offsets, traj, prior


def test_single_hypothesis_is_sum_of_log_policy(orc):
    K, s = 8, 0.1
    ks = [0, 1, 1, 2, 0, 7, 0, 0]
    z = _grid_walk(K, s, ks)
    m = orc.Model(K, 1.0, s, [[2.0, 1.0]], [2.5])
    L, _, _, _ = orc.loglik_grad(m, [0, len(z)], z, [0.0])
    want = sum(orc.log_policy(m, z[t], 2.5, (2.0, 1.0))[k] for t, k in enumerate(ks))
    assert L == pytest.approx(want, abs=1e-12)


def test_loglik_is_sum_of_bayes_normalisers(orc):
    """log sum_j prior_j prod_t pi_j(u_t) = sum_t log sum_j pi_j(u_t) b^t_j."""
    K, s = 8, 0.1
    goals = np.array([[2.0, 1.0], [-1.0, 2.0]])
    beta = np.array([0.5, 4.0])
    m = orc.Model(K, 1.0, s, goals, beta)
    ks = [0, 1, 0, 2, 1, 1, 0, 3, 0]
    z = _grid_walk(K, s, ks)
    prior = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    L, _, _, _ = orc.loglik_grad(m, [0, len(z)], z, prior)
    acc = 0.0
    b = prior.copy()
    for t, k in enumerate(ks):
        lp = np.array([orc.log_policy(m, z[t], beta[j % 2], goals[j // 2])[k] for j in range(4)])
        acc += np.logaddexp.reduce(lp + b)
        b, _ = orc.update_posterior(m, z[t:t + 2], b)
    assert L == pytest.approx(acc, abs=1e-12)


def test_gradient_matches_central_differences(orc):
    m, off, traj, prior = _small_set(orc)
    L, dg, dv, dw = orc.loglik_grad(m, off, traj, prior)
    h = 1e-4

    def f(goals=None, v=None, w1=None, w2=None):
        mm = orc.Model(m.K, m.v if v is None else v, m.dt, m.goals if goals is None else goals,
                       m.beta, w1=m.w1 if w1 is None else w1, w2=m.w2 if w2 is None else w2)
        return orc.loglik_grad(mm, off, traj, prior)[0]

    def check(an, fd):
        assert abs(an - fd) <= 1e-6 * max(abs(fd), abs(an)) + 1e-8, (an, fd)

    for g in range(m.G):
        for c in range(2):
            gp = m.goals.copy(); gp[g, c] += h
            gm = m.goals.copy(); gm[g, c] -= h
            check(dg[g, c], (f(goals=gp) - f(goals=gm)) / (2 * h))
    check(dv, (f(v=m.v + h) - f(v=m.v - h)) / (2 * h))
    check(dw[1], (f(w2=m.w2 + h) - f(w2=m.w2 - h)) / (2 * h))
    check(dw[0], (f(w1=m.w1 + h) - f(w1=m.w1 - h)) / (2 * h))


def test_dw1_is_exactly_zero(orc):
    m, off, traj, prior = _small_set(orc, seed=3, M=6)
    L, dg, dv, dw = orc.loglik_grad(m, off, traj, prior)
    scale = np.abs(dg).sum() + abs(dv) + abs(dw[1])
    assert abs(dw[0]) <= 1e-12 * scale


def test_translation_invariance(orc):
    m, off, traj, prior = _small_set(orc, seed=4)
    L, dg, dv, dw = orc.loglik_grad(m, off, traj, prior)
    shift = np.array([3.25, -1.5])
    ms = orc.Model(m.K, m.v, m.dt, m.goals + shift, m.beta)
    L2, dg2, _, _ = orc.loglik_grad(ms, off, traj + shift, prior)
    assert L2 == pytest.approx(L, abs=1e-9)
    np.testing.assert_allclose(dg2, dg, atol=1e-8)
