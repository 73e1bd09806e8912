"""Pins of the oracle's snapped observed heading: with the snap flag the
observed control of a step is the enabled heading nearest to its direction
(the discrete control of Eq. 2), not the continuous heading. Checked against
the discrete policy itself, the nearest-heading rule around the midpoints
between headings, masked headings, several speeds, the marginal likelihood
built by hand, and central differences."""
import math

import numpy as np
import pytest

GOALS = [[4.0, 1.0], [-2.0, 3.0]]
BETA = [0.5, 2.0]
K = 8


def _m(orc, **kw):
    args = dict(K=K, v=1.0, dt=0.1, goals=GOALS, beta=BETA)
    args.update(kw)
    return orc.Model(args.pop("K"), args.pop("v"), args.pop("dt"), args.pop("goals"), args.pop("beta"), **args)


def _step(z, theta, length):
    return np.array([z, [z[0] + length * math.cos(theta), z[1] + length * math.sin(theta)]])


def _normalised(x):
    x = np.asarray(x, np.float64)
    return x - (np.log(np.exp(x - x.max()).sum()) + x.max())


def _one_step_want(orc, m, z, u, prior):
    """Posterior after one step whose observed control is u, from log_policy."""
    return _normalised([prior[g * 2 + b] + orc.log_policy(m, z, BETA[b], GOALS[g])[u]
                        for g in range(2) for b in range(2)])


@pytest.mark.parametrize("frac,k_want", [(0.0, 3), (0.3, 3), (-0.9, 3), (0.9, 3), (1.1, 4), (-1.1, 2), (3.6, 5)])
def test_snapped_step_is_the_nearest_discrete_control(orc, frac, k_want):
    """A step in direction theta_3 + frac * (half the spacing) is read as
    heading 3 while |frac| < 1, and as the next heading past a midpoint;
    the one-step posterior is then the prior plus log pi of that heading."""
    m = _m(orc, snap=True)
    z = np.array([0.4, -0.3])
    theta = 2 * math.pi * 3 / K + frac * math.pi / K
    prior = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    post, _ = orc.update_posterior(m, _step(z, theta, 0.1), prior)
    assert np.allclose(post, _one_step_want(orc, m, z, k_want, prior), atol=1e-12)
    if frac != 0.0:
        cont, _ = orc.update_posterior(_m(orc), _step(z, theta, 0.1), prior)
        assert np.max(np.abs(cont - post)) > 1e-6  # the flag changes the reading


def test_snap_skips_masked_headings(orc):
    """Heading 3 disabled: a step just past theta_3 snaps to heading 4, the
    nearest enabled one (theta_2 is farther)."""
    m = _m(orc, snap=True, mask_off=1 << 3)
    z = np.array([1.0, 0.5])
    theta = 2 * math.pi * 3 / K + 0.2 * math.pi / K
    prior = np.log(np.full(4, 0.25))
    post, _ = orc.update_posterior(m, _step(z, theta, 0.1), prior)
    assert np.allclose(post, _one_step_want(orc, m, z, 4, prior), atol=1e-12)


def test_snap_on_lattice_steps_changes_nothing(orc):
    """Steps drawn from the model lie on the heading lattice: the snapped and
    the continuous readings give the same posterior."""
    m0 = _m(orc)
    m1 = _m(orc, snap=True)
    obs = orc.simulate(m0, 1, [0.0, 0.0], 30, 5, 2)
    prior = np.log(np.full(4, 0.25))
    a, _ = orc.update_posterior(m0, obs, prior)
    b, _ = orc.update_posterior(m1, obs, prior)
    assert np.allclose(a, b, atol=1e-12)


def test_snap_with_several_speeds(orc):
    """Speeds {0.5, 1, 1.5}: a step of length 1.45 v dt in direction
    theta_6 - 0.4 (half spacing) is control (speed 2, heading 6)."""
    speeds = [0.5, 1.0, 1.5]
    m = _m(orc, snap=True, speeds=speeds)
    z = np.array([-0.5, 0.7])
    theta = 2 * math.pi * 6 / K - 0.4 * math.pi / K
    prior = np.log(np.array([0.4, 0.3, 0.2, 0.1]))
    post, _ = orc.update_posterior(m, _step(z, theta, 1.45 * 0.1), prior)
    assert np.allclose(post, _one_step_want(orc, m, z, 2 * K + 6, prior), atol=1e-12)


def _trajectory(rng, speeds, n):
    """Points whose steps leave the lattice by up to 0.6 of half a spacing
    (never near a midpoint), with the snapped control of each step."""
    z = np.array([0.2, 0.1])
    pts, ctrl = [z], []
    for _ in range(n):
        s, k = int(rng.integers(0, len(speeds))), int(rng.integers(0, K))
        theta = 2 * math.pi * k / K + rng.uniform(-0.6, 0.6) * math.pi / K
        ctrl.append(s * K + k)
        pts.append(pts[-1] + 0.1 * speeds[s] * np.array([math.cos(theta), math.sin(theta)]))
    return np.array(pts), ctrl


@pytest.mark.parametrize("speeds", [[1.0], [0.5, 1.0, 1.5]])
def test_snapped_loglik_is_the_marginal_of_the_discrete_policy(orc, speeds):
    rng = np.random.default_rng(17)
    m = _m(orc, snap=True, speeds=speeds)
    traj, ctrl = _trajectory(rng, speeds, 14)
    prior = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    L, _, _, _ = orc.loglik_grad(m, [0, len(traj)], traj, prior)
    A = np.array([sum(orc.log_policy(m, traj[t], BETA[b], GOALS[g])[ctrl[t]] for t in range(len(ctrl)))
                  for g in range(2) for b in range(2)])
    want = np.log(np.exp(prior + A - (prior + A).max()).sum()) + (prior + A).max()
    assert L == pytest.approx(want, abs=1e-10)


@pytest.mark.parametrize("speeds", [[1.0], [0.5, 1.0, 1.5]])
def test_snapped_gradient_matches_central_differences(orc, speeds):
    """With the observed controls fixed on the lattice, L is smooth in the
    goals, v and w; the analytic gradient equals central differences."""
    rng = np.random.default_rng(23)
    traj, _ = _trajectory(rng, speeds, 12)
    traj2, _ = _trajectory(rng, speeds, 9)
    pts = np.concatenate([traj, traj2])
    off = [0, len(traj), len(pts)]
    prior = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    base = dict(snap=True, speeds=speeds, w1=0.8, w2=1.3)

    def L_of(goals=GOALS, v=1.0, w1=0.8, w2=1.3):
        m = _m(orc, **dict(base, goals=goals, v=v, w1=w1, w2=w2))
        return orc.loglik_grad(m, off, pts, prior)[0]

    _, dg, dv, dw = orc.loglik_grad(_m(orc, **base), off, pts, prior)
    h = 1e-5
    g = np.array(GOALS)
    for gi in range(2):
        for c in range(2):
            gp, gm = g.copy(), g.copy()
            gp[gi, c] += h
            gm[gi, c] -= h
            fd = (L_of(goals=gp) - L_of(goals=gm)) / (2 * h)
            assert dg[gi, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    # the step of a control scales with v, but the data do not move: the
    # snapped reading keeps every observed control as v changes slightly
    assert dv == pytest.approx((L_of(v=1 + h) - L_of(v=1 - h)) / (2 * h), rel=1e-6, abs=1e-8)
    assert dw[0] == pytest.approx((L_of(w1=0.8 + h) - L_of(w1=0.8 - h)) / (2 * h), rel=1e-6, abs=1e-8)
    assert dw[1] == pytest.approx((L_of(w2=1.3 + h) - L_of(w2=1.3 - h)) / (2 * h), rel=1e-6, abs=1e-8)
