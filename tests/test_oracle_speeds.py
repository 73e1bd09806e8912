"""Pins of the oracle's multi-speed control set (speeds x headings, with
stationary masking of speeds, Sec. IV-B) against invariants, closed forms
and finite differences."""
import math

import numpy as np
import pytest

GOALS = [[4.0, 1.0], [-2.0, 3.0]]
BETA = [0.5, 2.0]


def _m(orc, **kw):
    args = dict(K=8, v=1.0, dt=0.1, goals=GOALS, beta=BETA)
    args.update(kw)
    return orc.Model(args.pop("K"), args.pop("v"), args.pop("dt"), args.pop("goals"), args.pop("beta"), **args)


def test_duplicated_speed_halves_every_probability(orc):
    one = _m(orc)
    two = _m(orc, speeds=[1.0, 1.0])
    for z in ([0.3, -0.2], [3.0, 2.0]):
        lp1 = orc.log_policy(one, z, 1.3, GOALS[0])
        lp2 = orc.log_policy(two, z, 1.3, GOALS[0])
        assert np.allclose(lp2[:8], lp1 - math.log(2.0), atol=1e-13)
        assert np.allclose(lp2[8:], lp1 - math.log(2.0), atol=1e-13)


def test_masked_speeds_leave_the_single_speed_model(orc):
    """Speeds {0.5, 1, 1.5} with speeds 1 and 1.5 disabled (a stationary human)
    is the one-speed model at v * 0.5; the disabled controls get pi = 0."""
    multi = _m(orc, speeds=[0.5, 1.0, 1.5], speed_off=0b110)
    slow = _m(orc, v=0.5)
    lp = orc.log_policy(multi, [1.0, 0.5], 2.0, GOALS[1])
    assert np.allclose(lp[:8], orc.log_policy(slow, [1.0, 0.5], 2.0, GOALS[1]), atol=1e-13)
    assert np.all(lp[8:] == -np.inf)


def test_beta_zero_is_uniform_over_enabled_controls(orc):
    m = _m(orc, speeds=[0.5, 1.0, 2.0], speed_off=0b010, mask_off=0b1)
    lp = orc.log_policy(m, [0.2, 0.1], 0.0, GOALS[0])
    enabled = np.array([(k != 0) and (s != 1) for s in range(3) for k in range(8)])
    assert np.allclose(lp[enabled], -math.log(enabled.sum()), atol=1e-14)
    assert np.all(lp[~enabled] == -np.inf)


def test_uniform_walk_mean_square_displacement(orc):
    """beta = 0 over 2 speeds x K = 8 headings: E||z_t - z0||^2 = t * mean(step^2)."""
    m = orc.Model(8, 1.0, 0.1, [[0.0, 0.0]], [0.0], speeds=[0.5, 1.5])
    n, T = 4000, 12
    r = orc.rollout(m, [0.0], (0.0, 0.0), T, 9, 3, 0, n, want_counts=False, want_states64=True,
                    want_headings=True)
    msd = (r["states64"] ** 2).sum(2).mean(0)
    want = np.arange(1, T + 1) * 0.01 * (0.25 + 2.25) / 2
    assert np.all(np.abs(msd - want) <= 5 * want * math.sqrt(2.0 / n) + 1e-12)
    assert r["headings"].max() >= 8  # the second speed is drawn


def test_observed_speed_snaps_to_the_nearest_multiplier(orc):
    """One observed step of length 0.95 * v dt along heading 2 is the control
    (speed 1.0, heading 2) of speeds {0.5, 1.0, 1.5}: the one-step posterior
    is the prior plus that control's log-probability, renormalised."""
    m = _m(orc, speeds=[0.5, 1.0, 1.5])
    z = np.array([0.4, -0.3])
    step = 0.95 * 0.1 * np.array([0.0, 1.0])  # heading 2 of K = 8 is +y
    obs = np.stack([z, z + step])
    prior = np.log(np.full(4, 0.25))
    post, skipped = orc.update_posterior(m, obs, prior)
    assert skipped == 0
    want = np.array([prior[g * 2 + b] + orc.log_policy(m, z, BETA[b], GOALS[g])[1 * 8 + 2]
                     for g in range(2) for b in range(2)])
    want -= np.log(np.exp(want - want.max()).sum()) + want.max()
    assert np.allclose(post, want, atol=1e-12)


def test_w1_is_identifiable_with_several_speeds(orc):
    """With one speed dL/dw1 = 0 exactly; with two it is not, and the analytic
    gradient matches central differences of the FP64 loss."""
    rng = np.random.default_rng(4)
    trajs, offs = [], [0]
    for m_ in range(6):
        z = rng.uniform(-1, 1, size=2)
        pts = [z]
        for _ in range(15):
            h = rng.integers(0, 8)
            sp = [0.5, 1.0][rng.integers(0, 2)]
            pts.append(pts[-1] + 0.1 * sp * np.array([math.cos(2 * math.pi * h / 8), math.sin(2 * math.pi * h / 8)]))
        trajs.append(np.array(pts))
        offs.append(offs[-1] + len(pts))
    traj = np.concatenate(trajs)
    prior = np.log(np.full(4, 0.25))
    base = dict(speeds=[0.5, 1.0])
    L, dg, dv, dw = orc.loglik_grad(_m(orc, **base), offs, traj, prior)
    assert abs(dw[0]) > 1e-3
    h = 1e-5
    Lp = orc.loglik_grad(_m(orc, w1=1.0 + h, **base), offs, traj, prior)[0]
    Lm = orc.loglik_grad(_m(orc, w1=1.0 - h, **base), offs, traj, prior)[0]
    assert dw[0] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6)
    Lp = orc.loglik_grad(_m(orc, v=1.0 + h, **base), offs, traj, prior)[0]
    Lm = orc.loglik_grad(_m(orc, v=1.0 - h, **base), offs, traj, prior)[0]
    assert dv == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5)
    assert abs(orc.loglik_grad(_m(orc), offs, traj, prior)[3][0]) < 1e-12


def test_speed_term_alone_closed_form(orc):
    """With w2 = 0 only the speed term is left: pi(s, k) is uniform over the
    headings and proportional to exp(-beta w1 v m_s dt) over the speeds."""
    speeds = [0.5, 1.0, 1.5]
    m = _m(orc, speeds=speeds, w1=2.0, w2=0.0, speed_off=0b100)
    beta, v, dt = 1.3, 1.0, 0.1
    lp = orc.log_policy(m, [0.7, -0.4], beta, GOALS[1])
    logits = np.array([-beta * 2.0 * v * ms * dt for ms in speeds])
    logits[2] = -np.inf
    want = np.repeat(logits - (math.log(8.0) + np.log(np.exp(logits[:2]).sum())), 8)
    assert np.all(lp[16:] == -np.inf)
    assert np.allclose(lp[:16], want[:16], atol=1e-14)


def test_observed_speed_snaps_among_enabled_speeds(orc):
    """With the middle speed masked, a step of 0.95 v dt is read at the nearest
    enabled multiplier (0.5), never at the masked one: the one-step posterior
    is the prior plus that control's log-probability."""
    m = _m(orc, speeds=[0.5, 1.0, 1.5], speed_off=0b010)
    z = np.array([0.4, -0.3])
    obs = np.stack([z, z + 0.95 * 0.1 * np.array([0.0, 1.0])])  # heading 2
    prior = np.log(np.full(4, 0.25))
    post, _ = orc.update_posterior(m, obs, prior)
    want = np.array([prior[g * 2 + b] + orc.log_policy(m, z, BETA[b], GOALS[g])[0 * 8 + 2]
                     for g in range(2) for b in range(2)])
    want -= np.log(np.exp(want - want.max()).sum()) + want.max()
    assert np.all(np.isfinite(post))
    assert np.allclose(post, want, atol=1e-12)


def test_loglik_is_the_marginal_of_the_policy(orc):
    """L of loglik_grad equals log sum_j prior_j prod_t pi_j(u_t | z_t), built
    here from log_policy with each observed step read at its heading and the
    nearest multiplier (headings on the lattice: every step is a control)."""
    rng = np.random.default_rng(11)
    speeds = [0.5, 1.0, 1.5]
    m = _m(orc, speeds=speeds)
    z = np.array([0.2, 0.1])
    pts, ctrl = [z], []
    for _ in range(12):
        s, h = int(rng.integers(0, 3)), int(rng.integers(0, 8))
        ctrl.append(s * 8 + h)
        pts.append(pts[-1] + 0.1 * speeds[s] * np.array([math.cos(2 * math.pi * h / 8), math.sin(2 * math.pi * h / 8)]))
    traj = np.array(pts)
    prior = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    L, _, _, _ = orc.loglik_grad(m, [0, len(pts)], traj, prior)
    A = np.array([sum(orc.log_policy(m, traj[t], BETA[b], GOALS[g])[ctrl[t]] for t in range(12))
                  for g in range(2) for b in range(2)])
    want = np.log(np.exp(prior + A - (prior + A).max()).sum()) + (prior + A).max()
    assert L == pytest.approx(want, abs=1e-10)
