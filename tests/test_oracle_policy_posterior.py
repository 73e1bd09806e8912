"""Pins of the oracle's policy (Eq. 2) and belief update (Eq. 3 / Eq. 7).

Every expected value here comes from a closed form for a special geometry,
an invariant the paper states, or an identity of Bayes' rule -- never from
the oracle's own general formula.
"""
import math

import numpy as np
import pytest

import workloads


def _model(orc, K=4, v=1.0, dt=1.0, goals=((3.0, 0.0),), beta=(1.0,), w1=1.0, w2=1.0, mask_off=0):
    return orc.Model(K, v, dt, goals, beta, w1=w1, w2=w2, mask_off=mask_off)


# ----------------------------------------------------------------------------- policy
@pytest.mark.parametrize("w2", [1.0, 3.0, 0.25])
def test_policy_closed_form_lattice_geometry(orc, w2):
    """K = 4, step 1, z = 0, beta * w2 = ln 2: pi_k is proportional to 2^-d_k
    with d_k the distance from the next state z + e_k to the goal."""
    beta = math.log(2.0) / w2
    m = _model(orc, beta=(beta,), w1=0.37, w2=w2)
    # goal (0, 3): next states (1,0),(0,1),(-1,0),(0,-1) -> d = sqrt10, 2, sqrt10, 4
    d = np.array([math.sqrt(10), 2.0, math.sqrt(10), 4.0])
    want = 2.0 ** -d / (2.0 ** -d).sum()
    got = np.exp(orc.log_policy(m, (0.0, 0.0), beta, (0.0, 3.0)))
    np.testing.assert_allclose(got, want, rtol=1e-13)
    # goal (3, 0): heading 0 (+x) is the best one
    d = np.array([2.0, math.sqrt(10), 4.0, math.sqrt(10)])
    want = 2.0 ** -d / (2.0 ** -d).sum()
    got = np.exp(orc.log_policy(m, (0.0, 0.0), beta, (3.0, 0.0)))
    np.testing.assert_allclose(got, want, rtol=1e-13)


def test_sampling_rule_ties_and_zero_weights(orc):
    """Smallest k with u*S < C_k: a zero-weight index is never drawn, and a
    target exactly on a boundary C_k goes to the next index."""
    assert orc.sample_index([0.0, 1.0, 1.0], 0.0) == 1
    assert orc.sample_index([1.0, 1.0], 0.5) == 1
    assert orc.sample_index([1.0, 1.0], 0.5 - 2.0 ** -24) == 0
    assert orc.sample_index([1.0, 0.0, 0.0, 2.0], 0.25) == 0
    assert orc.sample_index([1.0, 0.0, 0.0, 2.0], 1.0 / 3.0) == 3
    assert orc.sample_index([0.0, 0.0, 5.0, 0.0], 1.0 - 2.0 ** -24) == 2


def test_policy_normalised_and_beta_zero_uniform(orc):
    m = _model(orc, K=36, v=1.0, dt=0.02)
    rng = np.random.default_rng(0)
    for _ in range(20):
        z = rng.uniform(0, 10, 2)
        g = rng.uniform(0, 10, 2)
        lp = orc.log_policy(m, z, rng.uniform(0.01, 100), g)
        assert abs(np.exp(lp).sum() - 1.0) < 1e-12
        lp0 = orc.log_policy(m, z, 0.0, g)  # beta -> 0: uniformly random policy (Sec. III-A)
        np.testing.assert_allclose(lp0, -math.log(36), rtol=0, atol=1e-14)


def test_policy_large_beta_is_greedy(orc):
    """Large beta: all mass on the heading whose next state is closest to g."""
    m = _model(orc, K=8, v=1.0, dt=0.1)
    p = np.exp(orc.log_policy(m, (0.0, 0.0), 1e4, (4.0, 0.0)))
    assert p[0] > 1 - 1e-12
    p = np.exp(orc.log_policy(m, (0.0, 0.0), 1e4, (-3.0, -3.0)))
    assert p[5] > 1 - 1e-12  # heading 5 = 225 degrees


def test_policy_mask_gives_zero(orc):
    """Q = -inf for disabled controls gives pi = 0 there (Sec. IV-B)."""
    mask = (1 << 0) | (1 << 3)
    m = _model(orc, K=8, v=1.0, dt=0.1, mask_off=mask)
    lp = orc.log_policy(m, (0.0, 0.0), 2.0, (4.0, 0.0))
    assert lp[0] == -np.inf and lp[3] == -np.inf
    assert abs(np.exp(lp).sum() - 1.0) < 1e-12
    full = orc.log_policy(_model(orc, K=8, v=1.0, dt=0.1), (0.0, 0.0), 2.0, (4.0, 0.0))
    keep = [1, 2, 4, 5, 6, 7]
    np.testing.assert_allclose(np.exp(lp[keep]), np.exp(full[keep]) / np.exp(full[keep]).sum(), rtol=1e-12)


def test_policy_w1_cancels(orc):
    m1 = _model(orc, K=12, v=1.3, dt=0.2, w1=1.0)
    m2 = _model(orc, K=12, v=1.3, dt=0.2, w1=-5.0)
    a = orc.log_policy(m1, (1.0, 2.0), 3.0, (4.0, 5.0))
    b = orc.log_policy(m2, (1.0, 2.0), 3.0, (4.0, 5.0))
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


# -------------------------------------------------------------------------- posterior
def test_posterior_one_step_closed_form(orc):
    """K = 4, step 1, beta = ln 2, goals (3,0) and (0,3), one step from 0 along +x.
    Both goals give the same normaliser Z = 2^-2 + 2*2^-sqrt10 + 2^-4, so
    b(g0) = 2^-2 / (2^-2 + 2^-sqrt10)."""
    m = _model(orc, goals=((3.0, 0.0), (0.0, 3.0)), beta=(math.log(2.0),))
    post, skipped = orc.update_posterior(m, [[0, 0], [1, 0]], np.log([0.5, 0.5]))
    assert skipped == 0
    b0 = 2.0 ** -2 / (2.0 ** -2 + 2.0 ** -math.sqrt(10))
    np.testing.assert_allclose(np.exp(post), [b0, 1 - b0], rtol=1e-13)


def test_posterior_sequential_equals_batch(orc):
    """Eq. 7 applied step by step equals the normalised product of Eq. 3 over
    the whole history (the per-step normalisers are common to all (beta, g)).
    Observed steps run along grid headings, so log pi(u_t) is log_policy[k_t]."""
    K = 8
    goals = np.array([[4.0, 0.0], [0.0, 4.0], [-2.0, 3.0]])
    beta = np.array([0.1, 1.0, 10.0])
    m = orc.Model(K, 1.0, 0.1, goals, beta)
    rng = np.random.default_rng(3)
    ks = rng.integers(0, K, size=25)
    z = np.zeros((26, 2))
    for t, k in enumerate(ks):
        th = 2 * math.pi * k / K
        z[t + 1] = z[t] + 0.1 * np.array([math.cos(th), math.sin(th)])
    prior = np.log(np.full(9, 1 / 9))
    seq, _ = orc.update_posterior(m, z, prior)
    acc = prior.copy()
    for t, k in enumerate(ks):
        for j in range(9):
            g, b = divmod(j, 3)
            acc[j] += orc.log_policy(m, z[t], beta[b], goals[g])[k]
    batch = acc - np.logaddexp.reduce(acc)
    np.testing.assert_allclose(seq, batch, rtol=0, atol=1e-12)
    assert abs(np.exp(seq).sum() - 1) < 1e-13


def test_posterior_beta_zero_stays_uniform(orc):
    m = orc.Model(8, 1.0, 0.1, [[4, 0], [0, 4]], [0.0, 0.0, 0.0])
    obs = np.cumsum(np.random.default_rng(1).normal(0, 0.1, size=(21, 2)), axis=0)
    post, _ = orc.update_posterior(m, obs, np.log(np.full(6, 1 / 6)))
    np.testing.assert_allclose(post, math.log(1 / 6), atol=1e-13)


def test_posterior_mirror_symmetry(orc):
    """Mirroring goals and observations across the x-axis mirrors the belief."""
    K = 8
    goals = np.array([[4.0, 1.0], [1.0, 4.0]])
    beta = np.array([0.5, 3.0])
    rng = np.random.default_rng(5)
    obs = np.cumsum(rng.normal(0, 0.1, size=(15, 2)), axis=0)
    a, _ = orc.update_posterior(orc.Model(K, 1.0, 0.1, goals, beta), obs, np.log(np.full(4, 0.25)))
    mg = goals * [1, -1]
    mo = obs * [1, -1]
    b, _ = orc.update_posterior(orc.Model(K, 1.0, 0.1, mg, beta), mo, np.log(np.full(4, 0.25)))
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_posterior_zero_displacement_skipped(orc):
    m = orc.Model(8, 1.0, 0.1, [[4, 0], [0, 4]], [1.0, 2.0])
    prior = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    post, skipped = orc.update_posterior(m, [[1.0, 1.0], [1.0, 1.0], [1.0, 1.0 + 1e-9]], prior)
    assert skipped == 2
    np.testing.assert_allclose(post, prior, atol=1e-15)


def test_posterior_leans_to_true_goal(orc):
    """Statistical sanity on the plain_small workload: averaged over histories
    drawn from the truth, the posterior mass of the true goal exceeds its prior
    (E_x~p(.|H) P(H|x) >= P(H)), and more so for the more rational truth."""
    hu = workloads.plain_small()
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    means = {}
    for true_j in (1, 2):  # (beta = 1, goal 0) and (beta = 10, goal 0)
        ps = []
        for r in range(200):
            obs = orc.simulate(m, true_j, hu.start, hu.n_obs, hu.obs_seed + r, hu.human_id)
            post, _ = orc.update_posterior(m, obs, hu.uniform_log_prior())
            p = np.exp(post).reshape(hu.G, hu.B)
            assert abs(p.sum() - 1) < 1e-12
            ps.append(p[0].sum())
        ps = np.array(ps)
        assert ps.mean() > 0.5
        means[true_j] = ps.mean()
    assert means[2] > means[1]


def test_simulated_steps_have_model_length(orc):
    hu = workloads.paper_scale()
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id)
    step = np.linalg.norm(np.diff(obs, axis=0), axis=1)
    np.testing.assert_allclose(step, np.float32(1.0) * np.float32(0.02), rtol=1e-9)
    again = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id)
    np.testing.assert_array_equal(obs, again)
