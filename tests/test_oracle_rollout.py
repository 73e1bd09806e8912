"""Pins of the oracle's Algorithm 1 rollout, binning and exact propagation.

Expected values: the textbook closed form of the 2-D lattice random walk
(rotate the K = 4 walk by 45 degrees into two independent +-1 walks),
moments of the uniform random walk, deterministic greedy motion, the
definition of the half-open cell rule, and mass conservation. The exact
propagator of Eq. 4 / Eq. 5 and the Monte-Carlo rollout of Eq. 6 are two
independent computations of the same distribution and are checked against
each other with a statistical bound.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lattice_k4(t, i, j):
    """P(walk at (i, j) after t unit steps), 4 equally likely axis moves."""
    if (t + i + j) % 2:
        return 0.0
    a, b = (t + i + j) // 2, (t + i - j) // 2
    if not (0 <= a <= t and 0 <= b <= t):
        return 0.0
    return math.comb(t, a) * math.comb(t, b) / 4.0 ** t


def tv_bound(p_exact_t, p_oob_t, N):
    """Per-step TV allowance: mean of the empirical TV (Jensen) plus the
    3/sqrt(N) deviation term (McDiarmid: exceeded with prob <= exp(-18))."""
    p = np.concatenate([p_exact_t.ravel(), [p_oob_t]])
    return 0.5 * np.sqrt(p * (1 - p) / N).sum() + 3.0 / math.sqrt(N)


def tv(counts_t, oob_t, N, p_exact_t, p_oob_t):
    return 0.5 * (np.abs(counts_t / N - p_exact_t).sum() + abs(oob_t / N - p_oob_t))


def _centered_grid(n_half, res):
    """Grid of (2 n_half + 1)^2 cells of size res whose centre cell is centred on 0."""
    res32 = workloads.f32(res)
    x0 = workloads.f32(-(n_half + 0.5) * res)
    return (x0, x0, res32, 2 * n_half + 1, 2 * n_half + 1)


# ----------------------------------------------------------------------- binning rule
def test_binning_half_open_and_floor(orc):
    grid = (0.0, 0.0, 0.5, 4, 4)
    assert orc.bin_point(0.0, 0.0, grid) == (0, 0)
    assert orc.bin_point(0.5, 1.0, grid) == (1, 2)          # a cell edge belongs to the upper cell
    assert orc.bin_point(1.9999999, 0.25, grid) == (3, 0)
    assert orc.bin_point(2.0, 0.0, grid) is None            # x = x0 + W*res is outside
    assert orc.bin_point(-0.25, 0.0, grid) is None          # floor, not truncation toward 0
    assert orc.bin_point(-1e-7, 0.0, grid) is None
    assert orc.bin_point(float("nan"), 0.0, grid) is None
    assert orc.bin_point(0.1, 1e30, grid) is None


def test_inv_res_is_fp32_reciprocal(orc):
    for r in (0.05, 0.1, 0.3, 1.0 / 3.0):
        assert orc.inv_res(r) == np.float32(1.0) / np.float32(r)


# ------------------------------------------------------------ uniform random walk
def test_beta_zero_k4_matches_lattice_closed_form(orc):
    """beta = 0, K = 4, step = cell size, start at a cell centre: the histogram
    follows the lattice walk law within the TV allowance at every step."""
    T, N, res = 12, 20000, 0.1
    m = orc.Model(4, 1.0, workloads.f32(0.1), [[3.0, 1.0]], [0.0])
    grid = _centered_grid(T + 1, res)
    out = orc.rollout(m, [0.0], (0.0, 0.0), T, seed=11, human=2, i0=0, i1=N, grid=grid)
    c = T + 1
    for t in range(1, T + 1):
        p = np.zeros((2 * c + 1, 2 * c + 1))
        for i in range(-t, t + 1):
            for j in range(-t, t + 1):
                p[c + j, c + i] = lattice_k4(t, i, j)
        assert abs(p.sum() - 1) < 1e-12
        d = tv(out["counts"][t - 1], out["oob"][t - 1], N, p, 0.0)
        assert d <= tv_bound(p, 0.0, N), (t, d)
        assert out["counts"][t - 1].sum() + out["oob"][t - 1] == N


@pytest.mark.parametrize("K", [3, 6, 36])
def test_beta_zero_mean_square_displacement(orc, K):
    """Uniform heading choice: E z_t = z0 and E||z_t - z0||^2 = t s^2 (K >= 3)."""
    T, N = 16, 4000
    dt = workloads.f32(0.05)
    m = orc.Model(K, 1.0, dt, [[3.0, 1.0]], [0.0])
    out = orc.rollout(m, [0.0], (1.0, -2.0), T, seed=5, human=K, i0=0, i1=N, want_counts=False,
                      want_states64=True)
    z = out["states64"] - np.array([np.float32(1.0), np.float32(-2.0)])
    s2 = (1.0 * dt) ** 2
    for t in (1, 4, 16):
        r2 = (z[:, t - 1] ** 2).sum(axis=1)
        assert abs(r2.mean() - t * s2) <= 6 * r2.std() / math.sqrt(N) + 1e-15
        assert np.all(np.abs(z[:, t - 1].mean(axis=0)) <= 6 * z[:, t - 1].std(axis=0) / math.sqrt(N) + 1e-12)


# --------------------------------------------------------------------- greedy limit
def test_large_beta_goes_straight_to_goal(orc):
    """beta = 1e4: every particle takes heading 0 toward (4, 0), identical states."""
    hu = workloads.plain_small()
    m = orc.Model(hu.K, hu.speed, hu.dt, [[4.0, 0.0]], [1e4])
    out = orc.rollout(m, [0.0], (0.0, 0.0), hu.horizon, seed=1, human=0, i0=0, i1=500,
                      grid=hu.grid, want_headings=True, want_states32=True, want_states64=True)
    assert np.all(out["headings"] == 0)
    assert np.all(out["states32"] == out["states32"][0])
    np.testing.assert_allclose(out["states64"][0, :, 0], hu.dt * np.arange(1, hu.horizon + 1), rtol=1e-12)
    np.testing.assert_array_equal(out["states64"][0, :, 1], 0.0)
    for t in range(hu.horizon):
        assert out["counts"][t].max() == 500


def test_mask_disables_headings_in_rollout(orc):
    mask = 0b10100101  # headings 0, 2, 5, 7 disabled
    m = orc.Model(8, 1.0, 0.1, [[4.0, 0.0]], [0.5], mask_off=mask)
    out = orc.rollout(m, [0.0], (0.0, 0.0), 20, seed=3, human=1, i0=0, i1=300, want_headings=True)
    assert set(np.unique(out["headings"]).tolist()) <= {1, 3, 4, 6}


# ------------------------------------------------------------ bootstrapped belief draw
def test_component_draw_frequencies(orc):
    b = np.array([0.05, 0.25, 0.0, 0.4, 0.3])
    lb = np.log(np.where(b > 0, b, 1e-300))
    lb[2] = -np.inf
    N = 40000
    comp = np.array([orc.draw_component(lb, 77, 4, i) for i in range(N)])
    cnt = np.bincount(comp, minlength=5)
    assert cnt[2] == 0
    nz = b > 0
    chi2 = ((cnt[nz] - N * b[nz]) ** 2 / (N * b[nz])).sum()
    assert chi2 < 25  # 3 dof


def test_rollout_conservation_and_determinism(orc):
    hu = workloads.plain_small()
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    lb = hu.uniform_log_prior()
    a = orc.rollout(m, lb, (0.0, 0.0), hu.horizon, hu.seed, hu.human_id, 0, 2000, grid=hu.grid)
    b = orc.rollout(m, lb, (0.0, 0.0), hu.horizon, hu.seed, hu.human_id, 0, 2000, grid=hu.grid)
    np.testing.assert_array_equal(a["counts"], b["counts"])
    assert np.all(a["counts"].reshape(hu.horizon, -1).sum(1) + a["oob"] == 2000)
    # particles are independent: [0, 1000) + [1000, 2000) == [0, 2000)
    c1 = orc.rollout(m, lb, (0.0, 0.0), hu.horizon, hu.seed, hu.human_id, 0, 1000, grid=hu.grid)
    c2 = orc.rollout(m, lb, (0.0, 0.0), hu.horizon, hu.seed, hu.human_id, 1000, 2000, grid=hu.grid)
    np.testing.assert_array_equal(c1["counts"] + c2["counts"], a["counts"])
    other = orc.rollout(m, lb, (0.0, 0.0), hu.horizon, hu.seed, hu.human_id + 1, 0, 2000, grid=hu.grid)
    assert not np.array_equal(other["counts"], a["counts"])


# -------------------------------------------------------------- exact propagation
def test_exact_k4_beta_zero_equals_closed_form(orc):
    T = 10
    m = orc.Model(4, 1.0, 0.1, [[3.0, 1.0]], [0.0])
    grid = _centered_grid(T + 1, 0.1)
    p, po, em = orc.exact_occupancy(m, [0.0], (0.0, 0.0), T, grid)
    c = T + 1
    for t in range(1, T + 1):
        want = np.zeros_like(p[0])
        for i in range(-t, t + 1):
            for j in range(-t, t + 1):
                want[c + j, c + i] = lattice_k4(t, i, j)
        np.testing.assert_allclose(p[t - 1], want, rtol=0, atol=1e-15)
        assert po[t - 1] == 0.0
        assert em[t - 1] == 0.0


def test_exact_golden_first_steps(orc):
    """Hand-derived lattice probabilities for t = 1, 2 (tests/golden)."""
    with open(os.path.join(GOLDEN, "lattice_walk_k4.json")) as f:
        g = json.load(f)
    m = orc.Model(4, 1.0, 0.1, [[3.0, 1.0]], [0.0])
    grid = _centered_grid(3, 0.1)
    p, _, _ = orc.exact_occupancy(m, [0.0], (0.0, 0.0), 2, grid)
    for t_str, cells in g["probabilities"].items():
        t = int(t_str)
        for key, frac in cells.items():
            i, j = (int(v) for v in key.split(","))
            num, den = (int(v) for v in frac.split("/"))
            assert p[t - 1][3 + j, 3 + i] == pytest.approx(num / den, abs=1e-15)


def test_exact_mass_conservation_and_greedy(orc):
    hu = workloads.plain_small()
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    lb = np.log(np.array([0.1, 0.2, 0.05, 0.3, 0.15, 0.2]))
    p, po, _ = orc.exact_occupancy(m, lb, (0.0, 0.0), 8, hu.grid)
    np.testing.assert_allclose(p.reshape(8, -1).sum(1) + po, 1.0, rtol=0, atol=1e-12)
    g = orc.Model(hu.K, hu.speed, hu.dt, [[4.0, 0.0]], [1e4])
    p, po, _ = orc.exact_occupancy(g, [0.0], (0.0, 0.0), 6, hu.grid)
    for t in range(1, 7):
        cx = int(math.floor((t * hu.dt + 5.05) / 0.1))
        assert p[t - 1][50, cx] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.slow
def test_rollout_matches_exact_propagation_plain_small(orc):
    """Eq. 6 (Monte Carlo) against Eq. 4 / Eq. 5 (exact) on the plain_small
    workload with the posterior of its observed history, T = 20."""
    hu = workloads.plain_small()
    T = hu.horizon
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id)
    post, _ = orc.update_posterior(m, obs, hu.uniform_log_prior())
    post32 = post.astype(np.float32)
    z0 = obs[-1].astype(np.float32)
    p, po, em = orc.exact_occupancy(m, post32.astype(np.float64), z0.astype(np.float64), T, hu.grid)
    N = hu.n_particles
    out = orc.rollout(m, post32, z0, T, hu.seed, hu.human_id, 0, N, grid=hu.grid)
    for t in range(1, T + 1):
        d = tv(out["counts"][t - 1], out["oob"][t - 1], N, p[t - 1], po[t - 1])
        assert d <= tv_bound(p[t - 1], po[t - 1], N) + em[t - 1], (t, d)


# ----------------------------------------------------------- draws at the FP32 state
def test_decide_f32_takes_each_draw_at_the_fp32_state(orc):
    """With decide_f32 every draw is Eq. 2 evaluated at the FP32 shadow state
    (the oracle's FP64 state is ignored for the draws), and without it at the
    FP64 state: both are rebuilt draw by draw from the policy, the uniform and
    the inverse-CDF rule. At beta = 300 near the goal the two states' policies
    differ enough that the two runs part for some particles; a run whose
    steps are dyadic (every state exact in FP32) is the same in both modes."""
    hu = workloads.paper_scale()
    beta = np.float32([300.0])
    goals = np.float32([[5.3, 5.1]])
    m = orc.Model(hu.K, hu.speed, hu.dt, goals, beta)
    z0, T, n = np.float32([5.0, 5.0]), 40, 60
    kw = dict(want_counts=False, want_headings=True, want_states32=True, want_states64=True, want_comp=True)
    runs = {f: orc.rollout(m, [0.0], z0, T, 11, 2, 0, n, decide_f32=f, **kw) for f in (False, True)}
    for f, r in runs.items():
        for i in range(0, n, 7):
            for t in (1, 2, T // 2, T):
                if t == 1:
                    z = np.asarray(z0, np.float64)
                else:
                    z = (r["states32"][i, t - 2].astype(np.float64) if f else r["states64"][i, t - 2])
                lp = orc.log_policy(m, z, beta[0], goals[0])
                k = orc.sample_index(np.exp(lp), orc.uniform_step(11, 2, i, t))
                assert k == r["headings"][i, t - 1], (f, i, t)
    assert np.any(runs[False]["headings"] != runs[True]["headings"])
    # dyadic steps: s e_k exact for K = 4 with s = 1/8, every state exact in FP32
    m4 = orc.Model(4, 1.0, 0.125, goals, np.float32([2.0]))
    a = orc.rollout(m4, [0.0], z0, 30, 3, 4, 0, 200, decide_f32=False, **kw)
    b = orc.rollout(m4, [0.0], z0, 30, 3, 4, 0, 200, decide_f32=True, **kw)
    np.testing.assert_array_equal(a["headings"], b["headings"])
    np.testing.assert_array_equal(a["states64"], b["states32"].astype(np.float64))
