"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (stated once, used below):
  posterior   |log b_gpu - log b_64| <= 1e-5 where b_64 >= 1e-8, b_gpu <= 1e-7
              elsewhere, |sum b_gpu - 1| <= 1e-6;
  trajectories identical heading sequences and (beta, g) draws under the
              shared Philox streams, against the oracle taking its draws at
              the FP32 particle state (reading R4), except at most 1e-4 of
              the particles over the whole horizon (FP32 CDF boundaries):
              d <= 1e-4 n where 1e-4 n >= 1, else d below the count that a
              Poisson number at the rate 1e-4 reaches with probability
              < 1e-6; non-diverged particles have bit-identical FP32 states;
              every diverged particle differs first at a draw whose uniform
              lies within the error budget of a boundary of the exact CDF
              (gpu_util.explain_divergences), against the FP32-state and the
              FP64-state oracle alike;
  histogram   bit-exact given identical FP32 states;
  occupancy   per-step TV against exact propagation within the allowance of
              test_oracle_rollout.tv_bound.
"""
import math
import zlib

import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev, explain_divergences, posterior, predict
from test_oracle_rollout import lattice_k4, tv, tv_bound

pytestmark = pytest.mark.gpu

TRAJ_RATE = 1e-4


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def assert_posterior_close(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    big = np.exp(want) >= 1e-8
    assert np.all(np.abs(got[big] - want[big]) <= 1e-5), np.max(np.abs(got[big] - want[big]))
    assert np.all(np.exp(got[~big]) <= 1e-7)
    assert abs(np.exp(got).sum() - 1.0) <= 1e-6


def poisson_reject_at(N, rate=TRAJ_RATE, alpha=1e-6):
    """Smallest d with P(Poisson(N*rate) >= d) < alpha."""
    lam = N * rate
    p, cdf, d = math.exp(-lam), 0.0, 0
    while True:
        cdf += p
        d += 1
        if 1.0 - cdf < alpha:
            return d
        p *= lam / d


def compare_trajectories(got, ref):
    """Particles whose draws differ anywhere; states must be bit-equal elsewhere."""
    diff = np.any(got["headings"] != ref["headings"], axis=1) | (got["comp"] != ref["comp"])
    same = ~diff
    assert np.array_equal(got["states32"][same], ref["states32"][same])
    return int(diff.sum())


def trajectory_parity(orc, m, lb, z0, T, seed, human, got, n, label, grid=None):
    """Compare the traced particles [0, n) with the oracle twice.

    Parity proper (the tolerance's "diverging at FP32 CDF boundaries"): the
    oracle takes every draw at the FP32 particle state, in FP64 arithmetic
    (reading R4), so a draw can differ only through the kernel's FP32
    arithmetic of that draw. Beside it, the oracle with an FP64 state (the
    exact Monte Carlo): its divergences also carry the FP32 state's drift,
    and each must lie within the error budget of explain_divergences.
    Returns (d at the FP32 state, d at the FP64 state, the FP32-state run)."""
    kw = dict(want_headings=True, want_states32=True, want_states64=True, want_comp=True)
    ref32 = orc.rollout(m, lb, z0, T, seed, human, 0, n, grid=grid, want_counts=grid is not None,
                        decide_f32=True, **kw)
    d32 = compare_trajectories(got, ref32)
    assert explain_divergences(orc, m, lb, z0, seed, human, got, ref32, decide_f32=True) == d32
    ref64 = orc.rollout(m, lb, z0, T, seed, human, 0, n, grid=None, want_counts=False, **kw)
    d64 = compare_trajectories(got, ref64)
    assert explain_divergences(orc, m, lb, z0, seed, human, got, ref64) == d64
    print(f"[trajectories] {label}: {d32} of {n} particles diverged at the FP32 state "
          f"({d64} against the FP64-state oracle), T = {T}")
    return d32, d64, ref32


def _obs_and_post(orc, hu):
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, w1=hu.w1, w2=hu.w2)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    post, _ = orc.update_posterior(m, obs.astype(np.float64), hu.uniform_log_prior())
    return m, obs, post


# --------------------------------------------------------------------- generator
def test_philox_blocks_bit_exact(ctx, orc):
    import paper_2603_01122_gb300 as pm
    n = 4096
    for seed, human, purpose, p0, block in [(0, 0, 1, 0, 0), (20260301, 7, 2, 123456, 3),
                                            (2**64 - 1, 2**32 - 1, 2, 2**40, 2**50)]:
        out = torch.empty((n, 4), dtype=torch.int64, device="cuda:0")
        pm.pm_philox_blocks(ctx, seed, human, purpose, p0, block, n, out)
        got = out.cpu().numpy().view(np.uint64)
        for i in list(range(64)) + list(range(n - 64, n)):
            want = orc.philox4x64([(p0 + i) % 2**64, block, purpose, 0], [seed, human])
            np.testing.assert_array_equal(got[i], want)


# --------------------------------------------------------------------- posterior
@pytest.mark.parametrize("name", ["plain_small", "paper_scale"])
def test_posterior_matches_oracle(ctx, orc, name):
    hu = getattr(workloads, name)()
    m, obs, want = _obs_and_post(orc, hu)
    got = posterior(ctx, GpuHuman.of(hu), obs, hu.uniform_log_prior())
    assert_posterior_close(got, want)


def test_posterior_batched_workload_histories(ctx, orc):
    """All 16 humans of the batched workload (G = 2..6, 50 steps each)."""
    for hu in workloads.batched():
        m, obs, want = _obs_and_post(orc, hu)
        got = posterior(ctx, GpuHuman.of(hu), obs, hu.uniform_log_prior())
        assert_posterior_close(got, want)


def test_posterior_mask_stationary_and_weights(ctx, orc):
    hu = workloads.paper_scale()
    rng = np.random.default_rng(9)
    mask = int(rng.integers(0, 2**36)) & ~1  # heading 0 stays enabled
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, w1=0.3, w2=1.7, mask_off=mask)
    obs = orc.simulate(orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta), hu.true_j, hu.start, 30,
                       hu.obs_seed, hu.human_id).astype(np.float32)
    obs = np.concatenate([obs[:10], obs[9:10], obs[9:10], obs[10:]])  # two stationary steps
    prior = np.log(rng.dirichlet(np.ones(hu.G * hu.B))).astype(np.float32)
    want, skipped = orc.update_posterior(m, obs.astype(np.float64), prior)
    assert skipped == 2
    gh = GpuHuman(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, w1=0.3, w2=1.7, heading_off=mask)
    assert_posterior_close(posterior(ctx, gh, obs, prior), want)


def test_posterior_one_step_calls_equal_one_call(ctx, orc):
    """Serving form: 50 calls of one observed step each equal one 50-step call."""
    hu = workloads.paper_scale()
    m, obs, want = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    import paper_2603_01122_gb300 as pm
    obs_d = dev(obs)
    lb = dev(hu.uniform_log_prior())
    for t in range(hu.n_obs):
        pm.pm_update_posterior(ctx, gh.model, obs_d[t:t + 2], 1, lb)
    torch.cuda.synchronize()
    assert_posterior_close(lb.cpu().numpy(), want)


def test_posterior_out_of_place(ctx, orc):
    """pm_update_posterior_into reads the prior from one buffer and writes the
    posterior to another: the prior is unchanged, the posterior equals the
    oracle's and, bit for bit, the in-place call's; n_obs = 0 copies the
    prior; buffers that overlap without being the same are rejected."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    m, obs, want = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    obs_d = dev(obs)
    rng = np.random.default_rng(4)
    prior_np = np.log(rng.dirichlet(np.ones(hu.G * hu.B))).astype(np.float32)
    want_p, _ = orc.update_posterior(m, obs.astype(np.float64), prior_np.astype(np.float64))
    prior = dev(prior_np)
    out = torch.full_like(prior, float("nan"))
    pm.pm_update_posterior_into(ctx, gh.model, obs_d, hu.n_obs, prior, out)
    inplace = prior.clone()
    pm.pm_update_posterior(ctx, gh.model, obs_d, hu.n_obs, inplace)
    same = prior.clone()
    pm.pm_update_posterior_into(ctx, gh.model, obs_d, hu.n_obs, same, same)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(prior.cpu().numpy(), prior_np)
    assert_posterior_close(out.cpu().numpy(), want_p)
    np.testing.assert_array_equal(out.cpu().numpy(), inplace.cpu().numpy())
    np.testing.assert_array_equal(same.cpu().numpy(), inplace.cpu().numpy())
    copy = torch.full_like(prior, float("nan"))
    pm.pm_update_posterior_into(ctx, gh.model, obs_d, 0, prior, copy)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(copy.cpu().numpy(), prior_np)
    buf = torch.zeros(2 * hu.G * hu.B, device="cuda:0")
    with pytest.raises(pm.PmError):
        pm.pm_update_posterior_into(ctx, gh.model, obs_d, hu.n_obs, buf[:hu.G * hu.B], buf[1:hu.G * hu.B + 1])


def test_posterior_of_stationary_steps_is_the_prior(ctx, orc):
    """Steps shorter than 1e-6 m leave the belief unchanged (reading A4): a
    history of only such steps returns the prior bit for bit (no FP32
    renormalisation), and so does a batched update of such steps."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    gh = GpuHuman.of(hu)
    rng = np.random.default_rng(2)
    prior = np.log(rng.dirichlet(np.ones(hu.G * hu.B))).astype(np.float32)
    obs = np.repeat(np.float32([[4.2, 6.1]]), 9, axis=0)
    obs[3:] += np.float32(3e-7)  # one step of 4e-7 m, the rest of length zero
    got = posterior(ctx, gh, obs, prior)
    np.testing.assert_array_equal(got, prior)
    lb = dev(prior)
    obs_d = dev(obs)
    batch = pm.pm_batch_create(ctx, gh.model, 1)
    counts = torch.zeros((3, 4, 4), dtype=torch.int32, device="cuda:0")
    oob = torch.zeros(3, dtype=torch.int32, device="cuda:0")
    g = pm.make_grid(0.0, 0.0, 1.0, 4, 4)
    pm.pm_batch_set(batch, [pm.make_human(gh.goals, gh.beta, lb, obs_d[-1], 10, 3, g, 1, 2, counts, oob,
                                          obs_xy=obs_d, n_obs=8)])
    pm.pm_batch_update_posterior(batch)
    torch.cuda.synchronize()
    pm.pm_batch_destroy(batch)
    np.testing.assert_array_equal(lb.cpu().numpy(), prior)


def test_posterior_large_history_max_components(ctx, orc):
    """G*B = 256 components, 200 steps, K = 64."""
    rng = np.random.default_rng(4)
    goals = rng.uniform(0, 10, (16, 2)).astype(np.float32)
    beta = workloads.beta_grid(-2.0, 2.0, 16)
    m = orc.Model(64, 1.0, workloads.f32(0.05), goals, beta)
    obs = orc.simulate(m, 37, np.float32([5.0, 5.0]), 200, 3, 3).astype(np.float32)
    prior = np.full(256, -math.log(256), np.float32)
    want, _ = orc.update_posterior(m, obs.astype(np.float64), prior)
    got = posterior(ctx, GpuHuman(64, 1.0, workloads.f32(0.05), goals, beta), obs, prior)
    assert_posterior_close(got, want)


# -------------------------------------------------------------------- rollout
def test_plain_small_trajectories_and_histogram(ctx, orc):
    """Every particle of the plain_small workload traced: draws identical except
    <= 1e-4 of particles, histogram bit-exact given the FP32 states."""
    hu = workloads.plain_small()
    m, obs, post = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    z0 = obs[-1]
    N, T = hu.n_particles, hu.horizon
    got = predict(ctx, gh, lb, z0, N, T, hu.grid, hu.seed, hu.human_id, n_trace=N)
    d, _, ref = trajectory_parity(orc, m, lb, z0, T, hu.seed, hu.human_id, got, N, "plain_small", grid=hu.grid)
    assert d <= TRAJ_RATE * N, d
    c, o = orc.bin_states(got["states32"], hu.grid)
    np.testing.assert_array_equal(got["counts"], c)
    np.testing.assert_array_equal(got["oob"], o)
    if d == 0:
        np.testing.assert_array_equal(got["counts"], ref["counts"])


def test_plain_small_occupancy_vs_exact_propagation(ctx, orc):
    hu = workloads.plain_small()
    m, obs, post = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    z0 = obs[-1]
    got = predict(ctx, gh, lb, z0, hu.n_particles, hu.horizon, hu.grid, hu.seed, hu.human_id)
    p, po, em = orc.exact_occupancy(m, lb.astype(np.float64), z0.astype(np.float64), hu.horizon, hu.grid)
    for t in range(1, hu.horizon + 1):
        d = tv(got["counts"][t - 1], got["oob"][t - 1], hu.n_particles, p[t - 1], po[t - 1])
        assert d <= tv_bound(p[t - 1], po[t - 1], hu.n_particles) + em[t - 1], (t, d)


def test_beta_zero_lattice_walk(ctx, orc):
    T, N = 16, 100_000
    dt = workloads.f32(0.1)
    gh = GpuHuman(4, 1.0, dt, [[3.0, 1.0]], [0.0])
    res = workloads.f32(0.1)
    x0 = workloads.f32(-(T + 1.5) * 0.1)
    grid = (x0, x0, res, 2 * T + 3, 2 * T + 3)
    got = predict(ctx, gh, [0.0], (0.0, 0.0), N, T, grid, 5, 9)
    c = T + 1
    for t in range(1, T + 1):
        p = np.zeros((2 * c + 1, 2 * c + 1))
        for i in range(-t, t + 1):
            for j in range(-t, t + 1):
                p[c + j, c + i] = lattice_k4(t, i, j)
        d = tv(got["counts"][t - 1], got["oob"][t - 1], N, p, 0.0)
        assert d <= tv_bound(p, 0.0, N), (t, d)


def test_large_beta_straight_line(ctx, orc):
    hu = workloads.plain_small()
    gh = GpuHuman(hu.K, hu.speed, hu.dt, [[4.0, 0.0]], [1e4])
    got = predict(ctx, gh, [0.0], (0.0, 0.0), 3000, hu.horizon, hu.grid, 1, 0, n_trace=3000)
    assert np.all(got["headings"] == 0)
    assert np.all(got["states32"] == got["states32"][0])
    for t in range(hu.horizon):
        assert got["counts"][t].max() == 3000


def test_paper_scale_sampled_particles_full_launch(ctx, orc):
    """Full paper_scale launch (N = 100k, T = 150, the benchmark's configuration)
    with the first 20000 particles traced and recomputed one by one."""
    hu = workloads.paper_scale()
    m, obs, post = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    z0 = obs[-1]
    N, T, n = hu.n_particles, hu.horizon, 20000
    got = predict(ctx, gh, lb, z0, N, T, hu.grid, hu.seed, hu.human_id, n_trace=n)
    d, d64, _ = trajectory_parity(orc, m, lb, z0, T, hu.seed, hu.human_id, got, n, "paper_scale full launch")
    assert d <= TRAJ_RATE * n, d
    counts, oob = got["counts"], got["oob"]
    assert np.all(counts.reshape(T, -1).sum(1).astype(np.int64) + oob == N)
    # every count lies within reach of z0 after t steps (|z_t - z0| <= t v dt)
    x0, y0, res, W, H = hu.grid
    yy, xx = np.mgrid[0:H, 0:W]
    cxz, cyz = (z0[0] - x0) / res, (z0[1] - y0) / res
    dist = np.hypot(np.maximum(np.abs(xx + 0.5 - cxz) - 0.5, 0), np.maximum(np.abs(yy + 0.5 - cyz) - 0.5, 0)) * res
    for t in (1, 10, 75, 150):
        assert counts[t - 1][dist > t * hu.speed * hu.dt + 1e-4].sum() == 0
    # the traced particles' own histogram is a lower bound of the full one
    c_sub, _ = orc.bin_states(got["states32"], hu.grid)
    assert np.all(c_sub <= counts)


@pytest.mark.parametrize("case", ["ragged_N", "single", "T1", "corner", "outside", "K3", "K37_mask",
                                  "K64", "J256", "tiny_grid", "beta_neg_large", "beta_neg_large_mask", "T_max"])
def test_edge_cases_full_trace(ctx, orc, case):
    hu = workloads.paper_scale()
    K, goals, beta, heading_off = hu.K, hu.goals, hu.beta, 0
    N, T, z0, grid = 3001, 40, np.float32([5.0, 5.0]), hu.grid
    dt = hu.dt
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    if case == "ragged_N":
        N = 257 * 13 + 5
    elif case == "single":
        N = 1
    elif case == "T1":
        T = 1
    elif case == "corner":
        z0 = np.float32([0.02, 0.03])
    elif case == "outside":
        z0 = np.float32([-0.5, 10.2])
    elif case == "K3":
        K = 3
    elif case == "K37_mask":
        K, heading_off = 37, int(rng.integers(0, 2**37)) & ~0b111
    elif case == "K64":
        K = 64
    elif case == "J256":
        goals = rng.uniform(0, 10, (16, 2)).astype(np.float32)
        beta = workloads.beta_grid(-2.0, 2.0, 16)
    elif case in ("beta_neg_large", "beta_neg_large_mask"):
        # |beta| far above the bound-normalised range: the exact-extreme draw,
        # whose most probable heading is the farthest from the goal
        beta = np.float32([-3000.0, -40.0, 1e4])
        if case.endswith("mask"):
            heading_off = 0b101
    elif case == "tiny_grid":
        grid = (workloads.f32(4.9), workloads.f32(4.95), workloads.f32(0.05), 3, 2)
        dt = workloads.f32(0.05)
    elif case == "T_max":
        # the longest horizon the library takes (PM_MAX_HORIZON): histogram
        # planes, oob, Philox blocks and trace offsets at the end of their
        # range; moderate beta, so 4096 FP32 steps of state drift stay well
        # inside the draws' error budget
        N, T = 64, 4096
        beta = np.float32([0.1, 0.5, 1.0])
        grid = (workloads.f32(4.5), workloads.f32(4.5), workloads.f32(0.05), 20, 20)
    m = orc.Model(K, hu.speed, dt, goals, beta, mask_off=heading_off)
    J = m.G * m.B
    lb = np.log(rng.dirichlet(np.ones(J))).astype(np.float32)
    gh = GpuHuman(K, hu.speed, dt, goals, beta, heading_off=heading_off)
    got = predict(ctx, gh, lb, z0, N, T, grid, 77, 5, n_trace=N)
    d, _, _ = trajectory_parity(orc, m, lb, z0, T, 77, 5, got, N, f"edge case {case}")
    assert d < poisson_reject_at(N), d  # at most 1e-4 of particles, over the whole horizon
    c, o = orc.bin_states(got["states32"], grid)
    np.testing.assert_array_equal(got["counts"], c)
    np.testing.assert_array_equal(got["oob"], o)
    assert np.all(got["counts"].reshape(T, -1).sum(1).astype(np.int64) + got["oob"] == N)
    if heading_off:
        off = [k for k in range(K) if (heading_off >> k) & 1]
        assert not np.isin(got["headings"], off).any()


def test_determinism_and_streams(ctx, orc):
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    lb = hu.uniform_log_prior()
    a = predict(ctx, gh, lb, (0.0, 0.0), 20000, 20, hu.grid, 1, 2)
    b = predict(ctx, gh, lb, (0.0, 0.0), 20000, 20, hu.grid, 1, 2)
    np.testing.assert_array_equal(a["counts"], b["counts"])
    c = predict(ctx, gh, lb, (0.0, 0.0), 20000, 20, hu.grid, 1, 3)
    assert not np.array_equal(a["counts"], c["counts"])


def test_zero_and_rollout_halves_equal_predict(ctx, orc):
    """pm_zero_occupancy on a second stream beside pm_update_posterior_into,
    then pm_rollout_occupancy, equals pm_update_posterior + pm_predict_occupancy
    from garbage outputs; a second rollout without zeroing adds the counts
    again."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = dev(orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32))
    gh = GpuHuman.of(hu)
    x0, y0, res, W, H = hu.grid
    grid = pm.make_grid(x0, y0, res, W, H)
    N, T = 30000, 60
    prior = dev(hu.uniform_log_prior())
    z0 = obs[-1].cpu().numpy()
    lb1 = prior.clone()
    pm.pm_update_posterior(ctx, gh.model, obs, hu.n_obs, lb1)
    c1 = torch.full((T, H, W), 0x3C3C3C3C, dtype=torch.int32, device="cuda:0")
    o1 = torch.full((T,), 7, dtype=torch.int32, device="cuda:0")
    pm.pm_predict_occupancy(ctx, gh.model, lb1, float(z0[0]), float(z0[1]), N, T, grid, hu.seed, 5, c1, o1)
    lb2 = torch.empty_like(prior)
    c2 = torch.full_like(c1, 0x5A5A5A5A)
    o2 = torch.full_like(o1, 9)
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    side.wait_stream(main)
    pm.pm_zero_occupancy(ctx, T, grid, c2, o2, side)
    pm.pm_update_posterior_into(ctx, gh.model, obs, hu.n_obs, prior, lb2, main)
    main.wait_stream(side)
    pm.pm_rollout_occupancy(ctx, gh.model, lb2, float(z0[0]), float(z0[1]), N, T, grid, hu.seed, 5, c2, o2, main)
    torch.cuda.synchronize()
    assert torch.equal(lb1, lb2) and torch.equal(c1, c2) and torch.equal(o1, o2)
    pm.pm_rollout_occupancy(ctx, gh.model, lb2, float(z0[0]), float(z0[1]), N, T, grid, hu.seed, 5, c2, o2)
    torch.cuda.synchronize()
    assert torch.equal(c2, 2 * c1) and torch.equal(o2, 2 * o1)
    with pytest.raises(pm.PmError):
        pm.pm_zero_occupancy(ctx, 0, grid, c2, o2)


def test_host_api_matches_device_path(ctx, orc):
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    m, obs, post = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    N, T = 20000, 60
    want = predict(ctx, gh, lb, obs[-1], N, T, hu.grid, hu.seed, hu.human_id)
    x0, y0, res, W, H = hu.grid
    post_out = np.zeros(hu.G * hu.B, np.float32)
    counts = np.zeros((T, H, W), np.uint32)
    oob = np.zeros(T, np.uint32)
    pm.pm_predict_host(ctx, gh.model, np.ascontiguousarray(hu.goals), np.ascontiguousarray(hu.beta),
                       np.ascontiguousarray(obs), hu.n_obs, hu.uniform_log_prior(), N, T,
                       pm.make_grid(x0, y0, res, W, H), hu.seed, hu.human_id, post_out, counts, oob)
    np.testing.assert_array_equal(post_out, lb)
    np.testing.assert_array_equal(counts, want["counts"])
    np.testing.assert_array_equal(oob, want["oob"])


def test_async_host_api_in_a_pipeline(ctx, orc):
    """Five asynchronous host calls in a row (seeds and horizons vary, two
    sets of pinned outputs alternate, a larger grid midway forces a staging
    slot to grow): after the fence, each call's outputs equal the device path's
    for the same inputs. The inputs are pageable and are overwritten with NaN
    as soon as each call returns (a call reads them before it returns)."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    m, obs, post = _obs_and_post(orc, hu)
    gh = GpuHuman.of(hu)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    x0, y0, res, W, H = hu.grid
    N = 8000
    calls = [(60, hu.seed, W, H), (40, hu.seed + 1, W, H), (60, hu.seed + 2, W + 64, H + 32), (20, hu.seed + 3, W, H),
             (60, hu.seed + 4, W, H)]
    outs = []
    stream = torch.cuda.Stream()
    for i, (T, seed, Wc, Hc) in enumerate(calls):
        o = (torch.zeros(hu.G * hu.B, dtype=torch.float32).pin_memory(),
             torch.zeros((T, Hc, Wc), dtype=torch.int32).pin_memory(), torch.zeros(T, dtype=torch.int32).pin_memory())
        outs.append(o)
        ins = [np.array(hu.goals, np.float32), np.array(hu.beta, np.float32), np.array(obs, np.float32),
               np.array(hu.uniform_log_prior(), np.float32)]
        t_in = [torch.from_numpy(a) for a in ins]
        pm.pm_predict_host_async(ctx, gh.model, t_in[0], t_in[1], t_in[2], hu.n_obs, t_in[3], N, T,
                                 pm.make_grid(x0, y0, res, Wc, Hc), seed, hu.human_id, o[0], o[1], o[2], stream)
        for a in ins:
            a.fill(np.nan)
    pm.pm_host_fence(ctx, stream)
    stream.synchronize()
    for (T, seed, Wc, Hc), o in zip(calls, outs):
        want = predict(ctx, gh, lb, obs[-1], N, T, (x0, y0, res, Wc, Hc), seed, hu.human_id)
        np.testing.assert_array_equal(o[0].numpy(), lb)
        np.testing.assert_array_equal(o[1].numpy().view(np.uint32), want["counts"])
        np.testing.assert_array_equal(o[2].numpy().view(np.uint32), want["oob"])


def test_invalid_arguments_rejected(ctx):
    import paper_2603_01122_gb300 as pm
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    lb = dev(hu.uniform_log_prior())
    counts = torch.zeros((4, 100, 100), dtype=torch.int32, device="cuda:0")
    oob = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    g = pm.make_grid(*hu.grid)
    bad = [
        dict(n_particles=0), dict(horizon=0), dict(horizon=pm.PM_MAX_HORIZON + 1),
        dict(z0x=float("nan")), dict(grid=pm.make_grid(0, 0, 0.0, 10, 10)),
        dict(grid=pm.make_grid(0, 0, 0.1, 0, 10)), dict(grid=pm.make_grid(0, 0, 0.1, (1 << 22) + 1, 1)),
    ]
    for kw in bad:
        args = dict(n_particles=100, horizon=4, z0x=0.0, grid=g)
        args.update(kw)
        with pytest.raises(pm.PmError) as e:
            pm.pm_predict_occupancy(ctx, gh.model, lb, args["z0x"], 0.0, args["n_particles"],
                                    args["horizon"], args["grid"], 1, 1, counts, oob)
        assert e.value.status == pm.PM_EINVAL
    for field, val in [("K", 0), ("K", 65), ("G", 0), ("B", 300), ("dt", 0.0), ("speed", float("inf"))]:
        mm = pm.make_model(hu.K, hu.speed, hu.dt, gh.goals, gh.beta)
        setattr(mm, field, val)
        with pytest.raises(pm.PmError):
            pm.pm_predict_occupancy(ctx, mm, lb, 0.0, 0.0, 100, 4, g, 1, 1, counts, oob)
    mm = pm.make_model(hu.K, hu.speed, hu.dt, gh.goals, gh.beta, heading_off=0xFF)
    with pytest.raises(pm.PmError):
        pm.pm_update_posterior(ctx, mm, dev(np.zeros((3, 2), np.float32)), 2, lb)
    torch.cuda.synchronize()
    assert counts.sum().item() == 0  # nothing was queued
