"""Several speeds with stationary masking (controls = speeds x headings,
Sec. IV-B) on the GPU against the FP64 oracle: trajectories and histograms of
the rollout, the belief update, the batched launch and the adjoint.

Tolerances. Trajectories: at most 1e-4 of the particles diverge from the
oracle taking its draws at the FP32 state (as in test_gpu_parity), bit-identical
FP32 states for every particle whose draws agree, and every particle whose
draws differ must differ at a draw that the error budget explains
(``gpu_util.explain_divergences``): its uniform lies within the budget of a
boundary of the exact CDF between the two choices. Histograms
bit-exact given the states; |log b| within 1e-5; L relative 1e-6; gradients
relative 1e-3 in norm.
"""
import zlib

import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev, explain_divergences, posterior, predict
from test_gpu_parity import assert_posterior_close, compare_trajectories, poisson_reject_at, trajectory_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def _models(orc, K, speed, dt, goals, beta, speeds, speed_off=0, w1=1.0, w2=1.0, heading_off=0):
    m = orc.Model(K, speed, dt, goals, beta, w1=w1, w2=w2, mask_off=heading_off, speeds=speeds,
                  speed_off=speed_off)
    gh = GpuHuman(K, speed, dt, goals, beta, w1=w1, w2=w2, heading_off=heading_off, speeds=speeds,
                  speed_off=speed_off)
    return m, gh


CASES = ["U96", "stationary", "U256", "K36_U108", "one_mult", "w1_3", "beta_neg_large", "beta_large", "ragged"]


@pytest.mark.parametrize("case", CASES)
def test_trajectories_and_histogram(ctx, orc, case):
    hu = workloads.multi_speed(stationary=(case == "stationary"))
    K, speeds, speed_off, goals, beta, w1 = hu.K, hu.speeds, hu.speed_off, hu.goals, hu.beta, 1.0
    N, T, z0, grid = 3001, 40, np.float32([5.0, 5.0]), hu.grid
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    if case == "U256":
        K, speeds = 64, (0.25, 0.5, 1.0, 2.0)
    elif case == "K36_U108":
        K = 36
    elif case == "one_mult":
        K, speeds = 8, (1.5,)
    elif case == "w1_3":
        w1 = 3.0
    elif case == "beta_neg_large":
        beta = np.float32([-300.0, -20.0])
    elif case == "beta_large":
        beta = np.float32([1e4, 300.0])
    elif case == "ragged":
        N = 257 * 13 + 5
    m, gh = _models(orc, K, hu.speed, hu.dt, goals, beta, speeds, speed_off, w1=w1)
    J = m.G * m.B
    lb = np.log(rng.dirichlet(np.ones(J))).astype(np.float32)
    got = predict(ctx, gh, lb, z0, N, T, grid, 77, 5, n_trace=N)
    d, _, _ = trajectory_parity(orc, m, lb, z0, T, 77, 5, got, N, f"several speeds {case}")
    assert d < poisson_reject_at(N), d  # at most 1e-4 of particles, over the whole horizon
    c, o = orc.bin_states(got["states32"], grid)
    np.testing.assert_array_equal(got["counts"], c)
    np.testing.assert_array_equal(got["oob"], o)
    assert np.all(got["counts"].reshape(T, -1).sum(1).astype(np.int64) + got["oob"] == N)
    u = got["headings"].astype(np.int64)
    assert u.max() < len(speeds) * K
    if speed_off:
        assert np.all(((speed_off >> (u // K)) & 1) == 0)  # no masked speed is ever drawn
    elif len(speeds) > 1 and case != "beta_large":
        assert len(np.unique(u // K)) == len(speeds)  # every speed is drawn


@pytest.mark.parametrize("stationary", [False, True])
def test_full_launch_sampled_particles(ctx, orc, stationary):
    """The |U| = 96 workload at full size (N = 100k, T = 150, the bench's
    several-speed configuration), with and without the stationary mask, the
    first 20000 particles traced and recomputed one by one: at most 1e-4 of
    them may diverge."""
    hu = workloads.multi_speed(stationary=stationary)
    gen = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=hu.speeds)
    m, gh = _models(orc, hu.K, hu.speed, hu.dt, hu.goals, hu.beta, hu.speeds, hu.speed_off)
    obs = orc.simulate(gen, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    z0 = obs[-1]
    N, T, n = hu.n_particles, hu.horizon, 20000
    got = predict(ctx, gh, lb, z0, N, T, hu.grid, hu.seed, hu.human_id, n_trace=n)
    label = "|U| = 96 full launch" + (" (stationary mask)" if stationary else "")
    d, _, _ = trajectory_parity(orc, m, lb, z0, T, hu.seed, hu.human_id, got, n, label)
    assert d <= 1e-4 * n, d
    assert np.all(got["counts"].reshape(T, -1).sum(1).astype(np.int64) + got["oob"] == N)
    c_sub, _ = orc.bin_states(got["states32"], hu.grid)
    assert np.all(c_sub <= got["counts"])


@pytest.mark.parametrize("stationary", [False, True])
def test_posterior_matches_oracle(ctx, orc, stationary):
    """Histories drawn at all three speeds; with the stationary mask every
    observed step snaps to the one enabled (slow) speed."""
    hu = workloads.multi_speed(stationary=stationary)
    gen = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=hu.speeds)
    obs = orc.simulate(gen, hu.true_j, hu.start, 200, hu.obs_seed, hu.human_id).astype(np.float32)
    m, gh = _models(orc, hu.K, hu.speed, hu.dt, hu.goals, hu.beta, hu.speeds, hu.speed_off)
    # no observed step within 1e-4 of a midpoint between two multipliers (the
    # two sides snap in different precisions)
    ln = np.hypot(*np.diff(obs.astype(np.float64), axis=0).T) / (hu.speed * hu.dt)
    assert np.min(np.abs(ln[:, None] - np.array([0.75, 1.25])[None, :])) > 1e-4
    want, _ = orc.update_posterior(m, obs.astype(np.float64), hu.uniform_log_prior())
    got = posterior(ctx, gh, obs, hu.uniform_log_prior())
    assert_posterior_close(got, want)


def test_batch_equals_single(ctx, orc):
    """Four humans under one shared |U| = 96 model, two with their own speed
    masks (one standing still): the batched belief update and histograms equal
    the single-human calls under the same masks bit for bit."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.multi_speed()
    rng = np.random.default_rng(9)
    masks = [0, 0b110, 0, 0b001]
    ds = []
    for h in range(4):
        goals = rng.uniform(0, 10, size=(2 + h, 2)).astype(np.float32)
        m, gh = _models(orc, hu.K, hu.speed, hu.dt, goals, hu.beta, hu.speeds, speed_off=masks[h])
        start = rng.uniform(2, 8, size=2).astype(np.float32)
        obs = orc.simulate(m, h, start, 30, hu.obs_seed, 40 + h).astype(np.float32)
        N, T = int(rng.integers(5000, 40000)), int(rng.integers(20, 80))
        x0, y0, res, W, H = hu.grid
        lb = np.full(m.G * m.B, -np.log(m.G * m.B), np.float32)
        ds.append(dict(gh=gh, obs=dev(obs), n_obs=obs.shape[0] - 1, N=N, T=T, lb=dev(lb), z0=dev(obs[-1]),
                       grid=pm.make_grid(x0, y0, res, W, H), human=40 + h, counts=torch.empty((T, H, W), dtype=torch.int32, device="cuda:0"),
                       oob=torch.empty(T, dtype=torch.int32, device="cuda:0")))
    shared = pm.make_model(hu.K, hu.speed, hu.dt, ds[0]["gh"].goals, ds[0]["gh"].beta, speeds=hu.speeds)
    b = pm.pm_batch_create(ctx, shared, len(ds))
    try:
        singles = []
        for d in ds:
            lb = d["lb"].clone()
            pm.pm_update_posterior(ctx, d["gh"].model, d["obs"], d["n_obs"], lb)
            counts = torch.empty_like(d["counts"])
            oob = torch.empty_like(d["oob"])
            z0 = d["z0"].cpu().numpy()
            pm.pm_predict_occupancy(ctx, d["gh"].model, lb, float(z0[0]), float(z0[1]), d["N"], d["T"],
                                    d["grid"], hu.seed, d["human"], counts, oob)
            singles.append((lb.cpu().numpy(), counts.cpu().numpy(), oob.cpu().numpy()))
        humans = [pm.make_human(d["gh"].goals, d["gh"].beta, d["lb"], d["z0"], d["N"], d["T"], d["grid"],
                                hu.seed, d["human"], d["counts"], d["oob"], obs_xy=d["obs"], n_obs=d["n_obs"],
                                speed_off=mk)
                  for d, mk in zip(ds, masks)]
        for bad in (0b111, 0b1000 | 0b111):  # every speed of a human disabled
            h0 = humans[0]
            h0.speed_off = bad
            with pytest.raises(pm.PmError) as e:
                pm.pm_batch_set(b, humans)
            assert e.value.status == pm.PM_EINVAL
            h0.speed_off = 0
        pm.pm_batch_set(b, humans)
        pm.pm_batch_update_posterior(b)
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d, (lb1, c1, o1) in zip(ds, singles):
            np.testing.assert_array_equal(d["lb"].cpu().numpy(), lb1)
            np.testing.assert_array_equal(d["counts"].cpu().numpy(), c1)
            np.testing.assert_array_equal(d["oob"].cpu().numpy(), o1)
        with pytest.raises(pm.PmError) as e:
            pm.pm_batch_set_config(b, 256, 1, 0, 48)  # several speeds: warp emplacement only
        assert e.value.status == pm.PM_EINVAL
        pm.pm_batch_autotune(b)
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d, (_, c1, _) in zip(ds, singles):
            np.testing.assert_array_equal(d["counts"].cpu().numpy(), c1)
        # reachable-cell zeroing under several speeds (the fastest one, 1.5 v,
        # sets the boxes), with the starts moved on the device between calls
        pm.pm_batch_set_zeroing(b, 1)
        for step in range(3):
            for i, d in enumerate(ds):
                if step:
                    d["z0"].add_(torch.tensor([0.3 * (i + 1), -0.45 * step], device="cuda:0"))
            pm.pm_batch_predict(b)
            torch.cuda.synchronize()
            for d, (lb1, _, _) in zip(ds, singles):
                counts = torch.empty_like(d["counts"])
                oob = torch.empty_like(d["oob"])
                z0 = d["z0"].cpu().numpy()
                pm.pm_predict_occupancy(ctx, d["gh"].model, dev(lb1), float(z0[0]), float(z0[1]), d["N"], d["T"],
                                        d["grid"], hu.seed, d["human"], counts, oob)
                torch.cuda.synchronize()
                assert torch.equal(d["counts"], counts) and torch.equal(d["oob"], oob)
    finally:
        pm.pm_batch_destroy(b)


SPEEDS3 = (0.5, 1.0, 1.5)


def _speed_trajectories(orc, ts, K, M):
    """M observed trajectories of the differentiation workload, drawn with
    the three-speed control set over K headings."""
    trajs = []
    for i in range(M):
        g = int(ts.true_goal[i])
        mm = orc.Model(K, ts.speed, ts.dt, ts.goals[g:g + 1], [ts.true_beta[i]], speeds=SPEEDS3)
        trajs.append(orc.simulate(mm, 0, ts.starts[i], int(ts.lengths[i]), ts.obs_seed, i).astype(np.float32))
    return np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32), np.concatenate(trajs)


def test_adjoint_matches_oracle(ctx, orc):
    """Marginal log-likelihood and its gradient with three speeds; dL/dw1 is
    nonzero (identifiable) and matches the oracle."""
    import paper_2603_01122_gb300 as pm
    ts = workloads.differentiation()
    speeds = SPEEDS3
    M = 48
    K = ts.K - 4  # 32: a multiple of 4
    offsets, traj = _speed_trajectories(orc, ts, K, M)
    prior = np.full(ts.goals.shape[0] * ts.beta.shape[0], -np.log(ts.goals.shape[0] * ts.beta.shape[0]))
    m = orc.Model(K, ts.speed, ts.dt, ts.goals, ts.beta, w1=0.7, w2=1.3, speeds=speeds)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    g = dev(ts.goals)
    b = dev(ts.beta)
    model = pm.make_model(K, ts.speed, ts.dt, g, b, w1=0.7, w2=1.3, speeds=speeds)
    L = torch.empty(1, device="cuda:0")
    dg = torch.empty_like(g)
    dv = torch.empty(1, device="cuda:0")
    dw = torch.empty(2, device="cuda:0")
    pm.pm_loglik_backward(ctx, model, M, dev(offsets, torch.int32), traj.shape[0], dev(traj), dev(prior), 1.0,
                          L, dg, dv, dw)
    torch.cuda.synchronize()
    assert abs(L.item() - L64) <= 1e-6 * abs(L64)
    got = np.concatenate([dg.cpu().numpy().ravel(), [dv.item()], dw.cpu().numpy()])
    want = np.concatenate([dg64.ravel(), [dv64], dw64])
    gnorm = np.linalg.norm(want)
    assert np.linalg.norm(got - want) <= 1e-3 * gnorm, (got, want)
    ok = np.abs(got - want) <= np.maximum(1e-2 * np.abs(want), 1e-4 * gnorm)
    assert ok.all(), (got, want)
    assert abs(dw64[0]) > 1e-3  # dL/dw1 is identifiable with several speeds


def test_autograd_with_speeds(ctx, orc):
    """The autograd Function over the several-speed adjoint: all of goals,
    speed and both Q weights receive the oracle's gradient."""
    from paper_2603_01122_gb300.autograd import marginal_loglik
    ts = workloads.differentiation()
    K = ts.K - 4
    offsets, traj = _speed_trajectories(orc, ts, K, 24)
    J = ts.goals.shape[0] * ts.beta.shape[0]
    prior = np.full(J, -np.log(J), np.float32)
    goals = dev(ts.goals).requires_grad_(True)
    speed = torch.tensor(ts.speed, requires_grad=True)
    w = torch.tensor([1.2, 0.8], requires_grad=True)
    L = marginal_loglik(goals, speed, w, dev(ts.beta), K, ts.dt, dev(offsets, torch.int32), dev(traj), dev(prior),
                        ctx, speeds=SPEEDS3)
    (-1.5 * L).backward()
    m = orc.Model(K, ts.speed, ts.dt, ts.goals, ts.beta, w1=1.2, w2=0.8, speeds=SPEEDS3)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    assert abs(L.item() - L64) <= 1e-6 * abs(L64)
    got = np.concatenate([goals.grad.cpu().numpy().ravel(), [speed.grad.item()], w.grad.numpy()])
    want = -1.5 * np.concatenate([dg64.ravel(), [dv64], dw64])
    gnorm = np.linalg.norm(want)
    assert np.linalg.norm(got - want) <= 1e-3 * gnorm, (got, want)


def test_rejected_speed_sets(ctx):
    import paper_2603_01122_gb300 as pm
    g = dev(np.float32([[1.0, 2.0]]))
    b = dev(np.float32([1.0]))
    lb = dev(np.float32([0.0]))
    counts = torch.empty((2, 4, 4), dtype=torch.int32, device="cuda:0")
    oob = torch.empty(2, dtype=torch.int32, device="cuda:0")
    grid = pm.make_grid(0.0, 0.0, 0.1, 4, 4)
    bad = [dict(K=30, speeds=(0.5, 1.0)),                   # K not a multiple of 4
           dict(K=32, speeds=(0.5, 1.0), heading_off=0b1),  # a heading disabled
           dict(K=32, speeds=(0.5, 1.0), speed_off=0b11),   # every speed disabled
           dict(K=32, speeds=(0.5, -1.0)),                  # a multiplier <= 0
           dict(K=32, speeds=(0.5, float("nan")))]
    for kw in bad:
        model = pm.make_model(kw["K"], 1.0, 0.1, g, b, heading_off=kw.get("heading_off", 0), speeds=kw["speeds"],
                              speed_off=kw.get("speed_off", 0))
        with pytest.raises(pm.PmError) as e:
            pm.pm_predict_occupancy(ctx, model, lb, 0.0, 0.0, 16, 2, grid, 1, 0, counts, oob)
        assert e.value.status == pm.PM_EINVAL, kw


def test_rollout_half_after_zeroing_several_speeds(ctx, orc):
    """The several-speed kernel through the two halves: pm_zero_occupancy on a
    second stream, then pm_rollout_occupancy, three times in a row (each launch
    leaves the chunk counter at zero for the next); every call equals
    pm_predict_occupancy."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.multi_speed()
    m, gh = _models(orc, hu.K, hu.speed, hu.dt, hu.goals, hu.beta, hu.speeds)
    x0, y0, res, W, H = hu.grid
    grid = pm.make_grid(x0, y0, res, W, H)
    N, T = 20000, 40
    lb = dev(hu.uniform_log_prior())
    want = torch.empty((T, H, W), dtype=torch.int32, device="cuda:0")
    want_oob = torch.empty(T, dtype=torch.int32, device="cuda:0")
    pm.pm_predict_occupancy(ctx, gh.model, lb, float(hu.start[0]), float(hu.start[1]), N, T, grid, hu.seed, 3,
                            want, want_oob)
    got = torch.full_like(want, 0x3C3C3C3C)
    got_oob = torch.full_like(want_oob, 5)
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        side.wait_stream(main)
        pm.pm_zero_occupancy(ctx, T, grid, got, got_oob, side)
        main.wait_stream(side)
        pm.pm_rollout_occupancy(ctx, gh.model, lb, float(hu.start[0]), float(hu.start[1]), N, T, grid, hu.seed, 3,
                                got, got_oob, main)
        torch.cuda.synchronize()
        assert torch.equal(got, want) and torch.equal(got_oob, want_oob)
