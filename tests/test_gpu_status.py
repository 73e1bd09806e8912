"""Device status word: kernels latch the inputs they cannot use (non-finite
goals or beta, a NaN / +inf / empty log-belief, non-finite observed states or
trajectory points) and pm_sync_status reports and clears them. The work
around the bad input carries on: a NaN observed state skips its two steps,
and the belief equals the oracle's over the remaining steps."""
import math

import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev, posterior, predict
from test_gpu_parity import assert_posterior_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def _clear(pm, ctx):
    try:
        pm.pm_sync_status(ctx)
    except pm.PmError:
        pass


def _expect(pm, ctx, words):
    with pytest.raises(pm.PmError) as e:
        pm.pm_sync_status(ctx)
    assert e.value.status == pm.PM_EDEVICE
    for w in words:
        assert w in str(e.value), str(e.value)
    pm.pm_sync_status(ctx)  # cleared


def test_clean_calls_report_nothing(ctx, orc):
    import paper_2603_01122_gb300 as pm
    _clear(pm, ctx)
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    lb = posterior(ctx, gh, obs, hu.uniform_log_prior())
    predict(ctx, gh, lb, obs[-1], 2000, 10, hu.grid, 1, 2)
    pm.pm_sync_status(ctx)


@pytest.mark.parametrize("what", ["goal", "beta"])
def test_non_finite_model(ctx, what):
    import paper_2603_01122_gb300 as pm
    _clear(pm, ctx)
    hu = workloads.plain_small()
    goals, beta = hu.goals.copy(), hu.beta.copy()
    if what == "goal":
        goals[1, 0] = np.nan
    else:
        beta[2] = np.inf
    gh = GpuHuman(hu.K, hu.speed, hu.dt, goals, beta)
    out = predict(ctx, gh, hu.uniform_log_prior(), (0.0, 0.0), 1000, 5, hu.grid, 1, 2)
    assert np.all(out["counts"].reshape(5, -1).sum(1).astype(np.int64) + out["oob"] == 1000)
    _expect(pm, ctx, ["goal or beta"])


@pytest.mark.parametrize("kind", ["nan", "posinf", "empty"])
def test_bad_belief(ctx, kind):
    import paper_2603_01122_gb300 as pm
    _clear(pm, ctx)
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    lb = hu.uniform_log_prior().copy()
    if kind == "nan":
        lb[3] = np.nan
    elif kind == "posinf":
        lb[0] = np.inf
    else:
        lb[:] = -np.inf
    predict(ctx, gh, lb, (0.0, 0.0), 1000, 5, hu.grid, 1, 2)
    _expect(pm, ctx, ["log-belief"])


def test_nan_observation_skips_its_steps(ctx, orc):
    import paper_2603_01122_gb300 as pm
    _clear(pm, ctx)
    hu = workloads.paper_scale()
    gh = GpuHuman.of(hu)
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    bad = obs.copy()
    t = 17
    bad[t, 1] = np.nan
    got = posterior(ctx, gh, bad, hu.uniform_log_prior())
    _expect(pm, ctx, ["observed state"])
    # the steps into and out of state t are skipped: the oracle over the two
    # remaining runs, one after the other (Eq. 3 composes over steps)
    mid, _ = orc.update_posterior(m, obs[:t].astype(np.float64), hu.uniform_log_prior())
    want, _ = orc.update_posterior(m, obs[t + 1:].astype(np.float64), mid)
    assert_posterior_close(got, want)


def test_nan_trajectory_point(ctx, orc):
    import paper_2603_01122_gb300 as pm
    _clear(pm, ctx)
    ts = workloads.differentiation()
    trajs = []
    for i in range(4):
        g = int(ts.true_goal[i])
        mm = orc.Model(ts.K, ts.speed, ts.dt, ts.goals[g:g + 1], [ts.true_beta[i]])
        trajs.append(orc.simulate(mm, 0, ts.starts[i], 30, ts.obs_seed, i).astype(np.float32))
    trajs[2][11, 0] = np.inf
    offsets = np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32)
    traj = np.concatenate(trajs)
    J = ts.goals.shape[0] * ts.beta.shape[0]
    g, b = dev(ts.goals), dev(ts.beta)
    model = pm.make_model(ts.K, ts.speed, ts.dt, g, b)
    L = torch.empty(1, device="cuda:0")
    pm.pm_loglik_forward(ctx, model, 4, dev(offsets, torch.int32), traj.shape[0], dev(traj),
                         dev(np.full(J, -math.log(J), np.float32)), L)
    assert math.isfinite(L.item())
    _expect(pm, ctx, ["trajectory point"])


def test_batch_latches_and_other_humans_are_unaffected(ctx, orc):
    import paper_2603_01122_gb300 as pm
    _clear(pm, ctx)
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    x0, y0, res, W, H = hu.grid
    grid = pm.make_grid(x0, y0, res, W, H)
    T, N = 8, 3000
    lbs = [dev(hu.uniform_log_prior()), dev(np.where(np.arange(6) == 2, np.nan, hu.uniform_log_prior()))]
    z0 = dev(np.float32([0.0, 0.0]))
    outs = [(torch.empty((T, H, W), dtype=torch.int32, device="cuda:0"),
             torch.empty(T, dtype=torch.int32, device="cuda:0")) for _ in range(2)]
    b = pm.pm_batch_create(ctx, pm.make_model(hu.K, hu.speed, hu.dt, gh.goals, gh.beta), 2)
    try:
        humans = [pm.make_human(gh.goals, gh.beta, lbs[i], z0, N, T, grid, 5, 70 + i, outs[i][0], outs[i][1])
                  for i in range(2)]
        pm.pm_batch_set(b, humans)
        pm.pm_batch_predict(b)
        _expect(pm, ctx, ["log-belief"])
        single = predict(ctx, gh, hu.uniform_log_prior(), (0.0, 0.0), N, T, hu.grid, 5, 70)
        np.testing.assert_array_equal(outs[0][0].cpu().numpy().view(np.uint32), single["counts"])
        pm.pm_sync_status(ctx)
    finally:
        pm.pm_batch_destroy(b)
