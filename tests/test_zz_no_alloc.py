"""The belief update that allocates nothing, checked against the oracle and
against the context path. Some callers cannot allocate device memory (a
real-time loop that forbids allocation after start-up, work enqueued under a
stream capture that rejects cudaMalloc, an application with its own memory
pool); for them the library offers pm_update_posterior_noalloc, whose scratch
is a static device array. This file is collected last so that a failure here
does not stop the rest of the suite from running first.

Tolerances: the A14 reading of the posterior tolerance (|log b - log b_64| <=
1e-5 where b_64 >= 1e-8, else b <= 1e-7, |sum b - 1| <= 1e-6) against the
FP64 oracle, and the same bounds against the context call."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev
from test_gpu_parity import assert_posterior_close

pytestmark = pytest.mark.gpu


def _cases(orc):
    """(human, observed history, oracle model) for the three calls in a row."""
    cases = []
    hu = workloads.paper_scale()
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    cases.append((hu, orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id), m))
    # another model and a 200-step history with 256 components
    rng = np.random.default_rng(4)
    goals = rng.uniform(0, 10, (16, 2)).astype(np.float32)
    beta = workloads.beta_grid(-2.0, 2.0, 16)
    hu2 = workloads.Human(K=64, speed=1.0, dt=workloads.f32(0.05), goals=goals, beta=beta, true_j=37,
                          start=np.float32([5.0, 5.0]), n_obs=200, n_particles=1, horizon=1,
                          grid=(0, 0, 1, 1, 1), seed=0, human_id=3, obs_seed=3)
    m2 = orc.Model(64, 1.0, hu2.dt, goals, beta)
    cases.append((hu2, orc.simulate(m2, 37, hu2.start, 200, 3, 3), m2))
    # the several-speed control set (|U| = 96), history drawn at all speeds
    hu3 = workloads.multi_speed()
    m3 = orc.Model(hu3.K, hu3.speed, hu3.dt, hu3.goals, hu3.beta, speeds=hu3.speeds)
    cases.append((hu3, orc.simulate(m3, hu3.true_j, hu3.start, hu3.n_obs, hu3.obs_seed, hu3.human_id), m3))
    return cases


def _gpu_human(hu):
    return GpuHuman.of(hu, speeds=None if tuple(hu.speeds) == (1.0,) else hu.speeds)


def test_noalloc_matches_oracle_and_context_path(orc):
    import paper_2603_01122_gb300 as pm
    pm.build()
    ctx = pm.pm_create(0)
    try:
        for hu, obs, m in _cases(orc):
            obs = obs.astype(np.float32)
            gh = _gpu_human(hu)
            obs_d = dev(obs)
            prior = hu.uniform_log_prior()
            a = dev(prior)
            b = dev(prior)
            pm.pm_update_posterior(ctx, gh.model, obs_d, obs_d.shape[0] - 1, a)
            pm.pm_update_posterior_noalloc(gh.model, obs_d, obs_d.shape[0] - 1, b)
            torch.cuda.synchronize()
            want, _ = orc.update_posterior(m, obs.astype(np.float64), prior)
            assert_posterior_close(b.cpu().numpy(), want)                   # Eq. 3 / Eq. 7, A14
            assert_posterior_close(b.cpu().numpy(), a.cpu().numpy().astype(np.float64))
    finally:
        pm.pm_destroy(ctx)


def test_noalloc_replays_from_a_captured_graph(orc):
    """The stated use: after one call outside any capture, the call is
    captured in the global capture mode (which rejects allocation) and the
    graph replayed twice; each replay equals the context path's result."""
    import paper_2603_01122_gb300 as pm
    pm.build()
    ctx = pm.pm_create(0)
    try:
        hu, obs, m = _cases(orc)[0]
        gh = _gpu_human(hu)
        obs_d = dev(obs.astype(np.float32))
        prior = dev(hu.uniform_log_prior())
        ref = prior.clone()
        pm.pm_update_posterior(ctx, gh.model, obs_d, obs_d.shape[0] - 1, ref)
        lb = prior.clone()
        pm.pm_update_posterior_noalloc(gh.model, obs_d, obs_d.shape[0] - 1, lb)  # first call: outside
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
                lb.copy_(prior)
                pm.pm_update_posterior_noalloc(gh.model, obs_d, obs_d.shape[0] - 1, lb, s)
        want, _ = orc.update_posterior(m, obs.astype(np.float64), hu.uniform_log_prior())
        for _ in range(2):
            lb.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            assert_posterior_close(lb.cpu().numpy(), ref.cpu().numpy().astype(np.float64))
            assert_posterior_close(lb.cpu().numpy(), want)
    finally:
        pm.pm_destroy(ctx)


def test_noalloc_skips_a_nan_observation(orc):
    """A non-finite observed state is not reported (no status word) but its
    two steps are skipped as in the context call: the belief equals the
    oracle's over the two remaining runs of steps."""
    import paper_2603_01122_gb300 as pm
    hu, obs, m = _cases(orc)[0]
    obs = obs.astype(np.float32)
    gh = _gpu_human(hu)
    bad = obs.copy()
    t = 17
    bad[t, 0] = np.nan
    lb = dev(hu.uniform_log_prior())
    obs_d = dev(bad)
    pm.pm_update_posterior_noalloc(gh.model, obs_d, obs_d.shape[0] - 1, lb)
    torch.cuda.synchronize()
    mid, _ = orc.update_posterior(m, obs[:t].astype(np.float64), hu.uniform_log_prior())
    want, _ = orc.update_posterior(m, obs[t + 1:].astype(np.float64), mid)
    assert_posterior_close(lb.cpu().numpy(), want)


def test_noalloc_rejects_oversized_model():
    import paper_2603_01122_gb300 as pm
    g = torch.zeros((17, 2), device="cuda:0")
    b = torch.ones(16, device="cuda:0")
    model = pm.make_model(8, 1.0, 0.1, g, b)           # G*B = 272 > 256
    lb = torch.zeros(272, device="cuda:0")
    obs = torch.zeros((3, 2), device="cuda:0")
    with pytest.raises(pm.PmError) as e:
        pm.pm_update_posterior_noalloc(model, obs, 2, lb)
    assert e.value.status == pm.PM_EINVAL
    assert "256" in str(e.value)
