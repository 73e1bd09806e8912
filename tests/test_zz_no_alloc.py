"""The belief update that allocates nothing, checked against the context
path. Some callers cannot allocate device memory (a real-time loop that
forbids allocation after start-up, work enqueued under a stream capture
that rejects cudaMalloc, an application with its own memory pool); for
them the library offers pm_update_posterior_noalloc, whose scratch is a
static device array. This file is collected last so that a failure here
does not stop the rest of the suite from running first."""
import math

import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev

pytestmark = pytest.mark.gpu


def _close(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    big = np.exp(want) >= 1e-8
    assert np.all(np.abs(got[big] - want[big]) <= 1e-5)
    assert np.all(np.exp(got[~big]) <= 1e-7)


def test_noalloc_matches_context_path_twice(orc):
    import paper_2603_01122_gb300 as pm
    pm.build()
    ctx = pm.pm_create(0)
    try:
        cases = []
        hu = workloads.paper_scale()
        cases.append((hu, orc.simulate(orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta), hu.true_j,
                                       hu.start, hu.n_obs, hu.obs_seed, hu.human_id)))
        # second call: another model and a 200-step history with 256 components
        rng = np.random.default_rng(4)
        goals = rng.uniform(0, 10, (16, 2)).astype(np.float32)
        beta = workloads.beta_grid(-2.0, 2.0, 16)
        hu2 = workloads.Human(K=64, speed=1.0, dt=workloads.f32(0.05), goals=goals, beta=beta, true_j=37,
                              start=np.float32([5.0, 5.0]), n_obs=200, n_particles=1, horizon=1,
                              grid=(0, 0, 1, 1, 1), seed=0, human_id=3, obs_seed=3)
        cases.append((hu2, orc.simulate(orc.Model(64, 1.0, hu2.dt, goals, beta), 37, hu2.start, 200, 3, 3)))
        # third call: the several-speed control set (|U| = 96), history drawn at all speeds
        hu3 = workloads.multi_speed()
        cases.append((hu3, orc.simulate(orc.Model(hu3.K, hu3.speed, hu3.dt, hu3.goals, hu3.beta, speeds=hu3.speeds),
                                        hu3.true_j, hu3.start, hu3.n_obs, hu3.obs_seed, hu3.human_id)))
        for hu, obs in cases:
            gh = GpuHuman.of(hu, speeds=None if tuple(hu.speeds) == (1.0,) else hu.speeds)
            obs_d = dev(obs.astype(np.float32))
            prior = hu.uniform_log_prior()
            a = dev(prior)
            b = dev(prior)
            pm.pm_update_posterior(ctx, gh.model, obs_d, obs_d.shape[0] - 1, a)
            pm.pm_update_posterior_noalloc(gh.model, obs_d, obs_d.shape[0] - 1, b)
            torch.cuda.synchronize()
            _close(b.cpu().numpy(), a.cpu().numpy())
            assert abs(np.exp(b.cpu().numpy().astype(np.float64)).sum() - 1) <= 1e-6
    finally:
        pm.pm_destroy(ctx)


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
