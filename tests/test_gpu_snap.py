"""GPU parity of the snapped observed heading (the observed control read as
the nearest enabled heading, the discrete control of Eq. 2) against the FP64
oracle: the belief update, single and batched, and the log-likelihood with
its gradient, at one speed and at several. Every observed step is turned off
the heading lattice by up to 0.6 of half the spacing, never near a midpoint
between two headings, where the kernel's FP32 decision and the oracle's FP64
one could differ. The continuous reading of the same steps differs, so the
tests would fail if the flag were ignored."""
import math

import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev
from test_gpu_adjoint import check_grad
from test_gpu_parity import assert_posterior_close

pytestmark = pytest.mark.gpu
SPEEDS3 = (0.5, 1.0, 1.5)


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def _turned(obs, K, rng, frac=0.6):
    """The same steps, each turned by a uniform angle within frac * pi / K."""
    steps = np.diff(np.asarray(obs, np.float64), axis=0)
    a = rng.uniform(-frac, frac, steps.shape[0]) * math.pi / K
    c, s = np.cos(a), np.sin(a)
    rot = np.stack([c * steps[:, 0] - s * steps[:, 1], s * steps[:, 0] + c * steps[:, 1]], 1)
    return np.concatenate([obs[:1], obs[0] + np.cumsum(rot, 0)]).astype(np.float32)


@pytest.mark.parametrize("speeds", [None, SPEEDS3])
def test_posterior_matches_oracle(ctx, orc, speeds):
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    K = hu.K if speeds is None else 32
    sp = (1.0,) if speeds is None else speeds
    m0 = orc.Model(K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=sp)
    obs = _turned(orc.simulate(m0, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id), K,
                  np.random.default_rng(3))
    prior = hu.uniform_log_prior()
    want, _ = orc.update_posterior(orc.Model(K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=sp, snap=True),
                                   obs.astype(np.float64), prior)
    cont, _ = orc.update_posterior(m0, obs.astype(np.float64), prior)
    assert np.max(np.abs(want - cont)) > 1e-3
    gh = GpuHuman(K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=speeds, snap_heading=True)
    lb = dev(prior)
    pm.pm_update_posterior(ctx, gh.model, dev(obs), hu.n_obs, lb)
    torch.cuda.synchronize()
    assert_posterior_close(lb.cpu().numpy(), want)


def test_batched_posterior_equals_single(ctx, orc):
    """A batch whose shared model snaps: every human's belief equals the
    single-human call's, bit for bit."""
    import paper_2603_01122_gb300 as pm
    humans = workloads.batched()[:6]
    rng = np.random.default_rng(5)
    ds = []
    for hu in humans:
        m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
        obs = _turned(orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id), hu.K, rng)
        gh = GpuHuman.of(hu, snap_heading=True)
        ds.append(dict(hu=hu, gh=gh, obs=dev(obs), lb=dev(hu.uniform_log_prior()), z0=dev(obs[-1]),
                       counts=torch.empty((4, 8, 8), dtype=torch.int32, device="cuda:0"),
                       oob=torch.empty(4, dtype=torch.int32, device="cuda:0")))
    b = pm.pm_batch_create(ctx, ds[0]["gh"].model, len(ds))
    try:
        x0, y0, res = humans[0].grid[:3]
        pm.pm_batch_set(b, [pm.make_human(d["gh"].goals, d["gh"].beta, d["lb"], d["z0"], 64, 4,
                                          pm.make_grid(x0, y0, res, 8, 8), d["hu"].seed, d["hu"].human_id,
                                          d["counts"], d["oob"], obs_xy=d["obs"], n_obs=d["hu"].n_obs)
                            for d in ds])
        singles = []
        for d in ds:
            lb = dev(d["hu"].uniform_log_prior())
            pm.pm_update_posterior(ctx, d["gh"].model, d["obs"], d["hu"].n_obs, lb)
            singles.append(lb)
        pm.pm_batch_update_posterior(b)
        torch.cuda.synchronize()
        for d, lb in zip(ds, singles):
            assert torch.equal(d["lb"], lb)
    finally:
        pm.pm_batch_destroy(b)


def _trajectories(orc, ts, K, M, speeds, rng, mask_off=0):
    """Model-drawn trajectories (no disabled heading is ever taken, so no step
    lies midway between two enabled headings), each step turned."""
    trajs = []
    for i in range(M):
        g = int(ts.true_goal[i])
        mm = orc.Model(K, ts.speed, ts.dt, ts.goals[g:g + 1], [ts.true_beta[i]], speeds=speeds, mask_off=mask_off)
        trajs.append(_turned(orc.simulate(mm, 0, ts.starts[i], int(ts.lengths[i]), ts.obs_seed, i), K, rng))
    offsets = np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32)
    return offsets, np.concatenate(trajs)


@pytest.mark.parametrize("case", ["K36", "K36_speeds", "K37_mask"])
def test_adjoint_matches_oracle(ctx, orc, case):
    """The log-likelihood and gradient (goals, v, w2; w1 too with several
    speeds) with snapped controls, on the packed all-headings path, the
    several-speed path and the general path with a disabled heading."""
    import paper_2603_01122_gb300 as pm
    ts = workloads.differentiation()
    K, speeds, heading_off = {"K36": (36, None, 0), "K36_speeds": (32, SPEEDS3, 0),
                              "K37_mask": (37, None, (1 << 5) | (1 << 30))}[case]
    sp = (1.0,) if speeds is None else speeds
    offsets, traj = _trajectories(orc, ts, K, 24, sp, np.random.default_rng(11), heading_off)
    prior = np.log(np.random.default_rng(2).dirichlet(np.ones(40))).astype(np.float32)
    m = orc.Model(K, ts.speed, ts.dt, ts.goals, ts.beta, w1=0.9, w2=1.2, mask_off=heading_off, speeds=sp,
                  snap=True)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    g, b = dev(ts.goals), dev(ts.beta)
    model = pm.make_model(K, ts.speed, ts.dt, g, b, w1=0.9, w2=1.2, heading_off=heading_off, speeds=speeds,
                          snap_heading=True)
    L = torch.empty(1, device="cuda:0")
    dg = torch.empty_like(g)
    dv = torch.empty(1, device="cuda:0")
    dw = torch.empty(2, device="cuda:0")
    pm.pm_loglik_backward(ctx, model, len(offsets) - 1, dev(offsets, torch.int32), traj.shape[0], dev(traj),
                          dev(prior), 1.0, L, dg, dv, dw)
    torch.cuda.synchronize()
    assert abs(L.item() - L64) <= 1e-6 * abs(L64), (L.item(), L64)
    want = [dg64.ravel(), [dv64, dw64[1]]] + ([[dw64[0]]] if speeds else [])
    got = [dg.cpu().numpy().ravel(), [dv.item(), dw[1].item()]] + ([[dw[0].item()]] if speeds else [])
    check_grad(np.concatenate(got), np.concatenate(want))


def test_autograd_passes_the_flag(ctx, orc):
    """marginal_loglik(..., snap_heading=True): the value and the gradient
    equal the oracle's snapped ones."""
    from paper_2603_01122_gb300.autograd import marginal_loglik
    ts = workloads.differentiation()
    offsets, traj = _trajectories(orc, ts, 36, 12, (1.0,), np.random.default_rng(19))
    prior = np.full(40, -math.log(40.0), np.float32)
    goals = dev(ts.goals).requires_grad_(True)
    speed = torch.tensor(ts.speed, dtype=torch.float32, requires_grad=True)
    w = torch.tensor([1.0, 1.0], dtype=torch.float32, requires_grad=True)
    L = marginal_loglik(goals, speed, w, dev(ts.beta), 36, ts.dt, dev(offsets, torch.int32), dev(traj),
                        dev(prior), ctx, snap_heading=True)
    L.backward()
    m = orc.Model(36, ts.speed, ts.dt, ts.goals, ts.beta, snap=True)
    L64, dg64, dv64, _ = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    assert abs(L.item() - L64) <= 1e-6 * abs(L64)
    check_grad(np.concatenate([goals.grad.cpu().numpy().ravel(), [speed.grad.item()]]),
               np.concatenate([dg64.ravel(), [dv64]]))


def test_invalid_flag_rejected(ctx):
    import paper_2603_01122_gb300 as pm
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    gh.model.snap_heading = 2
    with pytest.raises(pm.PmError):
        pm.pm_update_posterior(ctx, gh.model, dev(np.zeros((2, 2), np.float32)), 1, dev(hu.uniform_log_prior()))
