"""GPU parity of the log-likelihood and its adjoint against the FP64 oracle.

Tolerances: L relative 1e-6; gradient vector relative 1e-3 in norm and each
component within 1e-2 relative or 1e-4 * ||grad||; dL/dw1 (zero in exact
arithmetic) within 1e-5 * ||grad||.
"""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def trajectories(orc, ts: workloads.TrajectorySet, M=None):
    M = ts.M if M is None else M
    trajs = []
    for m in range(M):
        mm = orc.Model(ts.K, ts.speed, ts.dt, ts.goals[ts.true_goal[m]:ts.true_goal[m] + 1],
                       [ts.true_beta[m]])
        trajs.append(orc.simulate(mm, 0, ts.starts[m], int(ts.lengths[m]), ts.obs_seed, m).astype(np.float32))
    offsets = np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32)
    return offsets, np.concatenate(trajs)


def gpu_loglik(ctx, ts, offsets, traj, prior, goals=None, speed=None, w=(1.0, 1.0), grad=True):
    import paper_2603_01122_gb300 as pm
    goals = ts.goals if goals is None else goals
    speed = ts.speed if speed is None else speed
    g = dev(goals)
    b = dev(ts.beta)
    model = pm.make_model(ts.K, speed, ts.dt, g, b, w1=w[0], w2=w[1])
    off = dev(offsets, torch.int32)
    tr = dev(traj)
    lp = dev(prior)
    L = torch.empty(1, device="cuda:0")
    if not grad:
        pm.pm_loglik_forward(ctx, model, len(offsets) - 1, off, traj.shape[0], tr, lp, L)
        torch.cuda.synchronize()
        return float(L.item())
    dg = torch.empty_like(g)
    dv = torch.empty(1, device="cuda:0")
    dw = torch.empty(2, device="cuda:0")
    pm.pm_loglik_backward(ctx, model, len(offsets) - 1, off, traj.shape[0], tr, lp, 1.0, L, dg, dv, dw)
    torch.cuda.synchronize()
    return float(L.item()), dg.cpu().numpy(), float(dv.item()), dw.cpu().numpy()


def check_grad(got, want):
    gnorm = np.linalg.norm(want)
    assert np.linalg.norm(got - want) <= 1e-3 * gnorm, (got, want)
    ok = np.abs(got - want) <= np.maximum(1e-2 * np.abs(want), 1e-4 * gnorm)
    assert ok.all(), (got, want)


@pytest.mark.parametrize("M", [16, 256])
def test_loglik_and_gradient_match_oracle(ctx, orc, M):
    ts = workloads.differentiation()
    offsets, traj = trajectories(orc, ts, M)
    prior = np.full(ts.goals.shape[0] * ts.beta.shape[0], -np.log(40.0), np.float32)
    m = orc.Model(ts.K, ts.speed, ts.dt, ts.goals, ts.beta)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    L, dg, dv, dw = gpu_loglik(ctx, ts, offsets, traj, prior)
    assert abs(L - L64) <= 1e-6 * abs(L64), (L, L64)
    want = np.concatenate([dg64.ravel(), [dv64, dw64[1]]])
    got = np.concatenate([dg.ravel(), [dv, dw[1]]])
    check_grad(got, want)
    assert abs(dw[0]) <= 1e-5 * np.linalg.norm(want)
    assert gpu_loglik(ctx, ts, offsets, traj, prior, grad=False) == L


def test_gradient_other_weights_and_prior(ctx, orc):
    ts = workloads.differentiation()
    offsets, traj = trajectories(orc, ts, 24)
    rng = np.random.default_rng(2)
    prior = np.log(rng.dirichlet(np.ones(40))).astype(np.float32)
    m = orc.Model(ts.K, 1.3, ts.dt, ts.goals, ts.beta, w1=0.7, w2=1.6)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    L, dg, dv, dw = gpu_loglik(ctx, ts, offsets, traj, prior, speed=1.3, w=(0.7, 1.6))
    assert abs(L - L64) <= 1e-6 * abs(L64)
    check_grad(np.concatenate([dg.ravel(), [dv, dw[1]]]), np.concatenate([dg64.ravel(), [dv64, dw64[1]]]))


def test_deterministic_and_ragged(ctx, orc):
    """A trajectory with a stationary step, an empty one and a one-point one."""
    ts = workloads.differentiation()
    offsets, traj = trajectories(orc, ts, 7)
    parts = [traj[offsets[i]:offsets[i + 1]] for i in range(7)]
    t0 = parts[0]
    parts[0] = np.concatenate([t0[:5], t0[4:5], t0[5:]])  # repeated point: zero displacement
    parts.insert(1, np.zeros((0, 2), np.float32))          # no points
    parts.insert(2, parts[3][:1])                          # one point, no step
    offsets = np.cumsum([0] + [len(p) for p in parts]).astype(np.int32)
    traj = np.concatenate(parts).astype(np.float32)
    prior = np.full(40, -np.log(40.0), np.float32)
    m = orc.Model(ts.K, ts.speed, ts.dt, ts.goals, ts.beta)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    a = gpu_loglik(ctx, ts, offsets, traj, prior)
    b = gpu_loglik(ctx, ts, offsets, traj, prior)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2] and np.array_equal(a[3], b[3])
    assert abs(a[0] - L64) <= 1e-6 * abs(L64)
    check_grad(np.concatenate([a[1].ravel(), [a[2], a[3][1]]]), np.concatenate([dg64.ravel(), [dv64, dw64[1]]]))


@pytest.mark.parametrize("K,sign", [(8, 1.0), (5, 1.0), (8, -1.0)])
def test_large_beta_takes_the_second_pass(ctx, orc, K, sign):
    """beta w2 s large against K: the bound on the largest logit is loose at
    many steps (the sum of the bound-normalised weights below 2^-8), so those
    steps are normalised by their largest logit in a second pass. K = 8 takes
    the packed form, K = 5 the scalar one; sign -1 walks away from the goals.
    Tolerance on L: the relative 1e-6 plus, per step, what the FP32 inputs
    allow at this beta: a heading vector rounded to FP32 (the table's e_k, the
    observed e_o = dz/|dz|) moves d = ||p + s e|| by at most s |de|, so a
    logit beta w2 (d_o - d_k) by at most |beta| w2 s 2^-21, plus 4e-6 of
    arithmetic rounding. The gradient keeps the A15 bounds."""
    from types import SimpleNamespace
    rng = np.random.default_rng(9)
    goals = rng.uniform(2.0, 8.0, size=(3, 2)).astype(np.float32)
    beta = (sign * np.array([300.0, 1000.0, 1500.0])).astype(np.float32)
    ts = SimpleNamespace(K=K, speed=2.0, dt=np.float32(0.1), goals=goals, beta=beta)
    m = orc.Model(K, 2.0, ts.dt, goals, beta)
    trajs = []
    for i in range(12):
        z0 = rng.uniform(0.0, 10.0, size=2).astype(np.float32)
        trajs.append(orc.simulate(m, (i % 3) * 3 + 2 - (i // 3) % 2, z0, 40, 77, i).astype(np.float32))
    offsets = np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32)
    traj = np.concatenate(trajs)
    # the inputs do exercise the second pass: loose steps in FP64
    th = 2 * np.pi * np.arange(K) / K
    E = np.stack([np.cos(th), np.sin(th)], 1)
    s = 2.0 * float(ts.dt)
    loose = 0
    for t in trajs:
        z = t[:-1].astype(np.float64)
        dz = np.diff(t.astype(np.float64), axis=0)
        eo = dz / np.linalg.norm(dz, axis=1, keepdims=True)
        for g in goals.astype(np.float64):
            p = z - g
            pn = np.linalg.norm(p, axis=1)
            do = np.linalg.norm(p + s * eo, axis=1)
            d = np.linalg.norm(p[:, None, :] + s * E[None], axis=2)
            for b in beta.astype(np.float64):
                c = np.abs(pn - np.sign(b) * s)
                lg = b * (do[:, None] - d)
                Bnd = b * (do - c)
                loose += int((np.exp(lg - Bnd[:, None]).sum(1) < 2.0 ** -8).sum())
    assert loose > 50, loose
    prior = np.full(9, -np.log(9.0), np.float32)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    L, dg, dv, dw = gpu_loglik(ctx, ts, offsets, traj, prior)
    n_steps = len(traj) - len(trajs)
    assert abs(L - L64) <= 1e-6 * abs(L64) + n_steps * (2.0 ** -21 * 1500.0 * s + 4e-6), (L, L64)
    want = np.concatenate([dg64.ravel(), [dv64, dw64[1]]])
    check_grad(np.concatenate([dg.ravel(), [dv, dw[1]]]), want)
    assert abs(dw[0]) <= 1e-5 * np.linalg.norm(want)
    assert gpu_loglik(ctx, ts, offsets, traj, prior, grad=False) == L


def test_autograd_function(ctx, orc):
    from paper_2603_01122_gb300.autograd import marginal_loglik
    ts = workloads.differentiation()
    offsets, traj = trajectories(orc, ts, 32)
    prior = np.full(40, -np.log(40.0), np.float32)
    goals = dev(ts.goals).requires_grad_(True)
    speed = torch.tensor(ts.speed, requires_grad=True)
    w = torch.tensor([1.0, 1.0], requires_grad=True)
    L = marginal_loglik(goals, speed, w, dev(ts.beta), ts.K, ts.dt, dev(offsets, torch.int32), dev(traj),
                        dev(prior), ctx)
    (2.5 * L).backward()
    m = orc.Model(ts.K, ts.speed, ts.dt, ts.goals, ts.beta)
    L64, dg64, dv64, dw64 = orc.loglik_grad(m, offsets, traj.astype(np.float64), prior)
    assert abs(L.item() - L64) <= 1e-6 * abs(L64)
    got = np.concatenate([goals.grad.cpu().numpy().ravel(), [speed.grad.item(), w.grad[1].item()]])
    check_grad(got, 2.5 * np.concatenate([dg64.ravel(), [dv64, dw64[1]]]))


def test_invalid_adjoint_arguments(ctx):
    import paper_2603_01122_gb300 as pm
    ts = workloads.differentiation()
    g = dev(ts.goals)
    b = dev(ts.beta)
    model = pm.make_model(ts.K, ts.speed, ts.dt, g, b)
    L = torch.empty(1, device="cuda:0")
    off = dev(np.array([0, 3], np.int32), torch.int32)
    tr = dev(np.zeros((3, 2), np.float32))
    lp = dev(np.zeros(40, np.float32))
    with pytest.raises(pm.PmError):
        pm.pm_loglik_forward(ctx, model, 0, off, 3, tr, lp, L)
    with pytest.raises(pm.PmError):
        pm.pm_loglik_backward(ctx, model, 1, off, 3, tr, lp, 1.0, L, None, None, None)
