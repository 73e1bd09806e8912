"""MPPI local planner on the GPU (Sec. III-C) against the FP64 oracle.

Tolerances. A sample's cost-to-go is a sum of at most T running costs, each a
few FP32 operations on states that carry the FP32 rounding of T Euler steps;
|S_gpu - S_64| <= 1e-4 * (1 + S_64) covers it with margin, except where the
two binnings of a robot position can fall in different cells: samples whose
looked-up positions come within 1e-3 cells of a cell edge are checked only
for the other terms (they may gain or lose one collision cost). The update is
checked twice: applied by the oracle to the GPU's own costs (the reduction
alone: FP32 sums of N terms, relative 1e-5 of max |delta|), and against the
oracle end to end, where a cost error dS moves a weight by a factor
exp(dS / tau): |du| <= 2 max|delta| (exp(max dS / tau) - 1) + 1e-5 max|delta|.
"""
import numpy as np
import pytest
import torch

from gpu_util import dev
from oracle import mppi as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def _scenario(N, T, seed, with_grid=True):
    rng = np.random.default_rng(seed)
    p = dict(dt=0.1, pred_stride=5, q=[3.0, 3.0, 10.0, 0.0], q_final=[0.6, 0.6, 2.0, 0.0], r=[2.0, 1.0],
             goal=[8.0, 4.0, 0.5, 0.0], coll_threshold=0.1, coll_cost=1000.0, step_cost=0.1, temperature=2.0)
    z0 = [1.0, 1.5, 0.3, 0.4]
    u_ref = np.stack([np.full(T, 0.2), np.full(T, 0.05)], 1).astype(np.float32)
    delta = (rng.normal(size=(T, N, 2)) * [0.6, 0.5]).astype(np.float32)
    grid = (0.0, 0.0, np.float32(0.1), 100, 60)
    prob = None
    if with_grid:
        # a blob of predicted occupancy across the robot's way, growing with time
        Tg = T * 5
        yy, xx = np.mgrid[0:60, 0:100]
        prob = np.zeros((Tg, 60, 100), np.float32)
        for k in range(Tg):
            cx, cy, s = 30 + k * 0.1, 22, 3 + 0.05 * k
            prob[k] = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s)).astype(np.float32) * 0.3
    return p, z0, u_ref, delta, prob, grid


def _gpu(ctx, p, z0, u_ref, delta, prob, grid):
    import paper_2603_01122_gb300 as pm
    T, N, _ = delta.shape
    params = pm.make_mppi(N, T, p["dt"], p["pred_stride"], p["q"], p["q_final"], p["r"], p["goal"],
                          p["coll_threshold"], p["coll_cost"], p["step_cost"], p["temperature"])
    ctg = torch.full((T, N), -1.0, device="cuda:0")
    u_opt = torch.full((T, 2), -1.0, device="cuda:0")
    pd = dev(prob) if prob is not None else None
    g = pm.make_grid(*grid) if prob is not None else None
    pm.pm_mppi_solve(ctx, params, np.float32(z0), dev(u_ref), dev(delta), pd, 0 if prob is None else prob.shape[0],
                     g, ctg, u_opt)
    torch.cuda.synchronize()
    return ctg.cpu().numpy().astype(np.float64), u_opt.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,T,with_grid", [(4096, 30, True), (1000, 17, True), (333, 5, False), (1, 8, True)])
def test_mppi_matches_oracle(ctx, N, T, with_grid):
    p, z0, u_ref, delta, prob, grid = _scenario(N, T, 7 + N + T, with_grid)
    S_gpu, u_gpu = _gpu(ctx, p, z0, u_ref, delta, prob, grid)
    u_orc, S0, S, edge = M.solve(p, np.float32(z0).astype(np.float64), u_ref, delta,
                                 prob if prob is not None else np.zeros((1, 1, 1), np.float32), grid)
    near = edge < 1e-3
    ok = np.abs(S_gpu - S) <= 1e-4 * (1.0 + S)
    assert np.all(ok[:, ~near]), np.max(np.abs(S_gpu - S)[:, ~near])
    # off the edges, costs agree; near one, the difference is at most the collision costs
    diff = np.abs(S_gpu - S)[:, near]
    assert np.all(np.isclose(diff / p["coll_cost"], np.round(diff / p["coll_cost"]), atol=1e-3))
    if with_grid and N > 100:
        assert (S0 > p["coll_cost"]).any()  # some samples did hit the predicted occupancy
    dmax = np.abs(delta).max()
    # the reduction alone, on the GPU's costs
    u_red = M.update(u_ref, delta, S_gpu, p["temperature"])
    assert np.all(np.abs(u_gpu - u_red) <= 1e-5 * dmax + 1e-7)
    # end to end: the oracle's costs, except that a sample on a cell edge keeps
    # the GPU's collision decisions (the one place where both readings are right)
    S_ref = S.copy()
    S_ref[:, near] = S[:, near] + p["coll_cost"] * np.round((S_gpu - S)[:, near] / p["coll_cost"])
    dS = np.max(np.abs(S_gpu - S_ref))
    tol = 2 * dmax * (np.exp(dS / p["temperature"]) - 1) + 1e-5 * dmax + 1e-7
    u_end = M.update(u_ref, delta, S_ref, p["temperature"])
    assert np.all(np.abs(u_gpu - u_end) <= tol)
    if not near.any():
        assert np.array_equal(u_end, u_orc)


def test_mppi_rejects_bad_parameters(ctx):
    import paper_2603_01122_gb300 as pm
    p, z0, u_ref, delta, prob, grid = _scenario(16, 4, 1, False)
    T, N = 4, 16
    ctg = torch.empty((T, N), device="cuda:0")
    u_opt = torch.empty((T, 2), device="cuda:0")
    for kw in (dict(n_samples=0), dict(horizon=0), dict(dt=0.0), dict(temperature=0.0), dict(pred_stride=0)):
        args = dict(n_samples=N, horizon=T, dt=0.1, pred_stride=5, temperature=1.0)
        args.update(kw)
        params = pm.make_mppi(args["n_samples"], args["horizon"], args["dt"], args["pred_stride"], p["q"],
                              p["q_final"], p["r"], p["goal"], temperature=args["temperature"])
        with pytest.raises(pm.PmError) as e:
            pm.pm_mppi_solve(ctx, params, z0, dev(u_ref), dev(delta), None, 0, None, ctg, u_opt)
        assert e.value.status == pm.PM_EINVAL
