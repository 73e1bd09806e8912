"""Guard regions around every output buffer: each output is a view into a
larger buffer whose words before and after it hold a canary pattern; after
the call every canary word must be unchanged. This is the out-of-bounds-write
check of the library's outputs, on the cases that stress the index arithmetic
(ragged sizes, particles leaving the grid, windows at the grid's edge, odd
offsets). The outputs themselves are checked against the oracle elsewhere;
here the cheap invariants (counts + oob = N, normalised beliefs) are checked
beside the canaries."""
import math

import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev

pytestmark = pytest.mark.gpu
GUARD = 1027  # words on each side (odd, so the output starts off a 16-byte boundary)
CANARY_I = 0x5EA5EA5E
CANARY_F = -1.2345e30


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


class Guarded:
    """A view of `shape` inside a canary-filled buffer."""

    def __init__(self, shape, dtype=torch.int32, fill=None, guard=GUARD):
        n = int(np.prod(shape))
        canary = CANARY_I if dtype in (torch.int32,) else CANARY_F
        self.guard = guard
        self.buf = torch.full((n + 2 * guard,), canary, dtype=dtype, device="cuda:0")
        self.canary = canary
        self.view = self.buf[guard:guard + n].view(*shape)
        if fill is not None:
            self.view.fill_(fill)

    def intact(self):
        b = self.buf.cpu()
        return bool((b[:self.guard] == self.canary).all()) and bool((b[-self.guard:] == self.canary).all())


def _hist_ok(counts, oob, N):
    tot = counts.view(counts.shape[0], -1).to(torch.int64).sum(1) + oob.to(torch.int64)
    return bool((tot == N).all())


@pytest.mark.parametrize("case", ["paper_scale_small_grid", "plain_ragged", "outside"])
def test_single_rollout(ctx, orc, case):
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale() if case == "paper_scale_small_grid" else workloads.plain_small()
    gh = GpuHuman.of(hu)
    x0, y0, res, W, H = hu.grid
    N, T = {"paper_scale_small_grid": (33333, 47), "plain_ragged": (10001, 21), "outside": (777, 5)}[case]
    if case == "paper_scale_small_grid":
        # a small grid around the start: many particles leave it
        x0, y0, W, H = float(hu.start[0]) - 0.3, float(hu.start[1]) - 1.0, 37, 29
    z0 = (float(x0) - 3.0, float(y0) + 1.0) if case == "outside" else tuple(map(float, hu.start))
    counts = Guarded((T, H, W), fill=123)
    oob = Guarded((T,), fill=456)
    states = Guarded((64, T, 2), torch.float32, guard=GUARD + 1)  # pairs: 8-byte aligned
    heads = torch.full((64 * T + 2 * GUARD,), 0xA5, dtype=torch.uint8, device="cuda:0")
    comps = Guarded((64,))
    lb = dev(hu.uniform_log_prior())
    pm.pm_predict_occupancy_traced(ctx, gh.model, lb, z0[0], z0[1], N, T, pm.make_grid(x0, y0, res, W, H), 3, 9,
                                   counts.view, oob.view, 64, states.view, heads[GUARD:GUARD + 64 * T], comps.view)
    torch.cuda.synchronize()
    for g in (counts, oob, states, comps):
        assert g.intact()
    h = heads.cpu()
    assert bool((h[:GUARD] == 0xA5).all()) and bool((h[-GUARD:] == 0xA5).all())
    assert _hist_ok(counts.view, oob.view, N)


@pytest.mark.parametrize("speeds", [None, (0.5, 1.0, 1.5)])
def test_posterior_and_host_call(ctx, orc, speeds):
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    K = hu.K if speeds is None else 32
    gh = GpuHuman(K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=speeds)
    m = orc.Model(K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=(1.0,) if speeds is None else speeds)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    J = hu.G * hu.B
    lb = Guarded((J,), torch.float32)
    lb.view.copy_(dev(hu.uniform_log_prior()))
    out = Guarded((J,), torch.float32)
    pm.pm_update_posterior(ctx, gh.model, dev(obs), hu.n_obs, lb.view)
    pm.pm_update_posterior_into(ctx, gh.model, dev(obs), hu.n_obs, dev(hu.uniform_log_prior()), out.view)
    torch.cuda.synchronize()
    assert lb.intact() and out.intact()
    assert abs(float(torch.exp(out.view.double()).sum()) - 1.0) < 1e-6


def test_noalloc_posterior(ctx, orc):
    import paper_2603_01122_gb300 as pm
    hu = workloads.paper_scale()
    gh = GpuHuman.of(hu)
    m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    lb = Guarded((hu.G * hu.B,), torch.float32)
    lb.view.copy_(dev(hu.uniform_log_prior()))
    pm.pm_update_posterior_noalloc(gh.model, dev(obs), hu.n_obs, lb.view)
    torch.cuda.synchronize()
    assert lb.intact()
    assert abs(float(torch.exp(lb.view.double()).sum()) - 1.0) < 1e-6


def test_batched_several_speeds(ctx, orc):
    """The several-speed batched kernel with per-human speed masks and block
    marks, ragged N and T, windows past the grid's edge."""
    import paper_2603_01122_gb300 as pm
    speeds = (0.5, 1.0, 1.5)
    hs = workloads.batched()[:4]
    ds = []
    for k, hu in enumerate(hs):
        m = orc.Model(32, hu.speed, hu.dt, hu.goals, hu.beta, speeds=speeds)
        obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
        x0, y0, res, W, H = hu.grid
        if k % 2:
            W = H = 61
        N, T = 2003 + 31 * k, 17 + 2 * k
        gh = GpuHuman(32, hu.speed, hu.dt, hu.goals, hu.beta, speeds=speeds)
        ds.append(dict(hu=hu, gh=gh, obs=dev(obs), z0=dev(obs[-1]), N=N, T=T, center=k % 2,
                       grid=pm.make_grid(x0, y0, res, W, H), lb=dev(hu.uniform_log_prior()),
                       counts=Guarded((T, H, W), fill=7), oob=Guarded((T,), fill=7), speed_off=0b110 if k == 2 else 0))
    b = pm.pm_batch_create(ctx, ds[0]["gh"].model, 4)
    try:
        pm.pm_batch_set_block_flags(b, 1)
        pm.pm_batch_set(b, [pm.make_human(d["gh"].goals, d["gh"].beta, d["lb"], d["z0"], d["N"], d["T"], d["grid"],
                                          d["hu"].seed, d["hu"].human_id, d["counts"].view, d["oob"].view,
                                          obs_xy=d["obs"], n_obs=d["hu"].n_obs, center=d["center"],
                                          speed_off=d["speed_off"]) for d in ds])
        pm.pm_batch_update_posterior(b)
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d in ds:
            assert d["counts"].intact() and d["oob"].intact()
            assert _hist_ok(d["counts"].view, d["oob"].view, d["N"])
    finally:
        pm.pm_batch_destroy(b)


def test_batched_full_grids_and_windows(ctx, orc):
    """Humans whose windows reach past the shared grid's edge, centred
    windows, ragged particle counts; then the smoothing and the union."""
    import paper_2603_01122_gb300 as pm
    hs = workloads.batched()[:5]
    ds = []
    for k, hu in enumerate(hs):
        m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
        obs = orc.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
        x0, y0, res, W, H = hu.grid
        if k % 2:
            W = H = 61  # centred window
        N, T = 3001 + 17 * k, 23 + k
        ds.append(dict(hu=hu, gh=GpuHuman.of(hu), obs=dev(obs), z0=dev(obs[-1]), N=N, T=T,
                       grid=pm.make_grid(x0, y0, res, W, H), center=k % 2, lb=dev(hu.uniform_log_prior()),
                       counts=Guarded((T, H, W), fill=7), oob=Guarded((T,), fill=7)))
    b = pm.pm_batch_create(ctx, ds[0]["gh"].model, 8)
    try:
        pm.pm_batch_set_block_flags(b, 1)
        pm.pm_batch_set(b, [pm.make_human(d["gh"].goals, d["gh"].beta, d["lb"], d["z0"], d["N"], d["T"], d["grid"],
                                          d["hu"].seed, d["hu"].human_id, d["counts"].view, d["oob"].view,
                                          obs_xy=d["obs"], n_obs=d["hu"].n_obs, center=d["center"]) for d in ds])
        pm.pm_batch_update_posterior(b)
        pm.pm_batch_predict(b)
        x0, y0, res = hs[0].grid[:3]
        Tu = max(d["T"] for d in ds)
        union = Guarded((Tu, 400, 400), torch.float32)
        pm.pm_batch_union(b, 1.5, Tu, pm.make_grid(x0, y0, res, 400, 400), union.view)
        d0 = ds[0]
        smooth = Guarded((d0["T"], 400, 400), torch.float32)
        pm.pm_smooth_occupancy(ctx, d0["counts"].view, d0["N"], d0["T"], d0["grid"], 2.0, smooth.view)
        torch.cuda.synchronize()
        for d in ds:
            assert d["counts"].intact() and d["oob"].intact()
            assert _hist_ok(d["counts"].view, d["oob"].view, d["N"])
        assert union.intact() and smooth.intact()
    finally:
        pm.pm_batch_destroy(b)


def test_adjoint_outputs(ctx, orc):
    import paper_2603_01122_gb300 as pm
    ts = workloads.differentiation()
    trajs = []
    for i in range(9):
        g = int(ts.true_goal[i])
        mm = orc.Model(ts.K, ts.speed, ts.dt, ts.goals[g:g + 1], [ts.true_beta[i]])
        trajs.append(orc.simulate(mm, 0, ts.starts[i], int(ts.lengths[i]), ts.obs_seed, i).astype(np.float32))
    offsets = np.cumsum([0] + [len(t) for t in trajs]).astype(np.int32)
    traj = np.concatenate(trajs)
    g, b = dev(ts.goals), dev(ts.beta)
    model = pm.make_model(ts.K, ts.speed, ts.dt, g, b)
    L, dg, dv, dw = (Guarded((1,), torch.float32), Guarded(tuple(g.shape), torch.float32),
                     Guarded((1,), torch.float32), Guarded((2,), torch.float32))
    pm.pm_loglik_backward(ctx, model, 9, dev(offsets, torch.int32), traj.shape[0], dev(traj),
                          dev(np.full(40, -math.log(40.0), np.float32)), 1.0, L.view, dg.view, dv.view, dw.view)
    torch.cuda.synchronize()
    assert all(x.intact() for x in (L, dg, dv, dw))
    assert math.isfinite(float(L.view.item()))


def test_pair_buffers_must_be_aligned(ctx):
    """Traced states and MPPI perturbations are accessed as 8-byte pairs: a
    pointer 4 bytes off is rejected on the host before any launch."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    buf = torch.zeros(2 * 8 * 5 + 2, device="cuda:0")
    with pytest.raises(pm.PmError, match="aligned"):
        pm.pm_predict_occupancy_traced(ctx, gh.model, dev(hu.uniform_log_prior()), 0.0, 0.0, 8, 5, None, 1, 1,
                                       None, None, 8, buf[1:1 + 80].view(8, 5, 2))
    params = pm.make_mppi(4, 3, 0.1, 1, [1.0] * 4, [1.0] * 4, [1.0, 1.0], [0.0] * 4)
    d = torch.zeros(2 * 3 * 4 + 2, device="cuda:0")
    with pytest.raises(pm.PmError, match="aligned"):
        pm.pm_mppi_solve(ctx, params, np.zeros(4, np.float32), torch.zeros((3, 2), device="cuda:0"),
                         d[1:1 + 24], None, 0, None, torch.zeros((3, 4), device="cuda:0"),
                         torch.zeros((3, 2), device="cuda:0"))
    torch.cuda.synchronize()


def test_mppi_outputs(ctx):
    import paper_2603_01122_gb300 as pm
    N, T = 1000, 13
    rng = np.random.default_rng(4)
    params = pm.make_mppi(N, T, 0.1, 5, [3.0, 3.0, 10.0, 0.0], [0.6, 0.6, 2.0, 0.0], [2.0, 1.0],
                          [8.0, 4.0, 0.5, 0.0], 0.1, 1000.0, 0.1, 2.0)
    prob = np.full((T * 5, 60, 100), 0.2, np.float32)
    ctg = Guarded((T, N), torch.float32)
    u_opt = Guarded((T, 2), torch.float32)
    pm.pm_mppi_solve(ctx, params, np.float32([1.0, 1.5, 0.3, 0.4]), dev(np.zeros((T, 2), np.float32)),
                     dev((rng.normal(size=(T, N, 2)) * 0.5).astype(np.float32)), dev(prob), prob.shape[0],
                     pm.make_grid(0.0, 0.0, np.float32(0.1), 100, 60), ctg.view, u_opt.view)
    torch.cuda.synchronize()
    assert ctg.intact() and u_opt.intact()
