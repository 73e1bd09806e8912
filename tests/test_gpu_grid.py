"""Grid epilogue on the GPU against the FP64 oracle: Gaussian smoothing of one
human's occupancy (Sec. III-B) and the pointwise-maximum union of a batch of
humans on one shared grid (Sec. IV-B).

Tolerance: every output is a sum of at most (2R + 1)^2 non-negative FP32
products (count x 1/N x tap x tap) accumulated in two passes of 2R + 1 FMAs,
so its relative error is at most (2 (2R + 1) + 4) * 2^-24 <= 4.3e-6 for R <= 16;
the tests use 1e-5 relative (plus 1e-12 absolute for cells the blur barely
reaches). The maximum of such values is off by no more than the largest one.
"""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev, predict
from oracle import grid_ops as G

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-12


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def _plain_counts(ctx, orc):
    hu = workloads.plain_small()
    gh = GpuHuman.of(hu)
    got = predict(ctx, gh, hu.uniform_log_prior(), (0.0, 0.0), hu.n_particles, hu.horizon, hu.grid, hu.seed,
                  hu.human_id)
    return hu, got["counts"]


@pytest.mark.parametrize("sigma", [0.0, 0.7, 2.0, 5.33])
def test_smoothing_matches_oracle(ctx, orc, sigma):
    import paper_2603_01122_gb300 as pm
    hu, counts = _plain_counts(ctx, orc)
    T, H, W = counts.shape
    x0, y0, res, _, _ = hu.grid
    cd = torch.as_tensor(counts.view(np.int32)).to("cuda:0")
    prob = torch.full((T, H, W), -1.0, device="cuda:0")
    pm.pm_smooth_occupancy(ctx, cd, hu.n_particles, T, pm.make_grid(x0, y0, res, W, H), sigma, prob)
    torch.cuda.synchronize()
    got = prob.cpu().numpy().astype(np.float64)
    want = G.smooth(counts.astype(np.int64), hu.n_particles, sigma, pad=0)
    assert np.all(np.abs(got - want) <= RTOL * want + ATOL), np.max(np.abs(got - want) / (want + 1e-30))
    if sigma == 0.0:
        # normalisation only: one FP32 product per cell
        assert np.all(np.abs(got - want) <= 2.0 ** -23 * want)


def test_smoothing_ragged_grid_and_edges(ctx, orc):
    """A grid that is not a multiple of the 64 x 16 tile, with mass in the corners."""
    import paper_2603_01122_gb300 as pm
    rng = np.random.default_rng(9)
    T, H, W, N = 3, 37, 131, 1000
    counts = rng.integers(0, 40, size=(T, H, W)).astype(np.int64)
    counts[:, 0, 0] = 500
    counts[:, H - 1, W - 1] = 500
    prob = torch.empty((T, H, W), device="cuda:0")
    pm.pm_smooth_occupancy(ctx, dev(counts, torch.int32), N, T, pm.make_grid(0, 0, 1, W, H), 1.5, prob)
    torch.cuda.synchronize()
    want = G.smooth(counts, N, 1.5, pad=0)
    got = prob.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - want) <= RTOL * want + ATOL)


def _union_batch(ctx, orc):
    """Four humans in a 3 x 4 m room (60 x 80 cells at 5 cm): three with
    centred 31 x 31 windows (one reaching past the room's edge) and one with
    an explicit window offset; horizons 20, 30, 25 and 12."""
    import paper_2603_01122_gb300 as pm
    room = (0.0, 0.0, np.float32(0.05), 80, 60)
    starts = [(1.02, 1.53), (2.51, 1.04), (0.12, 2.87), (3.0, 2.0)]
    horizons = [20, 30, 25, 12]
    goals = np.array([[0.5, 2.5], [3.5, 0.5]], np.float32)
    beta = np.array([0.3, 3.0], np.float32)
    model = pm.make_model(36, 1.0, np.float32(0.02), dev(goals), dev(beta))
    recs, humans = [], []
    for i, (z, T) in enumerate(zip(starts, horizons)):
        center = 1 if i < 3 else 0
        Wh, Hh = (31, 31) if center else (21, 15)
        off = (0, 0) if center else (50, 30)
        N = 3000 + 1000 * i
        rec = dict(z0=dev(np.array(z, np.float32)), lb=dev(np.log(np.full(4, 0.25, np.float32))),
                   counts=torch.empty((T, Hh, Wh), dtype=torch.int32, device="cuda:0"),
                   oob=torch.empty(T, dtype=torch.int32, device="cuda:0"), T=T, N=N, center=center, off=off,
                   Wh=Wh, Hh=Hh, goals=dev(goals), beta=dev(beta))
        recs.append(rec)
        humans.append(pm.make_human(rec["goals"], rec["beta"], rec["lb"], rec["z0"], N, T,
                                    pm.make_grid(room[0], room[1], room[2], Wh, Hh), 7, 500 + i, rec["counts"],
                                    rec["oob"], center=center, cx_off=off[0], cy_off=off[1]))
    b = pm.pm_batch_create(ctx, model, len(humans))
    pm.pm_batch_set(b, humans)
    pm.pm_batch_predict(b)
    torch.cuda.synchronize()
    return pm, b, room, recs, starts


@pytest.mark.parametrize("sigma", [0.0, 1.2])
def test_union_matches_oracle(ctx, orc, sigma):
    pm, b, room, recs, starts = _union_batch(ctx, orc)
    try:
        x0, y0, res, W, H = room
        T = 30
        prob = torch.full((T, H, W), -1.0, device="cuda:0")
        pm.pm_batch_union(b, sigma, T, pm.make_grid(x0, y0, res, W, H), prob)
        torch.cuda.synchronize()
        got = prob.cpu().numpy().astype(np.float64)
        hs = []
        for r, z in zip(recs, starts):
            off = G.window_offset(z, room, r["Wh"], r["Hh"]) if r["center"] else r["off"]
            hs.append(dict(counts=r["counts"].cpu().numpy().view(np.uint32).astype(np.int64), n=r["N"], offset=off))
        want = G.union(hs, T, H, W, sigma)
        assert np.all(np.abs(got - want) <= RTOL * want + ATOL), np.max(np.abs(got - want))
        assert got.max() > 0.0
        # with block marks the union reads only marked blocks: the same result, bit for bit
        pm.pm_batch_set_block_flags(b, 1)
        pm.pm_batch_predict(b)
        prob2 = torch.full((T, H, W), -1.0, device="cuda:0")
        pm.pm_batch_union(b, sigma, T, pm.make_grid(x0, y0, res, W, H), prob2)
        torch.cuda.synchronize()
        for r, h in zip(recs, hs):  # the rollout is unchanged by the marks
            np.testing.assert_array_equal(r["counts"].cpu().numpy().view(np.uint32).astype(np.int64), h["counts"])
        np.testing.assert_array_equal(prob2.cpu().numpy(), prob.cpu().numpy())
        with pytest.raises(pm.PmError):
            pm.pm_batch_set_block_flags(b, 2)
    finally:
        pm.pm_batch_destroy(b)


def test_union_rejects_bad_sigma_and_grid(ctx, orc):
    pm, b, room, recs, starts = _union_batch(ctx, orc)
    try:
        x0, y0, res, W, H = room
        prob = torch.empty((30, H, W), device="cuda:0")
        for sigma in (-0.1, 5.34, float("nan")):
            with pytest.raises(pm.PmError) as e:
                pm.pm_batch_union(b, sigma, 30, pm.make_grid(x0, y0, res, W, H), prob)
            assert e.value.status == pm.PM_EINVAL
        with pytest.raises(pm.PmError):
            pm.pm_batch_union(b, 1.0, 30, pm.make_grid(x0 + 0.01, y0, res, W, H), prob)
    finally:
        pm.pm_batch_destroy(b)
