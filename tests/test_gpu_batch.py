"""Batched persistent launch: every human's result equals its single-human
result bit for bit (alone vs in the mix), for the belief update and the
histogram, under retiling by the autotuner and under CUDA-graph replay."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import GpuHuman, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def _setup(orc, humans, scale=1.0):
    """Device inputs for each human: observed history from the oracle's model."""
    import paper_2603_01122_gb300 as pm
    out = []
    for hu in humans:
        m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
        obs = orc.simulate(m, hu.true_j, hu.start, max(hu.n_obs, 1), hu.obs_seed, hu.human_id).astype(np.float32)
        gh = GpuHuman.of(hu)
        N = max(1, int(hu.n_particles * scale))
        T = hu.horizon
        x0, y0, res, W, H = hu.grid
        if hu.window:
            W = H = hu.window
        d = dict(hu=hu, gh=gh, obs=dev(obs), n_obs=obs.shape[0] - 1, N=N, T=T,
                 lb=dev(hu.uniform_log_prior()), z0=dev(obs[-1]), grid=pm.make_grid(x0, y0, res, W, H),
                 full_grid=pm.make_grid(x0, y0, res, hu.grid[3], hu.grid[4]),
                 # garbage: the batched rollout must zero every cell itself
                 counts=torch.full((T, H, W), 0x3C3C3C3C, dtype=torch.int32, device="cuda:0"),
                 oob=torch.full((T,), 777, dtype=torch.int32, device="cuda:0"))
        out.append(d)
    return out


def _pm_humans(ds, center=0):
    import paper_2603_01122_gb300 as pm
    return [pm.make_human(d["gh"].goals, d["gh"].beta, d["lb"], d["z0"], d["N"], d["T"], d["grid"],
                          d["hu"].seed, d["hu"].human_id, d["counts"], d["oob"], obs_xy=d["obs"],
                          n_obs=d["n_obs"], center=center) for d in ds]


def _single(ctx, d, lb):
    import paper_2603_01122_gb300 as pm
    T = d["T"]
    g = d["full_grid"]
    counts = torch.empty((T, g.H, g.W), dtype=torch.int32, device="cuda:0")
    oob = torch.empty(T, dtype=torch.int32, device="cuda:0")
    z0 = d["z0"].cpu().numpy()
    pm.pm_predict_occupancy(ctx, d["gh"].model, lb, float(z0[0]), float(z0[1]), d["N"], T, g, d["hu"].seed,
                            d["hu"].human_id, counts, oob)
    return counts, oob


def _shared_model(hu, gh):
    import paper_2603_01122_gb300 as pm
    return pm.make_model(hu.K, hu.speed, hu.dt, gh.goals, gh.beta)


def test_batched_workload_alone_equals_in_mix(ctx, orc):
    import paper_2603_01122_gb300 as pm
    humans = workloads.batched()
    ds = _setup(orc, humans)
    b = pm.pm_batch_create(ctx, _shared_model(humans[0], ds[0]["gh"]), len(ds))
    try:
        pm.pm_batch_set(b, _pm_humans(ds))
        # single-human posteriors first, from the same priors
        singles = []
        for d in ds:
            lb = d["lb"].clone()
            pm.pm_update_posterior(ctx, d["gh"].model, d["obs"], d["n_obs"], lb)
            singles.append(lb)
        pm.pm_batch_update_posterior(b)
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d, lb in zip(ds, singles):
            assert torch.equal(d["lb"], lb)
            c, o = _single(ctx, d, lb)
            torch.cuda.synchronize()
            assert torch.equal(d["counts"], c), d["hu"].human_id
            assert torch.equal(d["oob"], o)
            tot = d["counts"].view(d["T"], -1).sum(1, dtype=torch.int64) + d["oob"]
            assert torch.all(tot == d["N"])
    finally:
        pm.pm_batch_destroy(b)


def test_outputs_zeroed_at_odd_offsets(ctx, orc):
    """Outputs that start 4, 8 and 12 bytes past a 16-byte boundary and hold a
    word count that is no multiple of 4 (ragged head and tail of the batch's
    16-byte zeroing) come out equal to the single path, from garbage, on two
    launches in a row (the second reuses the dirty buffers), in both
    emplacement forms."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.plain_small()
    ds = _setup(orc, [hu, hu, hu], scale=0.5)
    shapes = [(37, 171, 83), (5, 13, 7), (61, 129, 255)]  # T, H, W: 525,141 / 455 / 2,006,595 words
    for k, (d, (T, H, W)) in enumerate(zip(ds, shapes)):
        buf = torch.full((T * H * W + 8,), 0x3C3C3C3C, dtype=torch.int32, device="cuda:0")
        d["counts"] = buf[k + 1:k + 1 + T * H * W].view(T, H, W)
        d["oob"] = torch.full((T + 3,), 777, dtype=torch.int32, device="cuda:0")[k + 1:k + 1 + T]
        d["T"] = T
        d["grid"] = d["full_grid"] = pm.make_grid(hu.grid[0], hu.grid[1], hu.grid[2], W, H)
        d["hu"] = hu
    b = pm.pm_batch_create(ctx, _shared_model(hu, ds[0]["gh"]), 4)
    try:
        for warp, threads in ((1, 128), (0, 256)):
            pm.pm_batch_set_config(b, threads, 0 if warp else 1, 0, 48)
            pm.pm_batch_set(b, _pm_humans(ds))
            for rep in range(2):
                pm.pm_batch_predict(b)
                torch.cuda.synchronize()
                for d in ds:
                    c, o = _single(ctx, d, d["lb"])
                    torch.cuda.synchronize()
                    assert torch.equal(d["counts"], c), (warp, rep, d["T"])
                    assert torch.equal(d["oob"], o)
        pm.pm_sync_status(ctx)
    finally:
        pm.pm_batch_destroy(b)


def test_centred_windows_equal_cropped_full_grid(ctx, orc):
    import paper_2603_01122_gb300 as pm
    arr = workloads.serving()["arrivals"][:6]
    ds = _setup(orc, [a.human for a in arr], scale=0.2)
    b = pm.pm_batch_create(ctx, _shared_model(arr[0].human, ds[0]["gh"]), 8)
    try:
        pm.pm_batch_set(b, _pm_humans(ds, center=1))
        pm.pm_batch_update_posterior(b)
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d in ds:
            full, full_oob = _single(ctx, d, d["lb"])
            torch.cuda.synchronize()
            x0, y0, res, W, H = d["hu"].grid
            z0 = d["z0"].cpu().numpy()
            r = np.float32
            cx = int(np.floor(r(r(r(z0[0]) - r(x0)) * (r(1.0) / r(res)))))
            cy = int(np.floor(r(r(r(z0[1]) - r(y0)) * (r(1.0) / r(res)))))
            w = d["hu"].window
            ox, oy = cx - (w - 1) // 2, cy - (w - 1) // 2
            f = full.cpu().numpy()
            want = np.zeros((d["T"], w, w), np.int64)
            xs, ys = max(ox, 0), max(oy, 0)
            xe, ye = min(ox + w, W), min(oy + w, H)
            want[:, ys - oy:ye - oy, xs - ox:xe - ox] = f[:, ys:ye, xs:xe]
            got = d["counts"].cpu().numpy()
            np.testing.assert_array_equal(got, want)
            outside = f.reshape(d["T"], -1).sum(1) - want.reshape(d["T"], -1).sum(1)
            np.testing.assert_array_equal(d["oob"].cpu().numpy(), full_oob.cpu().numpy() + outside)
    finally:
        pm.pm_batch_destroy(b)


def test_autotune_and_graph_replay(ctx, orc):
    import paper_2603_01122_gb300 as pm
    humans = workloads.batched()[:6]
    ds = _setup(orc, humans, scale=0.25)
    b = pm.pm_batch_create(ctx, _shared_model(humans[0], ds[0]["gh"]), 8)
    try:
        pm.pm_batch_set(b, _pm_humans(ds))
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        ref = [d["counts"].clone() for d in ds]
        pm.pm_batch_autotune(b)
        cfg = pm.pm_batch_get_config(b)
        assert cfg["threads"] in (128, 224, 256) and cfg["shared_window"] in (0, 1)
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d, r in zip(ds, ref):
            assert torch.equal(d["counts"], r)
        for t, sw, w in [(128, 0, 48), (256, 0, 48), (224, 1, 24), (256, 1, 96)]:
            pm.pm_batch_set_config(b, t, sw, 0, w)
            pm.pm_batch_predict(b)
            torch.cuda.synchronize()
            for d, r in zip(ds, ref):
                assert torch.equal(d["counts"], r)
        # capture one frame (belief update + prediction) in a CUDA graph
        s = torch.cuda.Stream()
        lb0 = [d["lb"].clone() for d in ds]
        with torch.cuda.stream(s):
            pm.pm_batch_update_posterior(b, s)
            pm.pm_batch_predict(b, s)
        s.synchronize()
        want = [d["counts"].clone() for d in ds]
        want_lb = [d["lb"].clone() for d in ds]
        g = torch.cuda.CUDAGraph()
        for d, l in zip(ds, lb0):
            d["lb"].copy_(l)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            pm.pm_batch_update_posterior(b, s)
            pm.pm_batch_predict(b, s)
        for d, l in zip(ds, lb0):
            d["lb"].copy_(l)
            d["counts"].fill_(7)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for d, w, wl in zip(ds, want, want_lb):
            assert torch.equal(d["counts"], w)
            assert torch.equal(d["lb"], wl)
        # the graph reads z0 from device memory: move one start and replay
        ds[0]["z0"].add_(0.5)
        for d, l in zip(ds, lb0):
            d["lb"].copy_(l)
        g.replay()
        torch.cuda.synchronize()
        c, o = _single(ctx, ds[0], ds[0]["lb"])
        torch.cuda.synchronize()
        assert torch.equal(ds[0]["counts"], c)
    finally:
        pm.pm_batch_destroy(b)


def test_batch_rejects_mixed_or_invalid(ctx, orc):
    import paper_2603_01122_gb300 as pm
    humans = workloads.batched()[:2]
    ds = _setup(orc, humans, scale=0.01)
    b = pm.pm_batch_create(ctx, _shared_model(humans[0], ds[0]["gh"]), 1)
    try:
        with pytest.raises(pm.PmError):
            pm.pm_batch_set(b, _pm_humans(ds))  # more than max_humans
        hs = _pm_humans(ds[:1])
        hs[0].horizon = 0
        with pytest.raises(pm.PmError):
            pm.pm_batch_set(b, hs)
        hs = _pm_humans(ds[:1], center=1)
        hs[0].grid = pm.make_grid(0, 0, 0.05, 120, 121)
        with pytest.raises(pm.PmError):
            pm.pm_batch_set(b, hs)
    finally:
        pm.pm_batch_destroy(b)


@pytest.mark.parametrize("center", [0, 1])
def test_reach_zeroing_equals_full_zeroing(ctx, orc, center):
    """pm_batch_set_zeroing(1) zeroes only the cells the previous and the
    current prediction of a slot can reach. Against a batch that zeroes every
    cell (same humans, same starts, its own buffers): equal counts and oob
    from garbage, with the starts moved between predictions (small steps, a
    jump across the grid, no move), directly and from a replayed CUDA graph
    whose starts change on the device; with the full grid and with centred
    41 x 41 windows."""
    import paper_2603_01122_gb300 as pm
    hu = workloads.plain_small()
    ds = _setup(orc, [hu, hu, hu], scale=0.5)
    x0, y0, res, W, H = hu.grid
    if center:
        for d in ds:
            d["grid"] = pm.make_grid(x0, y0, res, 41, 41)
            d["counts"] = torch.full((d["T"], 41, 41), 0x3C3C3C3C, dtype=torch.int32, device="cuda:0")
    full = [dict(d, counts=torch.full_like(d["counts"], 0x5A5A5A5A), oob=torch.full_like(d["oob"], 5)) for d in ds]
    model = _shared_model(hu, ds[0]["gh"])
    bf = pm.pm_batch_create(ctx, model, len(ds))
    br = pm.pm_batch_create(ctx, model, len(ds))
    try:
        pm.pm_batch_set(bf, _pm_humans(full, center))
        pm.pm_batch_set(br, _pm_humans(ds, center))
        pm.pm_batch_set_zeroing(br, 1)
        starts = [d["z0"].cpu().numpy().copy() for d in ds]
        moves = [(0.0, 0.0), (0.3, -0.2), (0.0, 0.0), (-3.1, 2.4), (0.05, 0.05), (4.0, 4.0)]

        def check():
            torch.cuda.synchronize()
            for d, f in zip(ds, full):
                assert torch.equal(d["counts"], f["counts"])
                assert torch.equal(d["oob"], f["oob"])
                tot = d["counts"].view(d["T"], -1).sum(1, dtype=torch.int64) + d["oob"]
                assert torch.all(tot == d["N"])

        for k, (mx, my) in enumerate(moves):
            for i, d in enumerate(ds):
                starts[i] += np.float32([mx * (1 + 0.5 * i), my])
                d["z0"].copy_(torch.tensor(starts[i], device="cuda:0"))
            pm.pm_batch_predict(bf)
            pm.pm_batch_predict(br)
            check()
        # graph replays: the starts change on the device between replays
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                pm.pm_batch_predict(br, s)
        for mx, my in [(1.0, 0.0), (0.0, 0.0), (-2.5, -1.5)]:
            for i, d in enumerate(ds):
                starts[i] += np.float32([mx, my * (1 + i)])
                d["z0"].copy_(torch.tensor(starts[i], device="cuda:0"))
            torch.cuda.synchronize()
            g.replay()
            pm.pm_batch_predict(bf)
            check()
    finally:
        pm.pm_batch_destroy(bf)
        pm.pm_batch_destroy(br)


def test_plain_crowd_alone_equals_in_mix(ctx, orc):
    """16 humans of the plain configuration's shape (K = 8: the 8-heading
    instantiations of the batched kernels) in one batch, with reachable-cell
    zeroing: every human's belief and counts equal its single-human calls."""
    import paper_2603_01122_gb300 as pm
    humans = workloads.plain_crowd(16)
    ds = _setup(orc, humans)
    b = pm.pm_batch_create(ctx, _shared_model(humans[0], ds[0]["gh"]), len(ds))
    try:
        pm.pm_batch_set(b, _pm_humans(ds))
        pm.pm_batch_set_zeroing(b, 1)
        singles = []
        for d in ds:
            lb = d["lb"].clone()
            pm.pm_update_posterior(ctx, d["gh"].model, d["obs"], d["n_obs"], lb)
            singles.append(lb)
        pm.pm_batch_update_posterior(b)
        for _ in range(2):  # the second prediction zeroes only the reachable cells
            pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        for d, lb in zip(ds, singles):
            assert torch.equal(d["lb"], lb)
            c, o = _single(ctx, d, lb)
            torch.cuda.synchronize()
            assert torch.equal(d["counts"], c), d["hu"].human_id
            assert torch.equal(d["oob"], o)
    finally:
        pm.pm_batch_destroy(b)


def test_zero_and_rollout_halves_equal_predict(ctx, orc):
    """pm_batch_zero + pm_batch_rollout on two streams joined by an event
    equal pm_batch_predict; a second rollout without zeroing adds the same
    counts again (the documented contract of pm_batch_rollout)."""
    import paper_2603_01122_gb300 as pm
    humans = workloads.plain_crowd(6)
    ds = _setup(orc, humans)
    b = pm.pm_batch_create(ctx, _shared_model(humans[0], ds[0]["gh"]), len(ds))
    try:
        pm.pm_batch_set(b, _pm_humans(ds))
        pm.pm_batch_predict(b)
        torch.cuda.synchronize()
        want = [(d["counts"].clone(), d["oob"].clone()) for d in ds]
        for d in ds:
            d["counts"].fill_(0x3C3C3C3C)
        main, side = torch.cuda.Stream(), torch.cuda.Stream()
        side.wait_stream(main)
        pm.pm_batch_zero(b, side)
        main.wait_stream(side)
        pm.pm_batch_rollout(b, main)
        torch.cuda.synchronize()
        for d, (c, o) in zip(ds, want):
            assert torch.equal(d["counts"], c) and torch.equal(d["oob"], o)
        pm.pm_batch_rollout(b, main)
        torch.cuda.synchronize()
        for d, (c, o) in zip(ds, want):
            assert torch.equal(d["counts"], 2 * c) and torch.equal(d["oob"], 2 * o)
    finally:
        pm.pm_batch_destroy(b)
