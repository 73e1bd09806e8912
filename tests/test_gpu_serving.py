"""Serving loop on the GPU: continuous batching with admission and departure;
every live human's frame output equals the single-human path on the same
belief and start (alone vs in the mix, bit-identical)."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2603_01122_gb300 as pm
    pm.build()
    c = pm.pm_create(0)
    yield c
    pm.pm_destroy(c)


def test_serving_frames_match_single_path(ctx, orc):
    import paper_2603_01122_gb300 as pm
    from paper_2603_01122_gb300.serving import Server, run_arrivals
    wl = workloads.serving(duration_s=6.0, rate_hz=3.0)
    arr = wl["arrivals"][:10]
    for a in arr:  # short dwell so that departures happen in the run
        a.t_leave = min(a.t_leave, a.t_arrive + 2.0)
    paths = []
    for a in arr:
        hu = a.human
        m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
        paths.append(orc.simulate(m, hu.true_j, hu.start, 400, hu.obs_seed, hu.human_id).astype(np.float32))
    hu0 = arr[0].human
    N, T, win = 3000, 40, 41
    srv = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, max_live=4, n_particles=N, horizon=T, window=win)
    checked = [0]

    def check(f, live):
        if f % 37 != 5 or not live:
            return
        torch.cuda.synchronize()
        for i, s in live.items():
            hu = arr[i].human
            goals = srv.goals[s, :hu.G].contiguous()
            beta = srv.beta[s, :hu.B].contiguous()
            model = pm.make_model(hu.K, hu.speed, hu.dt, goals, beta)
            lb = srv.log_b[s, :hu.G * hu.B].contiguous()
            z0 = srv.obs_dev[s, 1].cpu().numpy()
            x0, y0, res, W, H = hu.grid
            full = torch.empty((T, H, W), dtype=torch.int32, device="cuda:0")
            foob = torch.empty(T, dtype=torch.int32, device="cuda:0")
            pm.pm_predict_occupancy(ctx, model, lb, float(z0[0]), float(z0[1]), N, T,
                                    pm.make_grid(x0, y0, res, W, H), hu.seed, hu.human_id, full, foob)
            torch.cuda.synchronize()
            r = np.float32
            cx = int(np.floor(r(r(z0[0] - r(x0)) * (r(1.0) / r(res)))))
            cy = int(np.floor(r(r(z0[1] - r(y0)) * (r(1.0) / r(res)))))
            ox, oy = cx - (win - 1) // 2, cy - (win - 1) // 2
            f_np = full.cpu().numpy()
            want = np.zeros((T, win, win), np.int64)
            xs, ys, xe, ye = max(ox, 0), max(oy, 0), min(ox + win, W), min(oy + win, H)
            want[:, ys - oy:ye - oy, xs - ox:xe - ox] = f_np[:, ys:ye, xs:xe]
            np.testing.assert_array_equal(srv.counts[s].cpu().numpy(), want)
            checked[0] += 1

    try:
        out = run_arrivals(srv, arr, paths, frame_hz=125.0, duration_s=6.0, on_frame=check)
    finally:
        srv.close()
    assert checked[0] >= 5
    live = out["live"]
    assert live.max() == 4                      # the slot cap binds
    assert out["frames_waited"] > 0             # arrivals queued for a slot
    assert live[-1] < live.max() or live.min() < live.max()  # departures freed slots
    assert np.all(out["latency_s"] > 0)


def test_serving_frame_union_matches_oracle(ctx, orc):
    """With the grid epilogue on, a frame also leaves the blurred max-union of
    the live humans' windows on the room grid (the planner's input)."""
    from oracle import grid_ops as G
    from paper_2603_01122_gb300.serving import Server
    wl = workloads.serving(duration_s=6.0, rate_hz=3.0)
    arr = wl["arrivals"][:3]
    hu0 = arr[0].human
    N, T, win, sigma = 2000, 24, 31, 1.0
    srv = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, max_live=4, n_particles=N, horizon=T, window=win,
                 union_sigma=sigma)
    try:
        slots = []
        for i, a in enumerate(arr):
            hu = a.human
            slots.append(srv.admit(i, hu.goals, hu.beta, hu.start, hu.seed, hu.human_id))
        for _ in range(3):
            srv.frame()
        torch.cuda.synchronize()
        x0, y0, res, W, H = hu0.grid
        hs = []
        for s in slots:
            z0 = srv.obs_dev[s, 1].cpu().numpy()
            hs.append(dict(counts=srv.counts[s].cpu().numpy().view(np.uint32).astype(np.int64), n=N,
                           offset=G.window_offset(z0, hu0.grid, win, win)))
        want = G.union(hs, T, H, W, sigma)
        got = srv.union.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= 1e-5 * want + 1e-12)
        assert got.max() > 0.0
    finally:
        srv.close()


def test_serving_stationary_masking(ctx, orc):
    """Several speeds with stationary masking (Sec. IV-B): a human whose last
    observed step is shorter than stationary_eps keeps only the slow speed;
    each frame's window equals the single-human path under that human's mask."""
    import paper_2603_01122_gb300 as pm
    from paper_2603_01122_gb300.serving import Server
    hu = workloads.multi_speed()
    speeds, N, T, win = hu.speeds, 3000, 30, 31
    srv = Server(ctx, hu.K, hu.speed, hu.dt, hu.grid, max_live=3, n_particles=N, horizon=T, window=win,
                 speeds=speeds, stationary_off=0b110, stationary_eps=1e-4)
    rng = np.random.default_rng(5)
    try:
        slots = [srv.admit(i, hu.goals, hu.beta, [3.0 + i, 4.0], hu.seed, 60 + i) for i in range(3)]
        pos = [np.array([3.0 + i, 4.0]) for i in range(3)]
        for f in range(12):
            for i, s in enumerate(slots):
                moving = (i == 0) or (i == 2 and f % 4 < 2)
                if moving:
                    ang = rng.uniform(0, 2 * np.pi)
                    pos[i] = pos[i] + hu.speed * hu.dt * np.array([np.cos(ang), np.sin(ang)])
                srv.observe(s, pos[i].astype(np.float32))
            srv.frame()
            torch.cuda.synchronize()
            for i, s in enumerate(slots):
                mask = srv.meta[s]["speed_off"]
                moving = (i == 0) or (i == 2 and f % 4 < 2)
                assert mask == (0 if moving else 0b110)
                goals = srv.goals[s, :hu.G].contiguous()
                beta = srv.beta[s, :hu.B].contiguous()
                model = pm.make_model(hu.K, hu.speed, hu.dt, goals, beta, speeds=speeds, speed_off=mask)
                lb = srv.log_b[s, :hu.G * hu.B].contiguous()
                z0 = srv.obs_dev[s, 1].cpu().numpy()
                x0, y0, res, W, H = hu.grid
                full = torch.empty((T, H, W), dtype=torch.int32, device="cuda:0")
                foob = torch.empty(T, dtype=torch.int32, device="cuda:0")
                pm.pm_predict_occupancy(ctx, model, lb, float(z0[0]), float(z0[1]), N, T,
                                        pm.make_grid(x0, y0, res, W, H), hu.seed, 60 + i, full, foob)
                torch.cuda.synchronize()
                r = np.float32
                cx = int(np.floor(r(r(z0[0] - r(x0)) * (r(1.0) / r(res)))))
                cy = int(np.floor(r(r(z0[1] - r(y0)) * (r(1.0) / r(res)))))
                ox, oy = cx - (win - 1) // 2, cy - (win - 1) // 2
                np.testing.assert_array_equal(srv.counts[s].cpu().numpy(),
                                              full.cpu().numpy()[:, oy:oy + win, ox:ox + win])
    finally:
        srv.close()


def test_serving_resets_the_belief_when_a_human_leaves_a_goal(ctx):
    """With goal_radius, a human that reaches a goal and then moves away has its
    belief reset to uniform (Sec. IV-B) before the next frame's update."""
    from paper_2603_01122_gb300.serving import Server
    hu = workloads.paper_scale()
    srv = Server(ctx, hu.K, hu.speed, hu.dt, hu.grid, max_live=2, n_particles=2000, horizon=20, window=31,
                 goal_radius=0.1)
    try:
        g0 = np.asarray(hu.goals[0], np.float64)
        s = srv.admit("a", hu.goals, hu.beta, (g0 - [0.5, 0.0]).astype(np.float32), hu.seed, 7)
        J = hu.G * hu.B
        for k in range(1, 26):  # walk onto the goal along +x
            srv.observe(s, (g0 + [-0.5 + 0.02 * k, 0.0]).astype(np.float32))
            srv.frame()
        torch.cuda.synchronize()
        lb = srv.log_b[s, :J].cpu().numpy()
        assert np.max(np.abs(lb - (-np.log(J)))) > 1e-3  # the walk has informed the belief
        for k in range(1, 5):  # leave it along +y: the fourth step (0.12 m) passes the radius
            srv.observe(s, (g0 + [0.0, 0.03 * k]).astype(np.float32))
            if k < 4:
                srv.frame()
        srv.stream.synchronize()
        np.testing.assert_allclose(srv.log_b[s, :J].cpu().numpy(), -np.log(J), rtol=0, atol=1e-6)
    finally:
        srv.close()


def test_checkpoint_and_resume(ctx, orc):
    """Three humans served for 12 frames. At frame 5 one is exported, retired
    and re-admitted from its state, and another is moved to a second server
    the same way; every later frame of all three equals the uninterrupted
    run's, bit for bit (counts and beliefs)."""
    from paper_2603_01122_gb300.serving import Server
    arr = workloads.serving(duration_s=6.0, rate_hz=3.0)["arrivals"][:3]
    paths = []
    for a in arr:
        hu = a.human
        m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
        paths.append(orc.simulate(m, hu.true_j, hu.start, 20, hu.obs_seed, hu.human_id).astype(np.float32))
    hu0 = arr[0].human
    kw = dict(max_live=4, n_particles=2000, horizon=25, window=41)

    def admit_all(srv):
        return [srv.admit(i, a.human.goals, a.human.beta, paths[i][0], a.human.seed, a.human.human_id)
                for i, a in enumerate(arr)]

    ref = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, **kw)
    a_srv = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, **kw)
    b_srv = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, **kw)
    try:
        rs, as_ = admit_all(ref), admit_all(a_srv)
        where = {i: (a_srv, as_[i]) for i in range(3)}
        for f in range(1, 13):
            if f == 5:
                st0 = a_srv.export_state(where[0][1])
                a_srv.retire(where[0][1])
                where[0] = (a_srv, a_srv.import_state(st0))
                st2 = a_srv.export_state(where[2][1])
                a_srv.retire(where[2][1])
                where[2] = (b_srv, b_srv.import_state(st2))
            for i in range(3):
                ref.observe(rs[i], paths[i][f])
                srv, s = where[i]
                srv.observe(s, paths[i][f])
            ref.frame()
            a_srv.frame()
            if b_srv.slots.live:
                b_srv.frame()
            torch.cuda.synchronize()
            for i in range(3):
                srv, s = where[i]
                J = arr[i].human.G * arr[i].human.B
                assert torch.equal(srv.log_b[s, :J], ref.log_b[rs[i], :J]), (f, i)
                assert torch.equal(srv.counts[s], ref.counts[rs[i]]), (f, i)
                assert torch.equal(srv.oob[s], ref.oob[rs[i]]), (f, i)
    finally:
        ref.close()
        a_srv.close()
        b_srv.close()


def test_frame_without_observation_keeps_the_belief(ctx, orc):
    """A frame in which a human gets no new observation leaves its belief bit
    for bit as it was (the step applied has length zero), also for the first
    frame after import_state; a human observed in every frame meanwhile
    follows the oracle's posterior over its observed steps."""
    from paper_2603_01122_gb300.serving import Server
    from test_gpu_parity import assert_posterior_close
    arr = workloads.serving(duration_s=6.0, rate_hz=3.0)["arrivals"][:2]
    paths = []
    models = []
    for a in arr:
        hu = a.human
        m = orc.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
        models.append(m)
        paths.append(orc.simulate(m, hu.true_j, hu.start, 12, hu.obs_seed, hu.human_id).astype(np.float32))
    hu0 = arr[0].human
    srv = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, max_live=4, n_particles=2000, horizon=20, window=31)
    try:
        sl = [srv.admit(i, a.human.goals, a.human.beta, paths[i][0], a.human.seed, a.human.human_id)
              for i, a in enumerate(arr)]
        J = [a.human.G * a.human.B for a in arr]
        seen = [0, 0]  # index of each human's last observed state
        for f in range(1, 11):
            skip = f in (3, 4, 8)  # human 1 gets no observation in these frames
            if f == 7:             # human 1 is checkpointed and re-admitted before the frame
                st = srv.export_state(sl[1])
                srv.retire(sl[1])
                sl[1] = srv.import_state(st)
            srv.stream.synchronize()
            before = srv.log_b[sl[1], :J[1]].clone()
            seen[0] += 1
            srv.observe(sl[0], paths[0][seen[0]])
            if not skip and f != 7:
                seen[1] += 1
                srv.observe(sl[1], paths[1][seen[1]])
            srv.frame()
            torch.cuda.synchronize()
            if skip or f == 7:
                assert torch.equal(srv.log_b[sl[1], :J[1]], before), f
            for i in range(2):
                want, _ = orc.update_posterior(models[i], paths[i][:seen[i] + 1].astype(np.float64),
                                               np.full(J[i], -np.log(J[i])))
                assert_posterior_close(srv.log_b[sl[i], :J[i]].cpu().numpy(), want)
    finally:
        srv.close()


def test_graph_launch_rejects_a_null_graph():
    import paper_2603_01122_gb300 as pm
    with pytest.raises(pm.PmError) as e:
        pm.pm_graph_launch(0)
    assert e.value.status == pm.PM_EINVAL
