"""Benchmark of the prediction hot path on the paper-scale workload.

One step = the whole path on one human of the ``paper_scale`` workload:
the belief update over 50 observed steps (Eq. 3 / Eq. 7), then Algorithm 1
for N = 100k particles over T = 150 steps with K = 36 headings, emplaced on a
200 x 200 grid (counts zeroed and rebuilt every step). The metric is
particle-steps per second (N * T per step), device-timed with CUDA events
around each step on the launching stream; L2 is flushed (a 256 MiB write)
before every timed step. ``e2e`` runs the same step through the host-buffer
entry point pm_predict_host (inputs from pinned host memory, the posterior
and the 24 MB histogram copied back every step).

Multi-GPU (torchrun): every rank predicts its own human (human_id = rank), no
data-path collective; value = all ranks' particle-steps / the slowest rank's
time ("weak" scaling).

``--impl reference`` times the FP64 CPU oracle (the reference arm) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "particle-steps/s"


def _measured_peak(key, default):
    """A measured peak of this GPU type from MEASURED_PEAKS.json at the
    repository root (copy bandwidth, bf16 GEMM), else the given value."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, ValueError, KeyError, TypeError):
        return default


HBM_PEAK_GBS = _measured_peak("hbm_gbs", 6794.5)
# every source the rollout kernels are compiled from (the public header
# reaches them only through pm_limits.h; the traffic of a
# committed ncu summary is used only while these are unchanged)
ROLLOUT_SOURCES = ["paper_2603_01122_gb300/csrc/pm_rollout.cu", "paper_2603_01122_gb300/csrc/pm_rollout_dev.cuh",
                   "paper_2603_01122_gb300/csrc/pm_internal.cuh", "include/pm_limits.h"]


# main-line workloads: generator and the rollout kernel that dominates it
MAIN_WORKLOADS = {
    "paper_scale": (workloads.paper_scale, "rollout_warp_kernel<36,true>"),
    "multi_speed": (workloads.multi_speed, "rollout_multi_kernel<32>"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=20000, help="particles in the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched / serving / adjoint sections")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="run the Poisson arrival process for this many simulated seconds (0: skip)")
    ap.add_argument("--serving-frames", type=int, default=250, help="frames of the forced-64-live run")
    ap.add_argument("--sections", default="all", type=lambda v: set(v.split(",")),
                    help="extra sections to run: all, or a comma list of batched, batched_small, serving, speeds, table1, "
                         "differentiation (plain_small always runs)")
    ap.add_argument("--workload", default="paper_scale", choices=sorted(MAIN_WORKLOADS),
                    help="the main line's workload (paper_scale: one speed, K = 36; multi_speed: |U| = 96)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_human_id(base_id, rank):
    """Each rank predicts its own human (its own Philox key): the ranks share
    no data and exchange nothing on the data path."""
    return base_id + 1000 * rank


def max_over_ranks(x, world, tdist=None, device=None):
    """The largest of the ranks' values of x (the slowest rank's time)."""
    if world == 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job units per second: every rank's units over the slowest time."""
    return world * units_per_rank / seconds


def workload_config(hu, name="paper_scale"):
    x0, y0, res, W, H = hu.grid
    speeds = {} if tuple(hu.speeds) == (1.0,) else {"speeds": list(hu.speeds), "controls": hu.K * len(hu.speeds)}
    return {
        "workload": name,
        "humans_per_gpu": 1,
        "K": hu.K, **speeds, "G": hu.G, "B": hu.B, "n_obs": hu.n_obs,
        "n_particles": hu.n_particles, "horizon": hu.horizon,
        "grid": f"{W}x{H}@{res:.3g}m", "dt": round(hu.dt, 6),
        "l2": "flushed before every timed step (256 MiB write)",
    }


def sources_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self, t0, t1):
        """Keep only the samples stamped inside the wall-clock interval [t0, t1]."""
        self.t0, self.t1 = t0, t1

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import datetime
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t0", None), getattr(self, "t1", None)
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if t0 is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                    continue
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_threads():
    """Host cores the oracle may use (its C calls release the GIL, so Python
    threads over particle ranges run in parallel)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_sample(hu, n_particles, obs=None, threads=1):
    """Time the FP64 oracle (as it stands) on a bounded sample: the belief
    update, then the rollout of particles [0, n_particles) split into
    contiguous ranges over `threads` host threads."""
    import concurrent.futures as cf

    import oracle
    m = oracle.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, speeds=hu.speeds, speed_off=hu.speed_off)
    if obs is None:
        obs = oracle.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id).astype(np.float32)
    cuts = np.linspace(0, n_particles, threads + 1).astype(np.int64)
    t0 = time.perf_counter()
    post, _ = oracle.update_posterior(m, obs.astype(np.float64), hu.uniform_log_prior())
    lb = post.astype(np.float32)

    def part(r):
        return oracle.rollout(m, lb, obs[-1], hu.horizon, hu.seed, hu.human_id, int(cuts[r]), int(cuts[r + 1]),
                              grid=hu.grid)
    if threads == 1:
        part(0)
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(part, range(threads)))
    dt = time.perf_counter() - t0
    ps = n_particles * hu.horizon
    return {"value": ps / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{n_particles} of {hu.n_particles} particles x T={hu.horizon} + {hu.n_obs}-step belief "
                      f"update, FP64 C, {threads} host threads over particle ranges ({dt:.2f} s wall)"}


def oracle_other_configs(threads):
    """The oracle (as it stands) on the other configurations: the plain one
    (K = 8, N = 10k, T = 20) whole, a 1/50 sample of every batched human's
    particles (scaled by particle-steps), and the exact Markov propagation of
    the plain one's occupancy (Eq. 4 / Eq. 5, single-threaded)."""
    import concurrent.futures as cf

    import oracle
    out = {}
    hu = workloads.plain_small()
    cb = oracle_sample(hu, hu.n_particles, threads=threads)
    out["plain_small"] = {"value": cb["value"], "cores": threads, "sample": cb["sample"],
                          "one_thread": oracle_sample(hu, hu.n_particles)["value"]}
    hs = workloads.batched()
    jobs = []
    for h in hs:
        m = oracle.Model(h.K, h.speed, h.dt, h.goals, h.beta)
        obs = oracle.simulate(m, h.true_j, h.start, h.n_obs, h.obs_seed, h.human_id)
        jobs.append((h, m, obs, max(256, h.n_particles // 50)))
    t0 = time.perf_counter()
    parts = []
    for h, m, obs, n in jobs:
        post, _ = oracle.update_posterior(m, obs, h.uniform_log_prior())
        # each call bins into its own full grid: few, large ranges per human
        nr = max(1, threads // len(jobs))
        cuts = np.linspace(0, n, nr + 1).astype(np.int64)
        parts += [(h, m, post.astype(np.float32), obs[-1], int(cuts[r]), int(cuts[r + 1])) for r in range(nr)]
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda a: oracle.rollout(a[1], a[2], a[3], a[0].horizon, a[0].seed, a[0].human_id, a[4], a[5],
                                             grid=a[0].grid), parts))
    dt = time.perf_counter() - t0
    ps = sum(n * h.horizon for h, _, _, n in jobs)
    out["batched_sampled"] = {"value": ps / dt, "cores": threads,
                              "sample": f"1/50 of each of the 16 humans' particles ({ps:.3g} particle-steps) "
                                        f"+ their 50-step belief updates, FP64 C ({dt:.2f} s wall)"}
    m = oracle.Model(hu.K, hu.speed, hu.dt, hu.goals, hu.beta)
    obs = oracle.simulate(m, hu.true_j, hu.start, hu.n_obs, hu.obs_seed, hu.human_id)
    post, _ = oracle.update_posterior(m, obs, hu.uniform_log_prior())
    t0 = time.perf_counter()
    oracle.exact_occupancy(m, post, obs[-1], hu.horizon, hu.grid)
    out["exact_propagation_plain_small_s"] = time.perf_counter() - t0
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    hu = MAIN_WORKLOADS[args.workload][0]()
    per_step = []
    threads = host_threads()
    n = max(1000, args.cpu_sample // 4) * threads
    for _ in range(args.warmup):
        oracle_sample(hu, max(200, n // 10), threads=threads)
    for _ in range(args.steps):
        r = oracle_sample(hu, n, threads=threads)
        per_step.append(n * hu.horizon / r["value"])
    total = sum(per_step)
    value = n * hu.horizon * args.steps / total
    # n_gpus is the launch's N (the line pairs with the native arm's); the
    # oracle itself runs on rank 0's host cores only
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "gpus_used": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (model-drawn observations, seeded)", "config": workload_config(hu, args.workload),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": f"{n} of {hu.n_particles} particles x T={hu.horizon} per step, "
                                       f"{threads} host threads over particle ranges"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def load_profile_traffic(kernel_hash, workload="paper_scale"):
    """DRAM bytes per launch of the rollout kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"rollout_{workload}.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_sources_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_launch")


def gpu_paths(pm, ctx, torch, dev, hu, n_steps, human_id, start=None):
    """Observed trajectory drawn from the model on the GPU: one traced particle
    whose belief is a point mass on the true component."""
    goals = torch.tensor(hu.goals, device=dev)
    beta = torch.tensor(hu.beta, device=dev)
    model = pm.make_model(hu.K, hu.speed, hu.dt, goals, beta, speeds=speeds_of(hu))
    J = hu.G * hu.B
    onehot = torch.full((J,), -float("inf"), device=dev)
    onehot[hu.true_j] = 0.0
    st = torch.empty((1, n_steps, 2), device=dev)
    z = hu.start if start is None else start
    pm.pm_predict_occupancy_traced(ctx, model, onehot, float(z[0]), float(z[1]), 1, n_steps, None,
                                   hu.obs_seed, human_id, None, None, 1, st, None, None)
    return torch.cat([torch.tensor(np.asarray(z, np.float32), device=dev).view(1, 2), st[0]], 0).contiguous()


def speeds_of(hu):
    """The control set's speed multipliers (None: one speed)."""
    return None if tuple(hu.speeds) == (1.0,) else tuple(hu.speeds)


def time_events(torch, stream, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_extra(args, pm, ctx, torch, dev, stream, sfu_peak):
    """Batched, serving, differentiation and small-case numbers (secondary
    workloads; each quoted with its own unit)."""
    out = {}

    def want(name):
        return "all" in args.sections or name in args.sections

    # -- plain_small: latency of one prediction (1 human, K = 8, N = 10k, T = 20)
    hu = workloads.plain_small()
    g, b = torch.tensor(hu.goals, device=dev), torch.tensor(hu.beta, device=dev)
    model = pm.make_model(hu.K, hu.speed, hu.dt, g, b)
    obs = gpu_paths(pm, ctx, torch, dev, hu, hu.n_obs, hu.human_id)
    z0 = obs[-1].cpu().numpy()
    prior = torch.tensor(hu.uniform_log_prior(), device=dev)
    lb = torch.empty_like(prior)
    x0, y0, res, W, H = hu.grid
    grid = pm.make_grid(x0, y0, res, W, H)
    counts = torch.empty((hu.horizon, H, W), dtype=torch.int32, device=dev)
    oob = torch.empty(hu.horizon, dtype=torch.int32, device=dev)

    def small():
        pm.pm_update_posterior_into(ctx, model, obs, hu.n_obs, prior, lb, stream)
        pm.pm_predict_occupancy(ctx, model, lb, float(z0[0]), float(z0[1]), hu.n_particles, hu.horizon, grid,
                                hu.seed, hu.human_id, counts, oob, stream)
    ms = time_events(torch, stream, small, 200)
    out["plain_small"] = {"ms_per_prediction": ms, "hz": 1e3 / ms,
                          "particle_steps_per_s": hu.n_particles * hu.horizon / (ms * 1e-3)}

    if want("batched"):
        # -- batched: 16 humans, one persistent launch in a CUDA graph vs the plain per-human path
        hs = workloads.batched()
        recs = []
        # every human's prior and belief are slices of two flat buffers, so
        # one copy resets all beliefs before a replay
        offs = np.cumsum([0] + [h.G * h.B for h in hs])
        prior_flat = torch.tensor(np.concatenate([h.uniform_log_prior() for h in hs]), device=dev)
        lb_flat = prior_flat.clone()
        for k, h in enumerate(hs):
            gg, bb = torch.tensor(h.goals, device=dev), torch.tensor(h.beta, device=dev)
            ob = gpu_paths(pm, ctx, torch, dev, h, h.n_obs, h.human_id)
            x0, y0, res, W, H = h.grid
            recs.append(dict(h=h, g=gg, b=bb, obs=ob, prior=prior_flat[offs[k]:offs[k + 1]],
                             lb=lb_flat[offs[k]:offs[k + 1]], z0=ob[-1].clone(),
                             grid=pm.make_grid(x0, y0, res, W, H),
                             counts=torch.empty((h.horizon, H, W), dtype=torch.int32, device=dev),
                             oob=torch.empty(h.horizon, dtype=torch.int32, device=dev),
                             model=pm.make_model(h.K, h.speed, h.dt, gg, bb)))
        steps = sum(r["h"].n_particles * r["h"].horizon for r in recs)

        def plain_batched():
            for r in recs:
                pm.pm_update_posterior_into(ctx, r["model"], r["obs"], r["h"].n_obs, r["prior"], r["lb"], stream)
                z = r["z0h"]
                pm.pm_predict_occupancy(ctx, r["model"], r["lb"], z[0], z[1], r["h"].n_particles, r["h"].horizon,
                                        r["grid"], r["h"].seed, r["h"].human_id, r["counts"], r["oob"], stream)
        for r in recs:
            r["z0h"] = [float(v) for v in r["z0"].cpu().numpy()]
        plain_ms = time_events(torch, stream, plain_batched, 5)
        batch = pm.pm_batch_create(ctx, recs[0]["model"], len(recs))
        humans = [pm.make_human(r["g"], r["b"], r["lb"], r["z0"], r["h"].n_particles, r["h"].horizon, r["grid"],
                                r["h"].seed, r["h"].human_id, r["counts"], r["oob"], obs_xy=r["obs"],
                                n_obs=r["h"].n_obs) for r in recs]
        pm.pm_batch_set(batch, humans, stream)
        pm.pm_batch_set_zeroing(batch, 1, stream)  # only reachable cells: the outputs are only read
        t0 = time.perf_counter()
        pm.pm_batch_autotune(batch, stream)
        tune_s = time.perf_counter() - t0
        tuned = pm.pm_batch_get_config(batch)
        side = torch.cuda.Stream()

        def batched_step():
            # the zeroing on a second stream, beside the belief update
            lb_flat.copy_(prior_flat)
            side.wait_stream(stream)
            pm.pm_batch_zero(batch, side)
            pm.pm_batch_update_posterior(batch, stream)
            stream.wait_stream(side)
            pm.pm_batch_rollout(batch, stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            lb_flat.copy_(prior_flat)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=stream):
                batched_step()
        batch_ms = time_events(torch, stream, graph.replay, 10)
        # grid epilogue: every human's counts blurred (sigma 1.5 cells) and
        # max-united on the shared 400 x 400 grid
        x0, y0, res, W, H = recs[0]["h"].grid
        T_max = max(r["h"].horizon for r in recs)
        union = torch.empty((T_max, H, W), device=dev)
        ugrid = pm.make_grid(x0, y0, res, W, H)

        def do_union():
            pm.pm_batch_union(batch, 1.5, T_max, ugrid, union, stream)
        dense_ms = time_events(torch, stream, do_union, 10)  # no block marks: every region is read
        # with block marks: the rollout marks occupied 16 x 16 blocks, the union reads only those
        pm.pm_batch_set_block_flags(batch, 1, stream)
        graph_m = torch.cuda.CUDAGraph()  # the kernel variant is fixed at capture: capture again
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            with torch.cuda.graph(graph_m, stream=stream):
                batched_step()
        marked_batch_ms = time_events(torch, stream, graph_m.replay, 10)
        union_ms = time_events(torch, stream, do_union, 10)
        pm.pm_batch_set_block_flags(batch, 0, stream)
        torch.cuda.synchronize()
        dense_bytes = sum(r["h"].horizon for r in recs) * H * W * 4 + T_max * H * W * 4
        # algorithmic bytes: the occupied blocks' counts (what any union must read) + the output
        occ_blocks = 0
        for r in recs:
            c = r["counts"]
            Tb, Hc, Wc = c.shape
            cc = torch.nn.functional.pad(c, (0, (-Wc) % 16, 0, (-Hc) % 16))
            occ_blocks += int((cc.reshape(Tb, cc.shape[1] // 16, 16, cc.shape[2] // 16, 16).amax(dim=(2, 4)) > 0).sum())
        union_bytes = occ_blocks * 16 * 16 * 4 + T_max * H * W * 4
        pm.pm_batch_destroy(batch)
        out["batched"] = {"humans": len(recs), "particle_steps": steps,
                          "batched_ms": batch_ms, "batched_particle_steps_per_s": steps / (batch_ms * 1e-3),
                          "plain_ms": plain_ms, "plain_particle_steps_per_s": steps / (plain_ms * 1e-3),
                          "speedup_vs_plain": plain_ms / batch_ms, "autotune_s": tune_s,
                          "tuned": tuned,
                          "rate_vs_plain_small": steps / (batch_ms * 1e-3) / out["plain_small"]["particle_steps_per_s"],
                          "sfu_roofline_frac": steps / (batch_ms * 1e-3) * 2 * 36 / sfu_peak,
                          "union": {"ms": union_ms, "sigma_cells": 1.5, "bytes": union_bytes,
                                    "GB_per_s": union_bytes / (union_ms * 1e-3) / 1e9,
                                    "hbm_frac": union_bytes / (union_ms * 1e-3) / 1e9 / HBM_PEAK_GBS,
                                    "dense_ms": dense_ms, "dense_bytes": dense_bytes,
                                    "dense_GB_per_s": dense_bytes / (dense_ms * 1e-3) / 1e9,
                                    "batched_ms_with_marks": marked_batch_ms}}
        del recs

    if want("batched_small"):
        # -- 64 humans of the plain configuration's shape: one graph replay of the
        # batched form vs the same humans through the single-human calls in sequence
        hs = workloads.plain_crowd(64)
        offs = np.cumsum([0] + [h.G * h.B for h in hs])
        prior_flat = torch.tensor(np.concatenate([h.uniform_log_prior() for h in hs]), device=dev)
        lb_flat = prior_flat.clone()
        recs = []
        for k, h in enumerate(hs):
            gg, bb = torch.tensor(h.goals, device=dev), torch.tensor(h.beta, device=dev)
            ob = gpu_paths(pm, ctx, torch, dev, h, h.n_obs, h.human_id)
            x0, y0, res, W, H = h.grid
            recs.append(dict(h=h, g=gg, b=bb, obs=ob, prior=prior_flat[offs[k]:offs[k + 1]],
                             lb=lb_flat[offs[k]:offs[k + 1]], z0=ob[-1].clone(),
                             z0h=[float(v) for v in ob[-1].cpu().numpy()], grid=pm.make_grid(x0, y0, res, W, H),
                             counts=torch.empty((h.horizon, H, W), dtype=torch.int32, device=dev),
                             oob=torch.empty(h.horizon, dtype=torch.int32, device=dev),
                             model=pm.make_model(h.K, h.speed, h.dt, gg, bb)))
        steps = sum(r["h"].n_particles * r["h"].horizon for r in recs)

        def one_by_one():
            for r in recs:
                pm.pm_update_posterior_into(ctx, r["model"], r["obs"], r["h"].n_obs, r["prior"], r["lb"], stream)
                pm.pm_predict_occupancy(ctx, r["model"], r["lb"], r["z0h"][0], r["z0h"][1], r["h"].n_particles,
                                        r["h"].horizon, r["grid"], r["h"].seed, r["h"].human_id, r["counts"],
                                        r["oob"], stream)
        plain_ms = time_events(torch, stream, one_by_one, 10)
        batch = pm.pm_batch_create(ctx, recs[0]["model"], len(recs))
        try:
            humans = [pm.make_human(r["g"], r["b"], r["lb"], r["z0"], r["h"].n_particles, r["h"].horizon, r["grid"],
                                    r["h"].seed, r["h"].human_id, r["counts"], r["oob"], obs_xy=r["obs"],
                                    n_obs=r["h"].n_obs) for r in recs]
            pm.pm_batch_set(batch, humans, stream)
            pm.pm_batch_set_zeroing(batch, 1, stream)
            pm.pm_batch_autotune(batch, stream)
            side = torch.cuda.Stream()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.stream(stream):
                torch.cuda.synchronize()
                with torch.cuda.graph(graph, stream=stream):
                    lb_flat.copy_(prior_flat)
                    side.wait_stream(stream)
                    pm.pm_batch_zero(batch, side)  # beside the belief update
                    pm.pm_batch_update_posterior(batch, stream)
                    stream.wait_stream(side)
                    pm.pm_batch_rollout(batch, stream)
            batch_ms = time_events(torch, stream, graph.replay, 20)
            out["batched_small"] = {"humans": len(recs), "particle_steps": steps, "batched_ms": batch_ms,
                                    "batched_particle_steps_per_s": steps / (batch_ms * 1e-3),
                                    "one_by_one_ms": plain_ms,
                                    "one_by_one_particle_steps_per_s": steps / (plain_ms * 1e-3),
                                    "speedup_vs_one_by_one": plain_ms / batch_ms}
        finally:
            pm.pm_batch_destroy(batch)
        del recs

    if want("serving"):
        # -- serving: 64 live humans forced, one frame per observation
        from paper_2603_01122_gb300.serving import Server, run_arrivals
        wl = workloads.serving()
        arr = wl["arrivals"]
        hu0 = arr[0].human
        srv = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, max_live=64, n_particles=hu0.n_particles,
                     horizon=hu0.horizon, window=hu0.window)
        try:
            live = []
            paths = []
            for i in range(64):
                h = arr[i % len(arr)].human
                p = gpu_paths(pm, ctx, torch, dev, h, args.serving_frames + 1, h.human_id + 100000 * (i // len(arr)))
                paths.append(p.cpu().numpy())
                s_ = srv.admit(i, h.goals, h.beta, paths[-1][0], h.seed, h.human_id + 100000 * (i // len(arr)))
                live.append(s_)
            lat = []
            for f in range(args.serving_frames):
                for i, s_ in enumerate(live):
                    if f >= 1:
                        srv.observe(s_, paths[i][f])
                lat.append(srv.frame())
            lat = np.array(lat[5:])
            ps = srv.particle_steps_per_frame()
            # plain path for the same 64 humans: one belief update and one prediction per human
            x0, y0, res, W, H = hu0.grid
            win = hu0.window
            plain_counts = torch.empty((hu0.horizon, win, win), dtype=torch.int32, device=dev)
            plain_oob = torch.empty(hu0.horizon, dtype=torch.int32, device=dev)
            models = []
            for s_ in live:
                m_ = srv.meta[s_]
                models.append((pm.make_model(hu0.K, hu0.speed, hu0.dt, srv.goals[s_, :m_["G"]].contiguous(),
                                             srv.beta[s_, :m_["B"]].contiguous()), s_, m_))
            zh = srv.obs_dev[:, 1].cpu().numpy()

            def plain_frame():
                for model_, s_, m_ in models:
                    pm.pm_update_posterior(ctx, model_, srv.obs_dev[s_], 1, srv.log_b[s_], stream)
                    z = zh[s_]
                    gx0 = float(np.float32(x0 + (np.floor((z[0] - x0) / res) - (win - 1) // 2) * res))
                    gy0 = float(np.float32(y0 + (np.floor((z[1] - y0) / res) - (win - 1) // 2) * res))
                    pm.pm_predict_occupancy(ctx, model_, srv.log_b[s_], float(z[0]), float(z[1]), hu0.n_particles,
                                            hu0.horizon, pm.make_grid(gx0, gy0, res, win, win), m_["seed"],
                                            m_["human_id"], plain_counts, plain_oob, stream)
            plain_ms = time_events(torch, stream, plain_frame, 3)
            out["serving_forced_64"] = {
                "live": 64, "frames": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
                "particle_steps_per_frame": ps, "particle_steps_per_s": ps / float(np.median(lat)),
                "plain_path_ms_per_frame": plain_ms, "speedup_vs_plain": plain_ms / float(np.median(lat) * 1e3),
                "rate_vs_plain_small": ps / float(np.median(lat)) / out["plain_small"]["particle_steps_per_s"],
                "sfu_roofline_frac": ps / float(np.median(lat)) * 2 * 36 / sfu_peak}
            # the same frames with the grid epilogue (blur + max-union on the room grid) in the graph
            srv_u = Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, max_live=64, n_particles=hu0.n_particles,
                           horizon=hu0.horizon, window=hu0.window, union_sigma=1.5)
            try:
                live_u = []
                for i in range(64):
                    h = arr[i % len(arr)].human
                    live_u.append(srv_u.admit(i, h.goals, h.beta, paths[i][0], h.seed,
                                              h.human_id + 100000 * (i // len(arr))))
                lat_u = []
                for f in range(min(args.serving_frames, 120)):
                    for i, s_ in enumerate(live_u):
                        if f >= 1:
                            srv_u.observe(s_, paths[i][f])
                    lat_u.append(srv_u.frame())
                lat_u = np.array(lat_u[5:])
                out["serving_forced_64"]["with_union"] = {
                    "frames": int(lat_u.size), "p50_ms": float(np.percentile(lat_u, 50) * 1e3),
                    "p99_ms": float(np.percentile(lat_u, 99) * 1e3), "sigma_cells": 1.5}
                # MPPI local planner on that union grid: 8192 perturbed sequences of
                # 30 steps of 0.1 s (every 5th prediction step)
                Nm, Tm = 8192, 30
                rng = np.random.default_rng([workloads.MASTER_SEED, 9])
                mp = pm.make_mppi(Nm, Tm, 0.1, 5, [3.0, 3.0, 10.0, 0.0], [0.6, 0.6, 2.0, 0.0], [2.0, 1.0],
                                  [15.0, 15.0, 0.5, 0.0], 0.1, 1000.0, 0.1, 2.0)
                u_ref = torch.zeros((Tm, 2), device=dev)
                delta = torch.tensor((rng.normal(size=(Tm, Nm, 2)) * [0.6, 0.5]).astype(np.float32), device=dev)
                ctg = torch.empty((Tm, Nm), device=dev)
                u_opt = torch.empty((Tm, 2), device=dev)
                x0, y0, res, W, H = hu0.grid
                rg = pm.make_grid(x0, y0, res, W, H)

                def mppi():
                    pm.pm_mppi_solve(ctx, mp, [5.0, 5.0, 0.5, 0.6], u_ref, delta, srv_u.union, hu0.horizon, rg, ctg,
                                     u_opt, stream)
                mppi_ms = time_events(torch, stream, mppi, 20)
                out["mppi"] = {"ms_per_solve": mppi_ms, "samples": Nm, "steps": Tm,
                               "sample_steps_per_s": Nm * Tm / (mppi_ms * 1e-3)}
            finally:
                srv_u.close()
            if args.serving_seconds > 0:
                paths2 = []
                for a in arr:
                    n = int((a.t_leave - a.t_arrive) * wl["frame_hz"]) + 2
                    paths2.append(gpu_paths(pm, ctx, torch, dev, a.human, min(n, 4096), a.human.human_id).cpu().numpy())
                res2 = run_arrivals(srv_fresh := Server(ctx, hu0.K, hu0.speed, hu0.dt, hu0.grid, max_live=64,
                                                        n_particles=hu0.n_particles, horizon=hu0.horizon,
                                                        window=hu0.window),
                                    arr, paths2, frame_hz=wl["frame_hz"], duration_s=args.serving_seconds)
                srv_fresh.close()
                l2 = res2["latency_s"]
                out["serving_poisson"] = {"seconds": args.serving_seconds, "frames": int(l2.size),
                                          "p50_ms": float(np.percentile(l2, 50) * 1e3),
                                          "p99_ms": float(np.percentile(l2, 99) * 1e3),
                                          "mean_live": float(res2["live"].mean()), "max_live": int(res2["live"].max()),
                                          "frames_waited": res2["frames_waited"]}
        finally:
            srv.close()

    if want("speeds"):
        # -- several speeds: |U| = 96 controls (3 speeds x K = 32), and the same
        #    human standing still (the two faster speeds masked)
        for name, stationary in (("multi_speed", False), ("multi_speed_stationary", True)):
            hu = workloads.multi_speed(stationary=stationary)
            g, b = torch.tensor(hu.goals, device=dev), torch.tensor(hu.beta, device=dev)
            model = pm.make_model(hu.K, hu.speed, hu.dt, g, b, speeds=hu.speeds, speed_off=hu.speed_off)
            gen = workloads.multi_speed()
            obs = gpu_paths(pm, ctx, torch, dev, gen, hu.n_obs, hu.human_id)
            z0 = obs[-1].cpu().numpy()
            prior = torch.tensor(hu.uniform_log_prior(), device=dev)
            lb = torch.empty_like(prior)
            x0, y0, res, W, H = hu.grid
            grid = pm.make_grid(x0, y0, res, W, H)
            counts = torch.empty((hu.horizon, H, W), dtype=torch.int32, device=dev)
            oob = torch.empty(hu.horizon, dtype=torch.int32, device=dev)

            def ms_step():
                pm.pm_update_posterior_into(ctx, model, obs, hu.n_obs, prior, lb, stream)
                pm.pm_predict_occupancy(ctx, model, lb, float(z0[0]), float(z0[1]), hu.n_particles, hu.horizon,
                                        grid, hu.seed, hu.human_id, counts, oob, stream)
            ms = time_events(torch, stream, ms_step, 20)
            u_on = hu.K * sum(1 for q in range(len(hu.speeds)) if not (hu.speed_off >> q) & 1)
            rate = hu.n_particles * hu.horizon / (ms * 1e-3)
            out[name] = {"ms_per_prediction": ms, "particle_steps_per_s": rate, "controls_enabled": u_on,
                         "sfu_roofline_frac": rate * 2 * u_on / sfu_peak}

    if want("table1"):
        # -- Table 1's configuration (1 human, n = 8192, |G| = 10, |B| = 5, |U| = 96,
        #    50 x 50 grid) at T = 2..10: wall clock of one prediction, as the paper
        #    times it (warm, mean of repeated runs; here event-timed on the stream)
        t1 = {}
        for T in (2, 4, 6, 8, 10):
            hu = workloads.table1(horizon=T)
            g, b = torch.tensor(hu.goals, device=dev), torch.tensor(hu.beta, device=dev)
            model = pm.make_model(hu.K, hu.speed, hu.dt, g, b, speeds=hu.speeds)
            obs = gpu_paths(pm, ctx, torch, dev, hu, hu.n_obs, hu.human_id)
            z0 = obs[-1].cpu().numpy()
            prior = torch.tensor(hu.uniform_log_prior(), device=dev)
            lb = torch.empty_like(prior)
            x0, y0, res, W, H = hu.grid
            grid = pm.make_grid(x0, y0, res, W, H)
            counts = torch.empty((T, H, W), dtype=torch.int32, device=dev)
            oob = torch.empty(T, dtype=torch.int32, device=dev)

            def t1_step():
                pm.pm_update_posterior_into(ctx, model, obs, hu.n_obs, prior, lb, stream)
                pm.pm_predict_occupancy(ctx, model, lb, float(z0[0]), float(z0[1]), hu.n_particles, T, grid,
                                        hu.seed, hu.human_id, counts, oob, stream)
            t1[f"T{T}"] = time_events(torch, stream, t1_step, 200)
        out["table1"] = {"ms_per_prediction": t1,
                         "paper_ms_rtx2080ti_gpu_jit": {"T2": 7.0, "T4": 7.0, "T6": 7.0, "T8": 7.0, "T10": 8.0}}

    if want("differentiation"):
        # -- differentiation: 256 trajectories, adjoint of the marginal log-likelihood
        ts = workloads.differentiation()
        trajs = []
        for m in range(ts.M):
            h = workloads.Human(K=ts.K, speed=ts.speed, dt=ts.dt, goals=ts.goals[ts.true_goal[m]:ts.true_goal[m] + 1],
                                beta=ts.true_beta[m:m + 1], true_j=0, start=ts.starts[m], n_obs=0, n_particles=1,
                                horizon=1, grid=(0, 0, 1, 1, 1), seed=0, human_id=m, obs_seed=ts.obs_seed)
            trajs.append(gpu_paths(pm, ctx, torch, dev, h, int(ts.lengths[m]), m))
        offsets = torch.tensor(np.cumsum([0] + [t.shape[0] for t in trajs]), dtype=torch.int32, device=dev)
        traj = torch.cat(trajs, 0).contiguous()
        gg, bb = torch.tensor(ts.goals, device=dev), torch.tensor(ts.beta, device=dev)
        model = pm.make_model(ts.K, ts.speed, ts.dt, gg, bb)
        lp = torch.full((40,), -float(np.log(40.0)), device=dev)
        L = torch.empty(1, device=dev)
        dg, dv, dw = torch.empty_like(gg), torch.empty(1, device=dev), torch.empty(2, device=dev)

        def adj():
            pm.pm_loglik_backward(ctx, model, ts.M, offsets, traj.shape[0], traj, lp, 1.0, L, dg, dv, dw, stream)
        ms = time_events(torch, stream, adj, 20)
        nsteps = int(traj.shape[0]) - ts.M
        out["differentiation"] = {"ms_per_backward": ms, "trajectory_steps_per_s": nsteps / (ms * 1e-3),
                                  "q_evals_per_s": nsteps * 40 * (ts.K + 1) / (ms * 1e-3),
                                  # algorithmic SFU results: K + 1 distances and K exponentials
                                  # per step and component
                                  "sfu_roofline_frac": nsteps * 40 * (2 * ts.K + 1) / (ms * 1e-3) / sfu_peak}
    return out


def sig(x, n=4):
    """x rounded to n significant digits (None passes through)."""
    if x is None:
        return None
    x = float(x)
    return float(f"{x:.{n}g}")


def target_summary(line, extra):
    """The figures the targets are stated in, compact: the rollout's SFU
    fraction, the batched and served rates against the plain per-human path
    (the plain configuration's rate, and the same humans issued one by one,
    also for 64 humans of the plain configuration's shape) and the 64-human
    frame latency with and without the grid epilogue."""
    t = {"rollout_sfu_frac": sig(line["roofline"]["frac"], 3), "value": sig(line["value"])}
    if not extra:
        return t
    t["plain_small_rate"] = sig(extra["plain_small"]["particle_steps_per_s"])
    b = extra.get("batched")
    if b:
        t["batched"] = {"rate": sig(b["batched_particle_steps_per_s"]), "sfu_frac": sig(b["sfu_roofline_frac"], 3),
                        "x_plain_small": sig(b["rate_vs_plain_small"], 3),
                        "x_same_humans_one_by_one": sig(b["speedup_vs_plain"], 3), "ms": sig(b["batched_ms"])}
    c = extra.get("batched_small")
    if c:
        t["batched_small_64"] = {"rate": sig(c["batched_particle_steps_per_s"]), "ms": sig(c["batched_ms"]),
                                 "x_same_humans_one_by_one": sig(c["speedup_vs_one_by_one"], 3)}
    f = extra.get("serving_forced_64")
    if f:
        t["served_64"] = {"p50_ms": sig(f["p50_ms"]), "p99_ms": sig(f["p99_ms"]),
                          "with_union_p99_ms": sig(f.get("with_union", {}).get("p99_ms")),
                          "with_union_p50_ms": sig(f.get("with_union", {}).get("p50_ms")),
                          "rate": sig(f["particle_steps_per_s"]), "sfu_frac": sig(f["sfu_roofline_frac"], 3),
                          "x_plain_small": sig(f["rate_vs_plain_small"], 3),
                          "x_same_humans_one_by_one": sig(f["speedup_vs_plain"], 3)}
    p = extra.get("serving_poisson")
    if p:
        t["served_poisson"] = {"p50_ms": sig(p["p50_ms"]), "p99_ms": sig(p["p99_ms"]), "max_live": p["max_live"]}
    d = extra.get("differentiation")
    if d:
        t["adjoint_ms"] = sig(d["ms_per_backward"])
    m = extra.get("multi_speed")
    if m:
        t["multi_speed_sfu_frac"] = sig(m["sfu_roofline_frac"], 3)
    return t


def run_native(args):
    import torch
    import torch.distributed as tdist

    import paper_2603_01122_gb300 as pm

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    pm.build()
    ctx = pm.pm_create(local)
    stream = torch.cuda.Stream(device=dev)

    make_hu, kernel_name = MAIN_WORKLOADS[args.workload]
    hu = make_hu()
    human_id = rank_human_id(hu.human_id, rank)
    K, N, T = hu.K, hu.n_particles, hu.horizon
    U = K * sum(1 for q in range(len(hu.speeds)) if not (hu.speed_off >> q) & 1)  # enabled controls
    x0, y0, res, W, H = hu.grid
    goals = torch.tensor(hu.goals, device=dev)
    beta = torch.tensor(hu.beta, device=dev)
    model = pm.make_model(K, hu.speed, hu.dt, goals, beta, speeds=speeds_of(hu), speed_off=hu.speed_off)
    grid = pm.make_grid(x0, y0, res, W, H)

    # Observed history drawn from the model by the library itself: one traced
    # particle whose belief is a point mass on the true component.
    J = hu.G * hu.B
    onehot = torch.full((J,), -float("inf"), device=dev)
    onehot[hu.true_j] = 0.0
    hist_states = torch.empty((1, hu.n_obs, 2), device=dev)
    pm.pm_predict_occupancy_traced(ctx, model, onehot, float(hu.start[0]), float(hu.start[1]), 1, hu.n_obs,
                                   None, hu.obs_seed, human_id, None, None, 1, hist_states, None, None)
    obs = torch.cat([torch.tensor(hu.start, device=dev).view(1, 2), hist_states[0]], 0).contiguous()
    torch.cuda.synchronize()
    obs_host = obs.cpu().numpy()
    z0 = obs_host[-1]
    prior = torch.tensor(hu.uniform_log_prior(), device=dev)
    lb = torch.empty_like(prior)
    counts = torch.empty((T, H, W), dtype=torch.int32, device=dev)
    oob = torch.empty((T,), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    side = torch.cuda.Stream()

    def step(ev=None):
        """One step: the outputs zeroed on a second stream beside the belief
        update, then the rollout; ev = (start, after the update, rollout
        start, end) events on the main stream."""
        if ev:
            ev[0].record(stream)
        side.wait_stream(stream)
        pm.pm_zero_occupancy(ctx, T, grid, counts, oob, side)
        pm.pm_update_posterior_into(ctx, model, obs, hu.n_obs, prior, lb, stream)
        if ev:
            ev[1].record(stream)
        stream.wait_stream(side)
        if ev:
            ev[2].record(stream)
        pm.pm_rollout_occupancy(ctx, model, lb, float(z0[0]), float(z0[1]), N, T, grid, hu.seed, human_id,
                                counts, oob, stream)
        if ev:
            ev[3].record(stream)

    # SFU peak (roofline denominator), measured before the timed region
    sfu = {"ex2": pm.pm_probe_sfu(ctx, 0), "sqrt": pm.pm_probe_sfu(ctx, 1), "rsqrt": pm.pm_probe_sfu(ctx, 2)}
    info = pm.pm_device_info(ctx)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
    torch.cuda.synchronize()

    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(args.steps)]
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    phys = vis.split(",")[local] if vis and vis.split(",")[local].isdigit() else str(local)
    with ClockSampler(phys) as clk:
        # nvidia-smi samples every 200 ms, longer than a short timed region:
        # after it has started, the same steps run for about a second right
        # before the timed ones, and the clocks are those of the pre-roll and
        # the timed region together
        time.sleep(1.0)
        pre_t0 = time.time()
        pre = 0
        while time.time() - pre_t0 < 1.0:
            with torch.cuda.stream(stream):
                for _ in range(20):
                    flush.fill_(1.0)
                    step()
            torch.cuda.synchronize()
            pre += 20
        wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(float(i))
                step(ev[i])
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark(pre_t0, time.time())
        time.sleep(0.3)
    if world > 1:
        tdist.barrier()
    step_ms = [a.elapsed_time(d) for a, b, c, d in ev]
    roll_ms = [c.elapsed_time(d) for a, b, c, d in ev]
    post_ms = [a.elapsed_time(b) for a, b, c, d in ev]
    total_ms = max_over_ranks(sum(step_ms), world, tdist, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, N * T, ms_per_step * 1e-3)

    # roofline of the dominant kernel (the rollout): algorithmic SFU results
    # per launch (one exp + one sqrt per control and particle-step) / its
    # event-timed duration
    roll_avg_s = statistics.mean(roll_ms) * 1e-3
    sfu_ops = 2.0 * U * N * T
    achieved = sfu_ops / roll_avg_s / 1e9
    peak = 2.0 / (1.0 / sfu["ex2"] + 1.0 / sfu["sqrt"]) / 1e9
    khash = sources_hash(ROLLOUT_SOURCES)
    traffic = load_profile_traffic(khash, args.workload)

    # e2e through the host-buffer entry point (pinned buffers)
    goals_h = torch.tensor(hu.goals).pin_memory()
    beta_h = torch.tensor(hu.beta).pin_memory()
    obs_h = torch.tensor(obs_host).pin_memory()
    prior_h = torch.tensor(hu.uniform_log_prior()).pin_memory()
    post_h = torch.empty(J, dtype=torch.float32).pin_memory()
    counts_h = torch.empty((T, H, W), dtype=torch.int32).pin_memory()
    oob_h = torch.empty((T,), dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))

    def host_call():
        pm.pm_predict_host(ctx, model, goals_h, beta_h, obs_h, hu.n_obs, prior_h, N, T, grid, hu.seed,
                           human_id, post_h, counts_h, oob_h, stream)

    host_call()
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_call()
    e2e_sync_s = (time.perf_counter() - e0) / e2e_steps
    # the asynchronous host call, one prediction after another: each step
    # copies its inputs in and its posterior and histogram out (two sets of
    # pinned outputs alternate), and a step's copy-out overlaps the next step
    outs = [(post_h, counts_h, oob_h), (torch.empty(J, dtype=torch.float32).pin_memory(),
                                        torch.empty((T, H, W), dtype=torch.int32).pin_memory(),
                                        torch.empty((T,), dtype=torch.int32).pin_memory())]

    def host_async(i):
        po, co, oo = outs[i & 1]
        pm.pm_predict_host_async(ctx, model, goals_h, beta_h, obs_h, hu.n_obs, prior_h, N, T, grid, hu.seed,
                                 human_id, po, co, oo, stream)
    a_steps = max(3, min(args.steps, 50))
    for i in range(2):
        host_async(i)
    pm.pm_host_fence(ctx, stream)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(a_steps):
        host_async(i)
    pm.pm_host_fence(ctx, stream)
    stream.synchronize()
    e2e_s = (time.perf_counter() - e0) / a_steps
    h2d = (goals_h.numel() + beta_h.numel() + obs_h.numel() + prior_h.numel()) * 4
    d2h = (post_h.numel() + counts_h.numel() + oob_h.numel()) * 4
    e2e_value = job_throughput(world, N * T, max_over_ranks(e2e_s, world, tdist, dev))
    e2e_sync_value = job_throughput(world, N * T, max_over_ranks(e2e_sync_s, world, tdist, dev))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; observed history drawn from the model on the GPU)",
            "config": workload_config(hu, args.workload),
            # per step: the belief update, the zeroing of the outputs, the rollout
            "gpu_launches": 3 * args.steps,
            "wall_s": wall,
            "breakdown_ms": {"posterior": statistics.mean(post_ms), "rollout": statistics.mean(roll_ms)},
            "roofline": {"bound": "alu", "kernel": kernel_name, "achieved": achieved,
                         "peak": peak, "unit": "G SFU results/s", "frac": achieved / peak,
                         "traffic": traffic,
                         "peak_source": "measured by pm_probe_sfu (ex2/sqrt 1:1 harmonic mean); "
                                        f"ex2 {sfu['ex2'] / 1e9:.1f}, sqrt {sfu['sqrt'] / 1e9:.1f}, "
                                        f"rsqrt {sfu['rsqrt'] / 1e9:.1f} G/s",
                         "algorithmic": f"2U SFU results (U = {U} controls: U ex2 + U sqrt) per particle-step"},
            "device": info,
            "clocks": {**clk.summary(), "window": f"{pre} pre-roll steps + the timed region"},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "pm_predict_host_async (one prediction after another; each step's copy-out "
                           "overlaps the next step)", "steps": a_steps,
                    "sync_value": e2e_sync_value, "sync_api": "pm_predict_host (waits for each step's outputs)"},
            "paper_context": "125 Hz, 1 human, n=8192, T<=10, |U|=96, RTX 2080 Ti (Table 1)",
        }
        extra = None
        if not args.no_extra:
            extra = run_extra(args, pm, ctx, torch, dev, stream, peak * 1e9)
            line["extra"] = extra
        if not args.no_cpu_baseline:
            threads = host_threads()
            cb = oracle_sample(hu, args.cpu_sample * max(1, threads // 4), threads=threads)
            cb["one_thread"] = oracle_sample(hu, max(2000, args.cpu_sample // 4))["value"]
            cb["other_configs"] = oracle_other_configs(threads)
            line["cpu_baseline"] = cb
        # the target figures last, so that the end of the line carries them whole
        line["targets"] = target_summary(line, extra)
        print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    if world > 1:
        tdist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
