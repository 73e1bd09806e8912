"""125 Hz serving loop with continuous batching.

Every frame delivers one new observed state per live human and returns, for
every live human, the occupancy of the next T steps in a W x W window of the
room grid centred on the human's cell (Algorithm 1, bootstrapped belief).

* Continuous batching: humans are admitted into free slots between frames as
  soon as a slot and the device-memory budget allow, and retired when they
  leave; the next frame's single batched launch covers everyone live, so work
  of humans that arrived at different times overlaps on the device.
* Posteriors stay on the device: each slot keeps its log-belief; a frame
  updates it with the one new step (Eq. 3 / Eq. 7) and predicts from it.
* One frame = upload of the newest observations (page-locked host buffer ->
  device), the batched belief update beside the zeroing of the outputs (two
  streams) and the batched persistent rollout,
  replayed as one captured CUDA graph, launched with its completion event in
  one native call (``pm_graph_launch``). Membership changes re-upload the
  batch descriptors only; the graph reads them from device memory.
* Optionally (``union_sigma``) the frame also blurs every live human's window
  and max-unites them on the shared room grid (Sec. III-B, Sec. IV-B): the
  planner's input, in the same graph.
* Several speeds (``speeds``): a human seen standing still keeps only the
  controls that ``stationary_off`` leaves enabled (Sec. IV-B), set per human
  by ``set_stationary`` or, with ``stationary_eps``, from its last observed
  step; a change re-uploads the descriptors only. ``reset_belief`` returns a
  human to the uniform belief; with ``goal_radius`` the server does so itself
  when a human leaves a goal (``GoalDeparture``).
* Checkpoint and resume: ``export_state`` reads a live human's state (its
  device-resident log-belief, goals, beta grid, last two observed states,
  seed, human id, speed mask and goal-departure state) back as plain host
  data; ``import_state`` re-admits a human from it, on this server or on a
  new one, and the frames that follow equal those of an uninterrupted run.
* A frame in which a human has no new observation leaves its belief as it
  was (the step applied is of length zero) and predicts again from the same
  state.
* Each frame zeroes only the window cells that this frame's or the previous
  frame's particles of a slot can reach (``pm_batch_set_zeroing``; a frame
  after a membership change zeroes every cell): the occupancy tensors are the
  server's buffers, to be read, not written.
* Latency = host wall time from the start of the frame (observations in host
  memory) to the occupancy being ready on the device (event synchronised).

Only the slot bookkeeping is Python; every numeric step runs in libpm.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import (make_grid, make_human, make_model, pm_batch_create, pm_batch_destroy,
               pm_batch_rollout, pm_batch_set, pm_batch_set_block_flags, pm_batch_set_zeroing,
               pm_batch_union, pm_batch_update_posterior, pm_batch_zero, graph_launcher)


@dataclasses.dataclass
class SlotTable:
    """Admission by slots and a device-memory budget (host logic only)."""
    capacity: int
    budget_bytes: int
    slot_bytes: int

    def __post_init__(self):
        self.free: List[int] = list(range(self.capacity))[::-1]
        self.live: Dict[int, object] = {}

    @property
    def used_bytes(self) -> int:
        return len(self.live) * self.slot_bytes

    def can_admit(self) -> bool:
        return bool(self.free) and self.used_bytes + self.slot_bytes <= self.budget_bytes

    def admit(self, key) -> Optional[int]:
        if not self.can_admit():
            return None
        s = self.free.pop()
        self.live[s] = key
        return s

    def retire(self, slot: int) -> None:
        del self.live[slot]
        self.free.append(slot)
        self.free.sort(reverse=True)


@dataclasses.dataclass
class GoalDeparture:
    """Detects that a human has left a goal (host logic only): after one of its
    observed states came within ``radius`` of a goal, the first observed
    state farther than ``radius`` from every goal is a departure (the
    belief is then reset to uniform, Sec. IV-B)."""
    goals: np.ndarray
    radius: float

    def __post_init__(self):
        self.goals = np.asarray(self.goals, np.float64).reshape(-1, 2)
        self.at_goal = False

    def update(self, xy) -> bool:
        """Feed the newest observed state; True on a departure."""
        d = np.hypot(*(self.goals - np.asarray(xy, np.float64)[None, :]).T)
        near = bool((d <= self.radius).any())
        left = self.at_goal and not near
        self.at_goal = near
        return left


class Server:
    """Device-resident serving state for up to ``max_live`` humans sharing K, v,
    dt, w and the room grid; per-human goals (up to ``g_max``) and beta grid
    (up to ``b_max`` values)."""

    def __init__(self, ctx, K, speed, dt, room_grid, *, max_live=64, budget_bytes=4 << 30,
                 n_particles=50_000, horizon=150, window=121, g_max=6, b_max=10, w1=1.0, w2=1.0,
                 use_graph=True, device="cuda:0", union_sigma=None, speeds=None, stationary_off=0,
                 stationary_eps=None, goal_radius=None, snap_heading=False):
        import torch

        self.torch = torch
        self.ctx = ctx
        self.dev = torch.device(device)
        self.K, self.speed, self.dt, self.w1, self.w2 = K, speed, dt, w1, w2
        self.N, self.T, self.win = n_particles, horizon, window
        self.g_max, self.b_max = g_max, b_max
        self.room = room_grid
        x0, y0, res, _, _ = room_grid
        self.grid = make_grid(x0, y0, res, window, window)
        self.slot_bytes = (horizon * window * window + horizon) * 4 + (g_max * 2 + b_max + g_max * b_max + 4) * 4
        self.slots = SlotTable(max_live, budget_bytes, self.slot_bytes)
        cap = max_live
        self.counts = torch.zeros((cap, horizon, window, window), dtype=torch.int32, device=self.dev)
        self.oob = torch.zeros((cap, horizon), dtype=torch.int32, device=self.dev)
        self.goals = torch.zeros((cap, g_max, 2), dtype=torch.float32, device=self.dev)
        self.beta = torch.zeros((cap, b_max), dtype=torch.float32, device=self.dev)
        self.log_b = torch.zeros((cap, g_max * b_max), dtype=torch.float32, device=self.dev)
        self.obs_dev = torch.zeros((cap, 2, 2), dtype=torch.float32, device=self.dev)
        self.obs_host = torch.zeros((cap, 2, 2), dtype=torch.float32).pin_memory()
        self.meta: Dict[int, dict] = {}
        self.stream = torch.cuda.Stream(device=self.dev)
        self.side = torch.cuda.Stream(device=self.dev)
        self.done = torch.cuda.Event()
        shared_goals = torch.zeros((1, 2), device=self.dev)
        shared_beta = torch.ones(1, device=self.dev)
        self.speeds = None if speeds is None else tuple(float(m) for m in speeds)
        if stationary_off and (self.speeds is None or len(self.speeds) < 2):
            raise ValueError("stationary masking needs several speeds")
        self.stationary_off = int(stationary_off)
        self.stationary_eps = stationary_eps
        self.goal_radius = goal_radius
        self._shared = make_model(K, speed, dt, shared_goals, shared_beta, w1=w1, w2=w2, speeds=self.speeds,
                                  snap_heading=snap_heading)
        self.batch = pm_batch_create(ctx, self._shared, cap)
        pm_batch_set_zeroing(self.batch, 1)
        if union_sigma is not None:  # the union reads only the blocks the rollout marks
            pm_batch_set_block_flags(self.batch, 1)
        self.union_sigma = union_sigma
        self.union = None
        if union_sigma is not None:
            _, _, _, RW, RH = room_grid
            self.union_grid = make_grid(x0, y0, res, RW, RH)
            self.union = torch.zeros((horizon, RH, RW), dtype=torch.float32, device=self.dev)
        self.use_graph = use_graph
        self.graph = None
        self._launch = None  # the captured frame, launched and awaited natively
        self.dirty = True
        self.frames = 0

    def close(self):
        self.torch.cuda.synchronize()
        pm_batch_destroy(self.batch)

    # -- membership ------------------------------------------------------------
    def admit(self, key, goals, beta, start, seed, human_id) -> Optional[int]:
        """Take a free slot for a new human (uniform prior over its (beta, g),
        Sec. III-B); returns the slot or None when no slot or budget is left."""
        G, B = len(goals), len(beta)
        if G > self.g_max or B > self.b_max:
            raise ValueError("goal count or beta grid larger than the slot layout")
        s = self.slots.admit(key)
        if s is None:
            return None
        t = self.torch
        with t.cuda.stream(self.stream):
            self.goals[s, :G].copy_(t.as_tensor(np.asarray(goals, np.float32)))
            self.beta[s, :B].copy_(t.as_tensor(np.asarray(beta, np.float32)))
        self.meta[s] = dict(key=key, G=G, B=B, seed=int(seed), human_id=int(human_id), speed_off=0,
                            departure=None if self.goal_radius is None else GoalDeparture(goals, self.goal_radius))
        self.reset_belief(s)
        self.obs_host[s, 0] = t.as_tensor(np.asarray(start, np.float32))
        self.obs_host[s, 1] = self.obs_host[s, 0]
        self.dirty = True
        return s

    def retire(self, slot: int) -> None:
        self.slots.retire(slot)
        del self.meta[slot]
        self.dirty = True

    def reset_belief(self, slot: int) -> None:
        """Back to the uniform belief (done when a human leaves a goal, Sec. IV-B)."""
        m = self.meta[slot]
        J = m["G"] * m["B"]
        with self.torch.cuda.stream(self.stream):
            self.log_b[slot, :J].fill_(-float(np.log(J)))

    def set_stationary(self, slot: int, stationary: bool) -> None:
        """Mask (or restore) the speeds ``stationary_off`` for one human."""
        off = self.stationary_off if stationary else 0
        if self.meta[slot]["speed_off"] != off:
            self.meta[slot]["speed_off"] = off
            self.dirty = True

    def observe(self, slot: int, xy) -> None:
        """The newest observed state of a live human (host side, next frame)."""
        self.obs_host[slot, 0] = self.obs_host[slot, 1]
        self.obs_host[slot, 1, 0] = float(xy[0])
        self.obs_host[slot, 1, 1] = float(xy[1])
        if self.stationary_eps is not None:
            step = self.obs_host[slot, 1] - self.obs_host[slot, 0]
            self.set_stationary(slot, float(step.norm()) < self.stationary_eps)
        dep = self.meta[slot]["departure"]
        if dep is not None and dep.update(xy):
            self.reset_belief(slot)

    # -- frames ------------------------------------------------------------------
    def _humans(self):
        hs = []
        for s in sorted(self.slots.live):
            m = self.meta[s]
            hs.append(make_human(self.goals[s, :m["G"]], self.beta[s, :m["B"]], self.log_b[s],
                                 self.obs_dev[s, 1], self.N, self.T, self.grid, m["seed"], m["human_id"],
                                 self.counts[s], self.oob[s], obs_xy=self.obs_dev[s], n_obs=1, center=1,
                                 speed_off=m["speed_off"]))
        return hs

    def _enqueue(self):
        self.obs_dev.copy_(self.obs_host, non_blocking=True)
        # the zeroing (it reads the starts just copied) on a second stream,
        # beside the belief update; the rollout waits for both
        self.side.wait_stream(self.stream)
        pm_batch_zero(self.batch, self.side)
        pm_batch_update_posterior(self.batch, self.stream)
        self.stream.wait_stream(self.side)
        pm_batch_rollout(self.batch, self.stream)
        if self.union is not None:
            pm_batch_union(self.batch, self.union_sigma, self.T, self.union_grid, self.union, self.stream)

    def frame(self) -> float:
        """Run one frame for every live human; returns its latency in seconds."""
        t = self.torch
        t0 = time.perf_counter()
        if self.dirty:
            pm_batch_set(self.batch, self._humans(), self.stream)
            self.dirty = False
        if self._launch is not None and self.slots.live:
            # the captured frame, its completion event and the wait in one native call
            self._launch()
        else:
            with t.cuda.stream(self.stream):
                if self.use_graph and self.slots.live:
                    if self.graph is None:
                        self.graph = t.cuda.CUDAGraph()
                        with t.cuda.graph(self.graph, stream=self.stream):
                            self._enqueue()
                    self.graph.replay()
                elif self.slots.live:
                    self._enqueue()
                self.done.record(self.stream)
            self.done.synchronize()
            raw = getattr(self.graph, "raw_cuda_graph_exec", None)
            if self.graph is not None and raw is not None and self.done.cuda_event:
                self._launch = graph_launcher(raw(), self.stream, self.done)
        latency = time.perf_counter() - t0  # the occupancy is ready
        # the frame has applied each live human's step (prev -> cur): a later
        # frame without a new observation then applies a zero-length step,
        # which leaves the belief unchanged (the copy above has completed)
        self.obs_host[:, 0] = self.obs_host[:, 1]
        self.frames += 1
        return latency

    # -- checkpoint and resume ---------------------------------------------------
    def export_state(self, slot: int) -> dict:
        """A live human's state as plain host data (numpy arrays, Python
        scalars); waits for the server's stream so the belief is current."""
        m = self.meta[slot]
        self.stream.synchronize()
        dep = m["departure"]
        return dict(key=m["key"], goals=self.goals[slot, :m["G"]].cpu().numpy(),
                    beta=self.beta[slot, :m["B"]].cpu().numpy(),
                    log_b=self.log_b[slot, :m["G"] * m["B"]].cpu().numpy(),
                    obs=self.obs_host[slot].numpy().copy(), seed=m["seed"], human_id=m["human_id"],
                    speed_off=m["speed_off"], at_goal=None if dep is None else dep.at_goal)

    def import_state(self, state: dict) -> Optional[int]:
        """Re-admit a human from ``export_state``'s data; returns its slot, or
        None when no slot or budget is left."""
        s = self.admit(state["key"], state["goals"], state["beta"], state["obs"][1], state["seed"],
                       state["human_id"])
        if s is None:
            return None
        lb = np.asarray(state["log_b"], np.float32)
        with self.torch.cuda.stream(self.stream):
            self.log_b[s, :lb.shape[0]].copy_(self.torch.as_tensor(lb))
        self.obs_host[s].copy_(self.torch.as_tensor(np.asarray(state["obs"], np.float32)))
        self.meta[s]["speed_off"] = int(state["speed_off"])
        dep = self.meta[s]["departure"]
        if dep is not None and state.get("at_goal") is not None:
            dep.at_goal = bool(state["at_goal"])
        self.dirty = True
        return s

    def occupancy(self, slot: int):
        """(counts [T, W, W], oob [T]) of a live slot after the last frame (device)."""
        return self.counts[slot], self.oob[slot]

    def particle_steps_per_frame(self) -> int:
        return len(self.slots.live) * self.N * self.T


def run_arrivals(server: Server, arrivals, paths, frame_hz=125.0, duration_s=60.0, max_frames=None,
                 on_frame=None):
    """Drive ``server`` through an arrival process.

    ``arrivals[i]`` has t_arrive, t_leave and a ``human`` (goals, beta, seed,
    human_id); ``paths[i]`` is its observed trajectory [n, 2], one state per
    frame from its admission on. Humans that find no slot wait in arrival
    order. Returns per-frame latencies (s) and live counts.
    """
    n_frames = int(round(duration_s * frame_hz))
    if max_frames is not None:
        n_frames = min(n_frames, max_frames)
    pending = sorted(range(len(arrivals)), key=lambda i: arrivals[i].t_arrive)
    live: Dict[int, int] = {}
    first: Dict[int, int] = {}
    lat, nlive, waited = [], [], 0
    for f in range(n_frames):
        t = f / frame_hz
        for i, s in list(live.items()):
            if arrivals[i].t_leave <= t:
                server.retire(s)
                del live[i]
        while pending and arrivals[pending[0]].t_arrive <= t:
            i = pending[0]
            hu = arrivals[i].human
            s = server.admit(i, hu.goals, hu.beta, paths[i][0], hu.seed, hu.human_id)
            if s is None:
                waited += 1
                break
            live[i] = s
            first[i] = f
            pending.pop(0)
        for i, s in live.items():
            k = f - first[i]
            if k >= 1:
                server.observe(s, paths[i][min(k, len(paths[i]) - 1)])
        lat.append(server.frame())
        nlive.append(len(live))
        if on_frame is not None:
            on_frame(f, live)
    return {"latency_s": np.array(lat), "live": np.array(nlive), "frames_waited": waited}
