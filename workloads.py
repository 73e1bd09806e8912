"""Seeded synthetic workloads: sizes, parameters and random inputs only.

This module holds none of the prediction method's arithmetic (no policy, no
belief update, no rollout, no binning). It draws the synthetic inputs that
both the CUDA path and the CPU oracle consume, from numpy's PCG64 with fixed
seeds, with the shapes of the paper's experiments (Sec. IV-A, Table 1:
n = 8192, |B| = 5, |G| = 10, |U| = 96, 50 x 50 grid; Sec. IV-B: 5 cm cells)
scaled to the five workload definitions below. Observed histories are NOT
drawn here: they come from the model itself (the oracle's ``simulate`` in
tests, the library's ``pm_simulate`` in the benchmark), starting from the
start point and true component chosen here.

Workloads
---------
``plain_small``   1 human, K = 8, 2 goals, beta in {0.1, 1, 10}, N = 10k, T = 20,
                  100 x 100 grid at 0.1 m.
``paper_scale``   1 human, 3 goals in a 10 m room, 10 log-spaced beta 0.01..100,
                  K = 36, dt = 0.02, N = 100k, T = 150, 200 x 200 grid at 0.05 m.
``batched``       16 humans, G ~ U{2..6}, N ~ U[20k, 200k], T ~ U{50..300},
                  shared 400 x 400 grid at 0.05 m, per-human histograms.
``differentiation`` 256 trajectories, lengths U{50..200}, dt = 0.05, 4 goals,
                  10 log-spaced beta 0.1..10, true beta log-uniform in [0.1, 10].
``serving``       125 Hz for 60 s, Poisson arrivals (2/s), dwell U[5, 30] s,
                  at most 64 live, N = 50k, T = 150, 121 x 121 window at 0.05 m.
``multi_speed``   ``paper_scale`` with |U| = 96 controls (Table 1): K = 32 headings
                  at speeds {0.5, 1, 1.5} x 1 m/s; the stationary variant masks
                  the two faster speeds (Sec. IV-B).
``table1``        Table 1's running example as printed: 1 human, n = 8192
                  particles, |G| = 10, |B| = 5, |U| = 96 (3 speeds x 32), a 50 x 50
                  grid, T = 10; the unprinted values (dt = 0.1 s, 0.1 m cells, the
                  beta values, 20 observed steps) are chosen here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

MASTER_SEED = 20260301


def f32(x: float) -> float:
    """The FP32 value nearest to x, as a Python float (what the GPU sees)."""
    return float(np.float32(x))


def beta_grid(lo_exp: float, hi_exp: float, n: int) -> np.ndarray:
    """n log-spaced values 10^lo .. 10^hi (float32-valued)."""
    return np.float32(10.0) ** np.linspace(lo_exp, hi_exp, n, dtype=np.float32)


@dataclasses.dataclass
class Human:
    """One human's prediction problem (all floats FP32-valued)."""
    K: int
    speed: float
    dt: float
    goals: np.ndarray          # [G, 2] float32
    beta: np.ndarray           # [B] float32
    true_j: int                # component g*B + b that generates the history
    start: np.ndarray          # [2] float32, first observed state
    n_obs: int                 # observed steps (n_obs + 1 states)
    n_particles: int
    horizon: int
    grid: tuple                # (x0, y0, res, W, H)
    seed: int                  # Philox key word 0 for the rollout
    human_id: int              # Philox key word 1
    obs_seed: int              # Philox key word 0 for the observed history
    w1: float = 1.0
    w2: float = 1.0
    window: int = 0            # serving: side of the output window (0 = full grid)
    speeds: tuple = (1.0,)     # speed multipliers of the control set
    speed_off: int = 0         # bit s: speed s disabled (stationary masking)

    @property
    def G(self):
        return int(self.goals.shape[0])

    @property
    def B(self):
        return int(self.beta.shape[0])

    def uniform_log_prior(self) -> np.ndarray:
        """log(1/(|B||G|)) for every component (Sec. III-B initial belief), FP32."""
        return np.full(self.G * self.B, -math.log(self.G * self.B), dtype=np.float32)


def plain_small(seed: int = MASTER_SEED) -> Human:
    """1 human: K = 8, v = 1, dt = 0.1, goals (4,0),(0,4), beta {0.1,1,10}, 20 observed
    steps from (0,0) with true (beta = 1, goal 0), N = 10k, T = 20, 100 x 100 grid at
    0.1 m with origin (-5.05, -5.05) so that (0,0) is a cell centre."""
    return Human(K=8, speed=1.0, dt=f32(0.1),
                 goals=np.array([[4.0, 0.0], [0.0, 4.0]], np.float32),
                 beta=np.array([0.1, 1.0, 10.0], np.float32),
                 true_j=0 * 3 + 1, start=np.array([0.0, 0.0], np.float32), n_obs=20,
                 n_particles=10_000, horizon=20, grid=(f32(-5.05), f32(-5.05), f32(0.1), 100, 100),
                 seed=seed, human_id=0, obs_seed=seed + 1)


def plain_crowd(n: int = 64, seed: int = MASTER_SEED) -> list:
    """n humans of the plain configuration's shape (K = 8, v = 1, dt = 0.1, the same
    goals and beta grid, N = 10k, T = 20, 100 x 100 grid at 0.1 m), each with its own
    start uniform in [-3, 3]^2, true component, seed and human id: many small
    humans, where one call per human is bound by launch latency."""
    rng = np.random.default_rng([seed, 8])
    base = plain_small(seed)
    out = []
    for i in range(n):
        out.append(dataclasses.replace(base, start=rng.uniform(-3.0, 3.0, size=2).astype(np.float32),
                                       true_j=int(rng.integers(0, 6)), seed=seed + 1000 + i, human_id=1000 + i,
                                       obs_seed=seed + 2000 + i))
    return out


def paper_scale(seed: int = MASTER_SEED) -> Human:
    """1 human in a 10 m room: 3 goals uniform, 10 log-spaced beta 0.01..100, K = 36,
    dt = 0.02, N = 100k, T = 150, 200 x 200 grid at 0.05 m; 50 observed steps from a
    start uniform in [2, 8]^2 with true (beta_5 ~ 1.668, goal 0)."""
    rng = np.random.default_rng([seed, 1])
    goals = rng.uniform(0.0, 10.0, size=(3, 2)).astype(np.float32)
    start = rng.uniform(2.0, 8.0, size=2).astype(np.float32)
    beta = beta_grid(-2.0, 2.0, 10)
    return Human(K=36, speed=1.0, dt=f32(0.02), goals=goals, beta=beta, true_j=0 * 10 + 5,
                 start=start, n_obs=50, n_particles=100_000, horizon=150,
                 grid=(0.0, 0.0, f32(0.05), 200, 200), seed=seed, human_id=1, obs_seed=seed + 11)


def multi_speed(seed: int = MASTER_SEED, stationary: bool = False) -> Human:
    """``paper_scale`` with 3 speeds x K = 32 headings (|U| = 96); ``stationary``
    disables the speeds 1 and 1.5 m/s, leaving the slow walk."""
    hu = paper_scale(seed)
    return dataclasses.replace(hu, K=32, speeds=(0.5, 1.0, 1.5), speed_off=0b110 if stationary else 0,
                               human_id=3, obs_seed=seed + 31)


def table1(seed: int = MASTER_SEED, horizon: int = 10) -> Human:
    """Table 1's configuration: 10 goals uniform in a 5 m room, 5 log-spaced beta
    0.1..10, |U| = 96 = 3 speeds {0.5, 1, 1.5} x K = 32 at v = 1 m/s, dt = 0.1,
    n = 8192, T = ``horizon``, 50 x 50 grid at 0.1 m; 20 observed steps from a
    start uniform in [1.5, 3.5]^2 with true (beta_2, goal 0)."""
    rng = np.random.default_rng([seed, 6])
    goals = rng.uniform(0.0, 5.0, size=(10, 2)).astype(np.float32)
    start = rng.uniform(1.5, 3.5, size=2).astype(np.float32)
    return Human(K=32, speed=1.0, dt=f32(0.1), goals=goals, beta=beta_grid(-1.0, 1.0, 5), true_j=0 * 5 + 2,
                 start=start, n_obs=20, n_particles=8192, horizon=horizon,
                 grid=(0.0, 0.0, f32(0.1), 50, 50), seed=seed, human_id=4, obs_seed=seed + 41,
                 speeds=(0.5, 1.0, 1.5))


def batched(seed: int = MASTER_SEED, n_humans: int = 16) -> List[Human]:
    """16 humans in a 20 m room sharing a 400 x 400 grid at 0.05 m (per-human
    histograms): G ~ U{2..6}, N ~ U[20000, 200000], T ~ U{50..300}, K = 36,
    dt = 0.02, beta as ``paper_scale``, 50 observed steps from U[2, 18]^2."""
    rng = np.random.default_rng([seed, 2])
    beta = beta_grid(-2.0, 2.0, 10)
    out = []
    for h in range(n_humans):
        G = int(rng.integers(2, 7))
        goals = rng.uniform(0.0, 20.0, size=(G, 2)).astype(np.float32)
        N = int(rng.integers(20_000, 200_001))
        T = int(rng.integers(50, 301))
        start = rng.uniform(2.0, 18.0, size=2).astype(np.float32)
        true_j = int(rng.integers(0, G)) * 10 + int(rng.integers(0, 10))
        out.append(Human(K=36, speed=1.0, dt=f32(0.02), goals=goals, beta=beta, true_j=true_j,
                         start=start, n_obs=50, n_particles=N, horizon=T,
                         grid=(0.0, 0.0, f32(0.05), 400, 400), seed=seed, human_id=100 + h,
                         obs_seed=seed + 21))
    return out


@dataclasses.dataclass
class TrajectorySet:
    """Observed trajectories for the differentiation workload."""
    K: int
    speed: float
    dt: float
    goals: np.ndarray        # [4, 2] float32
    beta: np.ndarray         # [10] float32 (the inference grid)
    lengths: np.ndarray      # [M] int, steps per trajectory
    true_beta: np.ndarray    # [M] float32 (continuous, log-uniform)
    true_goal: np.ndarray    # [M] int
    starts: np.ndarray       # [M, 2] float32
    obs_seed: int
    w1: float = 1.0
    w2: float = 1.0

    @property
    def M(self):
        return int(self.lengths.shape[0])


def differentiation(seed: int = MASTER_SEED, M: int = 256) -> TrajectorySet:
    """256 trajectories, lengths U{50..200} at dt = 0.05, 4 goals uniform in [0, 10]^2,
    true beta log-uniform in [0.1, 10], true goal U{0..3}, starts uniform in the room;
    inference over 10 log-spaced beta 0.1..10 with w = (1, 1)."""
    rng = np.random.default_rng([seed, 3])
    goals = rng.uniform(0.0, 10.0, size=(4, 2)).astype(np.float32)
    lengths = rng.integers(50, 201, size=M)
    true_beta = (10.0 ** rng.uniform(-1.0, 1.0, size=M)).astype(np.float32)
    true_goal = rng.integers(0, 4, size=M)
    starts = rng.uniform(0.0, 10.0, size=(M, 2)).astype(np.float32)
    return TrajectorySet(K=36, speed=1.0, dt=f32(0.05), goals=goals, beta=beta_grid(-1.0, 1.0, 10),
                         lengths=lengths, true_beta=true_beta, true_goal=true_goal,
                         starts=starts, obs_seed=seed + 31)


@dataclasses.dataclass
class Arrival:
    t_arrive: float
    t_leave: float
    human: Human


def serving(seed: int = MASTER_SEED, duration_s: float = 60.0, rate_hz: float = 2.0,
            frame_hz: float = 125.0, max_live: int = 64) -> dict:
    """Arrival process of the serving workload: Poisson(rate) arrivals over
    ``duration_s``, dwell U[5, 30] s, each human ``batched``-like with N = 50k,
    T = 150, K = 36, dt = 0.02 and a 121 x 121 output window at 0.05 m centred on
    the cell of its latest observed state."""
    rng = np.random.default_rng([seed, 4])
    beta = beta_grid(-2.0, 2.0, 10)
    arrivals = []
    t = 0.0
    h = 0
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        dwell = float(rng.uniform(5.0, 30.0))
        G = int(rng.integers(2, 7))
        goals = rng.uniform(0.0, 20.0, size=(G, 2)).astype(np.float32)
        start = rng.uniform(4.0, 16.0, size=2).astype(np.float32)
        true_j = int(rng.integers(0, G)) * 10 + int(rng.integers(0, 10))
        hu = Human(K=36, speed=1.0, dt=f32(0.02), goals=goals, beta=beta, true_j=true_j, start=start,
                   n_obs=0, n_particles=50_000, horizon=150, grid=(0.0, 0.0, f32(0.05), 400, 400),
                   seed=seed, human_id=1000 + h, obs_seed=seed + 41, window=121)
        arrivals.append(Arrival(t, t + dwell, hu))
        h += 1
    return {"frame_hz": frame_hz, "duration_s": duration_s, "max_live": max_live,
            "arrivals": arrivals}
