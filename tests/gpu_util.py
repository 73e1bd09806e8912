"""Helpers for the GPU tests: run the library through its C ABI on torch
device buffers, and the matching oracle calls on the same inputs."""
import math

import numpy as np
import torch

import paper_2603_01122_gb300 as pm

DEV = "cuda:0"


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


class GpuHuman:
    """Device-side model of a workloads.Human (or explicit parameters)."""

    def __init__(self, K, speed, dt, goals, beta, w1=1.0, w2=1.0, heading_off=0, speeds=None, speed_off=0,
                 snap_heading=False):
        self.goals = dev(np.asarray(goals, np.float32).reshape(-1, 2))
        self.beta = dev(np.asarray(beta, np.float32).reshape(-1))
        self.model = pm.make_model(K, speed, dt, self.goals, self.beta, w1=w1, w2=w2,
                                   heading_off=heading_off, speeds=speeds, speed_off=speed_off,
                                   snap_heading=snap_heading)

    @classmethod
    def of(cls, hu, **kw):
        return cls(hu.K, hu.speed, hu.dt, hu.goals, hu.beta, w1=hu.w1, w2=hu.w2, **kw)


def posterior(ctx, gh, obs, log_prior):
    obs_d = dev(np.asarray(obs, np.float32).reshape(-1, 2))
    lb = dev(np.asarray(log_prior, np.float32))
    pm.pm_update_posterior(ctx, gh.model, obs_d, obs_d.shape[0] - 1, lb)
    torch.cuda.synchronize()
    return lb.cpu().numpy()


def predict(ctx, gh, log_b, z0, N, T, grid, seed, human, n_trace=0, hist=True):
    lb = dev(np.asarray(log_b, np.float32))
    out = {}
    counts = oob = None
    g = None
    if hist:
        x0, y0, res, W, H = grid
        counts = torch.full((T, H, W), 0xDEADBEEF & 0x7FFFFFFF, dtype=torch.int32, device=DEV)
        oob = torch.full((T,), 12345, dtype=torch.int32, device=DEV)
        g = pm.make_grid(x0, y0, res, W, H)
    states = heads = comps = None
    if n_trace:
        states = torch.empty((n_trace, T, 2), dtype=torch.float32, device=DEV)
        heads = torch.empty((n_trace, T), dtype=torch.uint8, device=DEV)
        comps = torch.empty((n_trace,), dtype=torch.int32, device=DEV)
    pm.pm_predict_occupancy_traced(ctx, gh.model, lb, float(np.float32(z0[0])), float(np.float32(z0[1])),
                                   N, T, g, seed, human, counts, oob, n_trace, states, heads, comps)
    torch.cuda.synchronize()
    if hist:
        out["counts"] = counts.cpu().numpy().view(np.uint32)
        out["oob"] = oob.cpu().numpy().view(np.uint32)
    if n_trace:
        out["states32"] = states.cpu().numpy()
        out["headings"] = heads.cpu().numpy()
        out["comp"] = comps.cpu().numpy()
    return out


def explain_divergences(orc, m, lb, z0, seed, human, got, ref, decide_f32=False):
    """Check each diverged particle at its first differing draw.

    ``decide_f32``: the oracle run ``ref`` took its draws at the FP32 state
    (``orc.rollout(..., decide_f32=True)``), so the state term of the budget
    below is zero and the exact CDF is taken at that state.

    The GPU draws with the inverse CDF of its FP32 policy, evaluated at its
    FP32 state, with 22-bit fixed-point weights; the oracle with the exact
    policy at its FP64 state. With C the exact CDF, C' the GPU's, u the shared
    uniform, kg the GPU's choice and ko the oracle's: kg < ko implies
    0 <= u - C[kg] < C'[kg] - C[kg], and kg > ko implies
    0 < C[kg-1] - u <= C[kg-1] - C'[kg-1]. So u lies within max |C' - C| of a
    boundary. Each logit error is at most A = |beta| (w2 dd + |w1| ds) with dd
    = |z32 - z64| + 1e-6 (1 + d) (state and FP32 distance errors) and ds =
    1e-7 max step, so the policy's CDF moves by at most expm1(2 A); the
    fixed-point weights (largest >= 2^21 units, each within 1.5 units) and the
    threshold rounding add (1.5 U + 1) 2^-21. The component draw has only the
    last kind of error, over J components. Returns the number checked."""
    diverged = np.flatnonzero(np.any(got["headings"] != ref["headings"], axis=1) | (got["comp"] != ref["comp"]))
    J = m.G * m.B
    Cb = np.cumsum(np.exp(np.asarray(lb, np.float64)))
    Cb /= Cb[-1]
    smax = m.v * m.dt * float(np.max(m.speeds))
    for i in diverged:
        i = int(i)
        kg, ko = int(got["comp"][i]), int(ref["comp"][i])
        if kg != ko:
            u = orc.uniform_select(seed, human, i)
            delta = (u - Cb[kg]) if kg < ko else (Cb[kg - 1] - u)
            assert 0.0 <= delta <= (2 * J + 1) * 2.0 ** -21, (i, kg, ko, delta)
            continue
        g, b = divmod(ko, m.B)
        t = int(np.flatnonzero(got["headings"][i] != ref["headings"][i])[0])
        z32 = np.asarray(z0, np.float64) if t == 0 else ref["states32"][i, t - 1].astype(np.float64)
        z64 = z32 if (decide_f32 or t == 0) else ref["states64"][i, t - 1]
        C = np.cumsum(np.exp(orc.log_policy(m, z64, m.beta[b], m.goals[g])))
        C /= C[-1]
        u = orc.uniform_step(seed, human, i, t + 1)
        kg, ko = int(got["headings"][i, t]), int(ref["headings"][i, t])
        delta = (u - C[kg]) if kg < ko else (C[kg - 1] - u)
        d = math.hypot(*(z64 - m.goals[g])) + smax
        A = abs(m.beta[b]) * (m.w2 * (math.hypot(*(z32 - z64)) + 1e-6 * (1 + d)) + abs(m.w1) * 1e-7 * smax)
        budget = math.expm1(2 * A) + (1.5 * m.U + 1) * 2.0 ** -21
        assert 0.0 <= delta <= budget, (i, t, kg, ko, delta, budget)
    return len(diverged)
