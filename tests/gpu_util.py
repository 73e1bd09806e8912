"""Helpers for the GPU tests: run the library through its C ABI on torch
device buffers, and the matching oracle calls on the same inputs."""
import numpy as np
import torch

import paper_2603_01122_gb300 as pm

DEV = "cuda:0"


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


class GpuHuman:
    """Device-side model of a workloads.Human (or explicit parameters)."""

    def __init__(self, K, speed, dt, goals, beta, w1=1.0, w2=1.0, heading_off=0, speeds=None, speed_off=0):
        self.goals = dev(np.asarray(goals, np.float32).reshape(-1, 2))
        self.beta = dev(np.asarray(beta, np.float32).reshape(-1))
        self.model = pm.make_model(K, speed, dt, self.goals, self.beta, w1=w1, w2=w2,
                                   heading_off=heading_off, speeds=speeds, speed_off=speed_off)

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
