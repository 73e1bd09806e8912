"""torch.autograd.Function over the library's log-likelihood adjoint.

``MarginalLogLik.apply(goals, speed, w, beta, K, dt, offsets, traj, log_prior, ctx, speeds, snap_heading)``
returns the marginal log-likelihood L of the observed trajectories (a CUDA
scalar). Its backward calls pm_loglik_backward with the incoming gradient,
so the gradient with respect to the goal coordinates, the speed and the Q
weights is computed by the adjoint kernel; this module only moves pointers
and scalars. ``speed`` and ``w`` are read to the host once per call (the
C ABI takes them as scalars). ``speeds`` (a tuple of multipliers, or None
for one speed) selects the control set of several speeds; ``snap_heading``
reads each observed heading as the nearest enabled heading.
"""
from __future__ import annotations

import torch

from . import make_model, pm_loglik_backward, pm_loglik_forward


class MarginalLogLik(torch.autograd.Function):
    @staticmethod
    def forward(fctx, goals, speed, w, beta, K, dt, offsets, traj, log_prior, ctx, speeds=None, snap_heading=False):
        v = float(speed.detach().reshape(()).item())
        w1, w2 = (float(x) for x in w.detach().reshape(2).tolist())
        goals_c = goals.detach().contiguous()
        model = make_model(K, v, dt, goals_c, beta, w1=w1, w2=w2, speeds=speeds, snap_heading=snap_heading)
        out = torch.empty((), dtype=torch.float32, device=goals.device)
        n_points = traj.shape[0]
        stream = torch.cuda.current_stream(goals.device)
        pm_loglik_forward(ctx, model, offsets.numel() - 1, offsets, n_points, traj, log_prior, out, stream)
        fctx.save_for_backward(goals_c, speed, w, beta, offsets, traj, log_prior)
        fctx.K, fctx.dt, fctx.ctx, fctx.speeds, fctx.snap = K, dt, ctx, speeds, snap_heading
        return out

    @staticmethod
    def backward(fctx, grad_out):
        goals, speed, w, beta, offsets, traj, log_prior = fctx.saved_tensors
        v = float(speed.detach().reshape(()).item())
        w1, w2 = (float(x) for x in w.detach().reshape(2).tolist())
        model = make_model(fctx.K, v, fctx.dt, goals, beta, w1=w1, w2=w2, speeds=fctx.speeds,
                           snap_heading=fctx.snap)
        dev = goals.device
        L = torch.empty((), dtype=torch.float32, device=dev)
        d_goals = torch.empty_like(goals)
        d_speed = torch.empty((), dtype=torch.float32, device=dev)
        d_w = torch.empty(2, dtype=torch.float32, device=dev)
        g = float(grad_out.detach().reshape(()).item())
        stream = torch.cuda.current_stream(dev)
        pm_loglik_backward(fctx.ctx, model, offsets.numel() - 1, offsets, traj.shape[0], traj, log_prior, g, L,
                           d_goals, d_speed, d_w, stream)
        need = fctx.needs_input_grad
        gg = d_goals if need[0] else None
        gs = d_speed.to(speed.device).reshape(speed.shape) if need[1] else None
        gw = d_w.to(w.device).reshape(w.shape) if need[2] else None
        return gg, gs, gw, None, None, None, None, None, None, None, None, None


def marginal_loglik(goals, speed, w, beta, K, dt, offsets, traj, log_prior, ctx, speeds=None, snap_heading=False):
    """Differentiable marginal log-likelihood (see MarginalLogLik)."""
    return MarginalLogLik.apply(goals, speed, w, beta, K, dt, offsets, traj, log_prior, ctx,
                                None if speeds is None else tuple(speeds), bool(snap_heading))
