"""Thin Python binding of libpm (include/pm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
plain pointers and sizes; every numeric step runs in the library's CUDA
kernels. Device buffers may be given as torch CUDA tensors (their data_ptr is
passed) or as integers. There is no CPU fallback: if libpm.so has not been
built, the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB as _LIB_PATH
from ._build import build  # noqa: F401  (re-exported for __graft_entry__)

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_EDEVICE = 0, 1, 2, 3, 5
PM_MAX_HEADINGS, PM_MAX_COMPONENTS, PM_MAX_GOALS, PM_MAX_HORIZON = 64, 256, 64, 4096
PURPOSE_SELECT, PURPOSE_STEP = 1, 2
_STATUS = {0: "PM_OK", 1: "PM_EINVAL", 2: "PM_ENOMEM", 3: "PM_ECUDA", 5: "PM_EDEVICE"}


class PmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class pm_model(C.Structure):
    _fields_ = [("K", C.c_int32), ("speed", C.c_float), ("dt", C.c_float), ("w1", C.c_float),
                ("w2", C.c_float), ("G", C.c_int32), ("B", C.c_int32), ("goals", C.c_void_p),
                ("beta", C.c_void_p), ("heading_off", C.c_uint64), ("n_speeds", C.c_int32),
                ("speed_mult", C.c_float * 4), ("speed_off", C.c_uint32), ("snap_heading", C.c_int32)]


class pm_mppi(C.Structure):
    _fields_ = [("n_samples", C.c_int32), ("horizon", C.c_int32), ("dt", C.c_float), ("pred_stride", C.c_int32),
                ("q", C.c_float * 4), ("q_final", C.c_float * 4), ("r", C.c_float * 2), ("goal", C.c_float * 4),
                ("coll_threshold", C.c_float), ("coll_cost", C.c_float), ("step_cost", C.c_float),
                ("temperature", C.c_float)]


def make_mppi(n_samples, horizon, dt, pred_stride, q, q_final, r, goal, coll_threshold=0.1, coll_cost=1000.0,
              step_cost=0.0, temperature=1.0) -> pm_mppi:
    return pm_mppi(int(n_samples), int(horizon), float(dt), int(pred_stride), (C.c_float * 4)(*q),
                   (C.c_float * 4)(*q_final), (C.c_float * 2)(*r), (C.c_float * 4)(*goal), float(coll_threshold),
                   float(coll_cost), float(step_cost), float(temperature))


class pm_grid(C.Structure):
    _fields_ = [("x0", C.c_float), ("y0", C.c_float), ("res", C.c_float), ("W", C.c_int32),
                ("H", C.c_int32)]


class pm_human(C.Structure):
    _fields_ = [("goals", C.c_void_p), ("beta", C.c_void_p), ("G", C.c_int32), ("B", C.c_int32),
                ("obs_xy", C.c_void_p), ("n_obs", C.c_int32), ("log_belief", C.c_void_p),
                ("z0_xy", C.c_void_p), ("n_particles", C.c_int32), ("horizon", C.c_int32),
                ("grid", pm_grid), ("center", C.c_int32), ("cx_off", C.c_int32), ("cy_off", C.c_int32),
                ("seed", C.c_uint64), ("human_id", C.c_uint32), ("counts", C.c_void_p), ("oob", C.c_void_p),
                ("speed_off", C.c_uint32)]


_lib = None
_vp = C.c_void_p


def _signatures(lib):
    P = C.POINTER
    sig = {
        "pm_create": ([P(_vp), C.c_int], C.c_int),
        "pm_destroy": ([_vp], None),
        "pm_last_error": ([], C.c_char_p),
        "pm_version": ([], C.c_char_p),
        "pm_sync_status": ([_vp, _vp], C.c_int),
        "pm_graph_launch": ([_vp, _vp, _vp, C.c_int32], C.c_int),
        "pm_batch_set_block_flags": ([_vp, C.c_int32, _vp], C.c_int),
        "pm_batch_set_zeroing": ([_vp, C.c_int32, _vp], C.c_int),
        "pm_batch_zero": ([_vp, _vp], C.c_int),
        "pm_batch_rollout": ([_vp, _vp], C.c_int),
        "pm_update_posterior": ([_vp, P(pm_model), _vp, C.c_int32, _vp, _vp], C.c_int),
        "pm_update_posterior_into": ([_vp, P(pm_model), _vp, C.c_int32, _vp, _vp, _vp], C.c_int),
        "pm_predict_occupancy": ([_vp, P(pm_model), _vp, C.c_float, C.c_float, C.c_int32, C.c_int32,
                                  P(pm_grid), C.c_uint64, C.c_uint32, _vp, _vp, _vp], C.c_int),
        "pm_rollout_occupancy": ([_vp, P(pm_model), _vp, C.c_float, C.c_float, C.c_int32, C.c_int32,
                                  P(pm_grid), C.c_uint64, C.c_uint32, _vp, _vp, _vp], C.c_int),
        "pm_zero_occupancy": ([_vp, C.c_int32, P(pm_grid), _vp, _vp, _vp], C.c_int),
        "pm_predict_occupancy_traced": ([_vp, P(pm_model), _vp, C.c_float, C.c_float, C.c_int32,
                                         C.c_int32, P(pm_grid), C.c_uint64, C.c_uint32, _vp, _vp,
                                         C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
        "pm_predict_host": ([_vp, P(pm_model), _vp, _vp, _vp, C.c_int32, _vp, C.c_int32, C.c_int32,
                             P(pm_grid), C.c_uint64, C.c_uint32, _vp, _vp, _vp, _vp], C.c_int),
        "pm_predict_host_async": ([_vp, P(pm_model), _vp, _vp, _vp, C.c_int32, _vp, C.c_int32, C.c_int32,
                                   P(pm_grid), C.c_uint64, C.c_uint32, _vp, _vp, _vp, _vp], C.c_int),
        "pm_host_fence": ([_vp, _vp], C.c_int),
        "pm_batch_create": ([_vp, P(pm_model), C.c_int32, P(_vp)], C.c_int),
        "pm_batch_set": ([_vp, P(pm_human), C.c_int32, _vp], C.c_int),
        "pm_batch_update_posterior": ([_vp, _vp], C.c_int),
        "pm_batch_predict": ([_vp, _vp], C.c_int),
        "pm_batch_autotune": ([_vp, _vp], C.c_int),
        "pm_batch_get_config": ([_vp] + [P(C.c_int32)] * 4, C.c_int),
        "pm_batch_set_config": ([_vp] + [C.c_int32] * 4, C.c_int),
        "pm_batch_destroy": ([_vp], None),
        "pm_smooth_occupancy": ([_vp, _vp, C.c_int32, C.c_int32, P(pm_grid), C.c_float, _vp, _vp], C.c_int),
        "pm_batch_union": ([_vp, C.c_float, C.c_int32, P(pm_grid), _vp, _vp], C.c_int),
        "pm_mppi_solve": ([_vp, P(pm_mppi), P(C.c_float), _vp, _vp, _vp, C.c_int32, P(pm_grid), _vp, _vp, _vp],
                          C.c_int),
        "pm_loglik_forward": ([_vp, P(pm_model), C.c_int32, _vp, C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
        "pm_loglik_backward": ([_vp, P(pm_model), C.c_int32, _vp, C.c_int32, _vp, _vp, C.c_float, _vp, _vp,
                                _vp, _vp, _vp], C.c_int),
        "pm_update_posterior_noalloc": ([P(pm_model), _vp, C.c_int32, _vp, _vp], C.c_int),
        "pm_philox_blocks": ([_vp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64,
                              C.c_int32, _vp, _vp], C.c_int),
        "pm_probe_sfu": ([_vp, C.c_int, P(C.c_double)], C.c_int),
        "pm_device_info": ([_vp, P(C.c_int), P(C.c_int), P(C.c_int)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = res
    return sig


def library():
    """The loaded libpm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libpm.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        lib = C.CDLL(_LIB_PATH)
        _signatures(lib)
        _lib = lib
    return _lib


def _p(x):
    """Device pointer of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _hp(x):
    """Host pointer of a numpy array or a pinned CPU torch tensor."""
    if x is None:
        return None
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st):
    if st != PM_OK:
        raise PmError(st, library().pm_last_error().decode())


def pm_version() -> str:
    return library().pm_version().decode()


def pm_last_error() -> str:
    return library().pm_last_error().decode()


def pm_sync_status(ctx, stream=None):
    """Wait for ``stream`` and raise PmError(PM_EDEVICE) if kernels of ``ctx``
    latched unusable inputs since the last call (the word is then cleared)."""
    _check(library().pm_sync_status(ctx, _stream(stream)))


def graph_launcher(graph_exec, stream=None, done=None, wait=True):
    """A zero-argument callable that runs pm_graph_launch with these arguments
    bound once (a frame loop then spends no time converting them per frame)."""
    fn = library().pm_graph_launch
    args = (C.c_void_p(int(graph_exec)), _stream(stream), None if done is None else C.c_void_p(done.cuda_event),
            1 if wait else 0)

    def launch():
        st = fn(*args)
        if st != PM_OK:
            _check(st)
    return launch


def pm_graph_launch(graph_exec, stream=None, done=None, wait=False):
    """Launch an instantiated CUDA graph (its cudaGraphExec_t as an integer,
    e.g. ``torch.cuda.CUDAGraph.raw_cuda_graph_exec()``) on ``stream``, record
    ``done`` (a torch.cuda.Event) after it and, with ``wait``, wait for it:
    one native call."""
    ev = None
    if done is not None:
        ev = C.c_void_p(done.cuda_event)
    _check(library().pm_graph_launch(C.c_void_p(int(graph_exec)), _stream(stream), ev, 1 if wait else 0))


def pm_create(device: int = 0) -> int:
    h = _vp()
    _check(library().pm_create(C.byref(h), int(device)))
    return h.value


def pm_destroy(ctx) -> None:
    library().pm_destroy(ctx)


def make_model(K, speed, dt, goals, beta, w1=1.0, w2=1.0, heading_off=0, speeds=None, speed_off=0,
               snap_heading=False) -> pm_model:
    """pm_model over device tensors ``goals`` [G, 2] and ``beta`` [B] (float32);
    ``speeds``: speed multipliers of the control set (None: one speed);
    ``snap_heading``: read observed headings as the nearest enabled heading."""
    G = int(goals.shape[0])
    B = int(beta.shape[0])
    mult = list(speeds) if speeds is not None else []
    m = pm_model(int(K), float(speed), float(dt), float(w1), float(w2), G, B, _p(goals), _p(beta),
                 int(heading_off), len(mult), (C.c_float * 4)(*(mult + [0.0] * (4 - len(mult)))), int(speed_off),
                 1 if snap_heading else 0)
    m._keep = (goals, beta)  # keep the tensors alive with the struct
    return m


def make_grid(x0, y0, res, W, H) -> pm_grid:
    return pm_grid(float(x0), float(y0), float(res), int(W), int(H))


def pm_update_posterior(ctx, model: pm_model, obs_xy, n_obs, log_belief, stream=None):
    _check(library().pm_update_posterior(ctx, C.byref(model), _p(obs_xy), int(n_obs), _p(log_belief),
                                         _stream(stream)))


def pm_update_posterior_into(ctx, model: pm_model, obs_xy, n_obs, log_prior, log_belief, stream=None):
    _check(library().pm_update_posterior_into(ctx, C.byref(model), _p(obs_xy), int(n_obs), _p(log_prior),
                                              _p(log_belief), _stream(stream)))


def pm_predict_occupancy(ctx, model: pm_model, log_belief, z0x, z0y, n_particles, horizon,
                         grid: pm_grid, seed, human_id, counts, oob, stream=None):
    _check(library().pm_predict_occupancy(ctx, C.byref(model), _p(log_belief), float(z0x), float(z0y),
                                          int(n_particles), int(horizon), C.byref(grid), int(seed),
                                          int(human_id), _p(counts), _p(oob), _stream(stream)))


def pm_zero_occupancy(ctx, horizon, grid: pm_grid, counts, oob, stream=None):
    _check(library().pm_zero_occupancy(ctx, int(horizon), C.byref(grid), _p(counts), _p(oob), _stream(stream)))


def pm_rollout_occupancy(ctx, model: pm_model, log_belief, z0x, z0y, n_particles, horizon,
                         grid: pm_grid, seed, human_id, counts, oob, stream=None):
    _check(library().pm_rollout_occupancy(ctx, C.byref(model), _p(log_belief), float(z0x), float(z0y),
                                          int(n_particles), int(horizon), C.byref(grid), int(seed),
                                          int(human_id), _p(counts), _p(oob), _stream(stream)))


def pm_predict_occupancy_traced(ctx, model: pm_model, log_belief, z0x, z0y, n_particles, horizon,
                                grid, seed, human_id, counts, oob, n_trace, states=None,
                                headings=None, components=None, stream=None):
    g = C.byref(grid) if grid is not None else None
    _check(library().pm_predict_occupancy_traced(
        ctx, C.byref(model), _p(log_belief), float(z0x), float(z0y), int(n_particles), int(horizon), g,
        int(seed), int(human_id), _p(counts), _p(oob), int(n_trace), _p(states), _p(headings),
        _p(components), _stream(stream)))


def pm_predict_host(ctx, model: pm_model, goals, beta, obs_xy, n_obs, log_prior, n_particles,
                    horizon, grid: pm_grid, seed, human_id, posterior_out, counts_out, oob_out,
                    stream=None):
    """Host-buffer form: numpy arrays or (pinned) CPU tensors in and out."""
    _check(library().pm_predict_host(ctx, C.byref(model), _hp(goals), _hp(beta), _hp(obs_xy), int(n_obs),
                                     _hp(log_prior), int(n_particles), int(horizon), C.byref(grid),
                                     int(seed), int(human_id), _hp(posterior_out), _hp(counts_out),
                                     _hp(oob_out), _stream(stream)))


def pm_predict_host_async(ctx, model: pm_model, goals, beta, obs_xy, n_obs, log_prior, n_particles,
                          horizon, grid: pm_grid, seed, human_id, posterior_out, counts_out, oob_out,
                          stream=None):
    """pm_predict_host without waiting (pinned CPU tensors; the outputs are
    complete after pm_host_fence and a synchronisation of the stream)."""
    _check(library().pm_predict_host_async(ctx, C.byref(model), _hp(goals), _hp(beta), _hp(obs_xy), int(n_obs),
                                           _hp(log_prior), int(n_particles), int(horizon), C.byref(grid),
                                           int(seed), int(human_id), _hp(posterior_out), _hp(counts_out),
                                           _hp(oob_out), _stream(stream)))


def pm_host_fence(ctx, stream=None):
    _check(library().pm_host_fence(ctx, _stream(stream)))


def make_human(goals, beta, log_belief, z0_xy, n_particles, horizon, grid: pm_grid, seed, human_id,
               counts, oob, obs_xy=None, n_obs=0, center=0, cx_off=0, cy_off=0, speed_off=0) -> pm_human:
    """pm_human over device tensors (the tensors are kept alive with the struct);
    ``speed_off`` disables speeds for this human (several-speed models only)."""
    h = pm_human(_p(goals), _p(beta), int(goals.shape[0]), int(beta.shape[0]), _p(obs_xy), int(n_obs),
                 _p(log_belief), _p(z0_xy), int(n_particles), int(horizon), grid, int(center), int(cx_off),
                 int(cy_off), int(seed), int(human_id), _p(counts), _p(oob), int(speed_off))
    h._keep = (goals, beta, log_belief, z0_xy, counts, oob, obs_xy)
    return h


def pm_batch_create(ctx, shared: pm_model, max_humans) -> int:
    h = _vp()
    _check(library().pm_batch_create(ctx, C.byref(shared), int(max_humans), C.byref(h)))
    return h.value


def pm_batch_set(batch, humans, stream=None):
    arr = (pm_human * max(1, len(humans)))(*humans)
    _check(library().pm_batch_set(batch, arr, len(humans), _stream(stream)))


def pm_batch_update_posterior(batch, stream=None):
    _check(library().pm_batch_update_posterior(batch, _stream(stream)))


def pm_batch_predict(batch, stream=None):
    _check(library().pm_batch_predict(batch, _stream(stream)))


def pm_smooth_occupancy(ctx, counts, n_particles, horizon, grid, sigma_cells, prob, stream=None):
    _check(library().pm_smooth_occupancy(ctx, _p(counts), int(n_particles), int(horizon), C.byref(grid),
                                         float(sigma_cells), _p(prob), _stream(stream)))


def pm_batch_union(batch, sigma_cells, horizon, grid, prob, stream=None):
    _check(library().pm_batch_union(batch, float(sigma_cells), int(horizon), C.byref(grid), _p(prob),
                                    _stream(stream)))


def pm_mppi_solve(ctx, params: pm_mppi, z0, u_ref, delta, prob, prob_T, grid, cost_to_go, u_opt, stream=None):
    z = (C.c_float * 4)(*[float(v) for v in z0])
    _check(library().pm_mppi_solve(ctx, C.byref(params), z, _p(u_ref), _p(delta), _p(prob), int(prob_T),
                                   C.byref(grid) if grid is not None else None, _p(cost_to_go), _p(u_opt),
                                   _stream(stream)))


def pm_batch_set_block_flags(batch, enable, stream=None):
    _check(library().pm_batch_set_block_flags(batch, int(enable), _stream(stream)))


def pm_batch_set_zeroing(batch, reach, stream=None):
    _check(library().pm_batch_set_zeroing(batch, int(reach), _stream(stream)))


def pm_batch_zero(batch, stream=None):
    _check(library().pm_batch_zero(batch, _stream(stream)))


def pm_batch_rollout(batch, stream=None):
    _check(library().pm_batch_rollout(batch, _stream(stream)))


def pm_batch_autotune(batch, stream=None):
    _check(library().pm_batch_autotune(batch, _stream(stream)))


def pm_batch_get_config(batch):
    t, sw, c, w = (C.c_int32() for _ in range(4))
    _check(library().pm_batch_get_config(batch, C.byref(t), C.byref(sw), C.byref(c), C.byref(w)))
    return {"threads": t.value, "shared_window": sw.value, "ctas_per_sm": c.value, "window_kib": w.value}


def pm_batch_set_config(batch, threads, shared_window, ctas_per_sm, window_kib):
    _check(library().pm_batch_set_config(batch, int(threads), int(shared_window), int(ctas_per_sm),
                                         int(window_kib)))


def pm_batch_destroy(batch):
    library().pm_batch_destroy(batch)


def pm_loglik_forward(ctx, model: pm_model, M, offsets, n_points, traj_xy, log_prior, loglik, stream=None):
    _check(library().pm_loglik_forward(ctx, C.byref(model), int(M), _p(offsets), int(n_points), _p(traj_xy),
                                       _p(log_prior), _p(loglik), _stream(stream)))


def pm_loglik_backward(ctx, model: pm_model, M, offsets, n_points, traj_xy, log_prior, grad_out, loglik,
                       d_goals, d_speed, d_w, stream=None):
    _check(library().pm_loglik_backward(ctx, C.byref(model), int(M), _p(offsets), int(n_points), _p(traj_xy),
                                        _p(log_prior), float(grad_out), _p(loglik), _p(d_goals), _p(d_speed),
                                        _p(d_w), _stream(stream)))


def pm_update_posterior_noalloc(model: pm_model, obs_xy, n_obs, log_belief, stream=None):
    """Belief update that allocates nothing (no context; static device scratch)."""
    _check(library().pm_update_posterior_noalloc(C.byref(model), _p(obs_xy), int(n_obs), _p(log_belief),
                                                 _stream(stream)))


def pm_philox_blocks(ctx, seed, human_id, purpose, particle0, block, n, out, stream=None):
    _check(library().pm_philox_blocks(ctx, int(seed), int(human_id), int(purpose), int(particle0),
                                      int(block), int(n), _p(out), _stream(stream)))


def pm_probe_sfu(ctx, op: int) -> float:
    v = C.c_double()
    _check(library().pm_probe_sfu(ctx, int(op), C.byref(v)))
    return v.value


def pm_device_info(ctx):
    sm, clk, cc = C.c_int(), C.c_int(), C.c_int()
    _check(library().pm_device_info(ctx, C.byref(sm), C.byref(clk), C.byref(cc)))
    return {"sm_count": sm.value, "clock_khz": clk.value, "cc": cc.value}
