"""FP64 CPU oracle for confidence-aware human prediction -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. It shares
no code with the CUDA library and never imports it.

The arithmetic lives in ``pm_oracle.c`` (plain C, doubles, single thread,
built with ``-ffp-contract=off``); this module only marshals numpy arrays.
Every function cites the passage of the paper it follows:

* :func:`log_policy`        -- Eq. 2 with the Q of the Sec. III-A running example
* :func:`update_posterior`  -- Eq. 3, in the log-space form of Eq. 7
* :func:`rollout`           -- Algorithm 1 with the bootstrapped belief (Sec. III-B)
* :func:`bin_states`        -- the "emplace onto a grid" step of Algorithm 1
* :func:`exact_occupancy`   -- Eq. 4 chained by Eq. 5 (exact, small K and T)
* :func:`loglik_grad`       -- marginal log-likelihood built on Eq. 2 / Eq. 3
* :func:`simulate`          -- observed trajectories drawn from the model (Eq. 1, Eq. 2)
* :func:`philox4x64`        -- Philox4x64-10 (Salmon et al., SC'11)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

PURPOSE_SELECT = 1
PURPOSE_STEP = 2


def build(force: bool = False) -> str:
    """Compile pm_oracle.c into oracle/_build/liboracle.so (gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_i32p = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)

_MODEL = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_int,
          C.POINTER(C.c_double), C.c_uint32, C.c_int]


def _declare(lib):
    lib.orc_philox4x64.argtypes = [_u64p, _u64p, _u64p]
    lib.orc_philox4x64.restype = None
    lib.orc_uniform_select.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64]
    lib.orc_uniform_select.restype = C.c_double
    lib.orc_uniform_step.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_int]
    lib.orc_uniform_step.restype = C.c_double
    lib.orc_log_policy.argtypes = _MODEL + [C.c_double] * 5 + [_dp]
    lib.orc_log_policy.restype = None
    lib.orc_update_posterior.argtypes = _MODEL + [C.c_int, _dp, C.c_int, _dp, _dp, C.c_int, _dp]
    lib.orc_update_posterior.restype = C.c_int
    lib.orc_sample_index.argtypes = [_dp, C.c_int, C.c_double]
    lib.orc_sample_index.restype = C.c_int
    lib.orc_draw_component.argtypes = [C.c_int, _dp, C.c_uint64, C.c_uint32, C.c_uint64]
    lib.orc_draw_component.restype = C.c_int
    lib.orc_bin.argtypes = [C.c_float] * 5 + [C.c_int, C.c_int, _i32p, _i32p]
    lib.orc_bin.restype = C.c_int
    lib.orc_inv_res.argtypes = [C.c_float]
    lib.orc_inv_res.restype = C.c_float
    lib.orc_rollout.argtypes = _MODEL + [C.c_int, _dp, C.c_int, _dp, _dp, C.c_float, C.c_float,
                                         C.c_int, C.c_uint64, C.c_uint32, C.c_int64, C.c_int64,
                                         C.c_float, C.c_float, C.c_float, C.c_int, C.c_int,
                                         _u32p, _u32p, _u8p, _fp, _dp, _i32p, C.c_int]
    lib.orc_rollout.restype = None
    lib.orc_bin_states.argtypes = [_fp, C.c_int64, C.c_int, C.c_float, C.c_float, C.c_float,
                                   C.c_int, C.c_int, _u32p, _u32p]
    lib.orc_bin_states.restype = None
    lib.orc_exact_occupancy.argtypes = _MODEL + [C.c_int, _dp, C.c_int, _dp, _dp, C.c_double,
                                                 C.c_double, C.c_int, C.c_double, C.c_double,
                                                 C.c_double, C.c_int, C.c_int, C.c_double,
                                                 _dp, _dp, _dp]
    lib.orc_exact_occupancy.restype = C.c_int
    lib.orc_loglik_grad.argtypes = _MODEL + [C.c_int, _dp, C.c_int, _dp, C.c_int, _i32p, _dp, _dp,
                                             _dp, _dp, _dp, _dp]
    lib.orc_loglik_grad.restype = C.c_int


def _ptr(a, typ):
    if a is None:
        return C.cast(None, typ)
    return a.ctypes.data_as(typ)


class Model:
    """Parameters of the human model (Sec. III-A).

    K headings theta_k = 2*pi*k/K; the controls are those headings at the
    speeds ``v * speeds[s]`` (default one speed, multiplier 1), control index
    u = s*K + k; step ``dt``;
    Q_u = -w1*v*m_s*dt - w2*||z + v*m_s*dt*e_theta - g||; ``goals`` [G, 2];
    ``beta`` [B]; ``mask_off`` bit k disables heading k and ``speed_off`` bit s
    disables speed s (Q = -inf: the stationary masking of Sec. IV-B).
    ``snap``: the observed heading is read as the nearest enabled heading
    (the discrete control) instead of the continuous one.
    Float inputs are kept exactly as given (FP32 inputs stay FP32-valued).
    """

    def __init__(self, K, v, dt, goals, beta, w1=1.0, w2=1.0, mask_off=0, speeds=(1.0,), speed_off=0,
                 snap=False):
        self.K = int(K)
        self.v = float(v)
        self.dt = float(dt)
        self.w1 = float(w1)
        self.w2 = float(w2)
        self.goals = np.ascontiguousarray(np.asarray(goals, dtype=np.float64).reshape(-1, 2))
        self.beta = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(-1))
        self.mask_off = int(mask_off)
        self.speeds = np.ascontiguousarray(np.asarray(speeds, dtype=np.float64).reshape(-1))
        self.speed_off = int(speed_off)
        self.snap = bool(snap)

    @property
    def S(self):
        return self.speeds.shape[0]

    @property
    def U(self):
        return self.S * self.K

    @property
    def G(self):
        return self.goals.shape[0]

    @property
    def B(self):
        return self.beta.shape[0]

    def _args(self):
        return [self.K, self.v, self.dt, self.w1, self.w2, C.c_uint64(self.mask_off), self.S,
                _ptr(self.speeds, _dp), C.c_uint32(self.speed_off), C.c_int(1 if self.snap else 0)]


def philox4x64(ctr, key):
    """One Philox4x64-10 block: ``ctr`` 4 x uint64, ``key`` 2 x uint64 -> 4 x uint64."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox4x64(_ptr(c, _u64p), _ptr(k, _u64p), _ptr(out, _u64p))
    return out


def uniform_select(seed, human, i):
    return _load().orc_uniform_select(seed, human, i)


def uniform_step(seed, human, i, t):
    return _load().orc_uniform_step(seed, human, i, t)


def log_policy(model: Model, z, beta, goal):
    """log pi(u | z; beta, g) for the controls u = s*K + k (Eq. 2)."""
    lib = _load()
    out = np.zeros(model.U, dtype=np.float64)
    lib.orc_log_policy(*model._args(), float(z[0]), float(z[1]), float(beta), float(goal[0]),
                       float(goal[1]), _ptr(out, _dp))
    return out


def update_posterior(model: Model, obs, log_b):
    """Sequential Eq. 7 over the observed states ``obs`` [n_obs+1, 2].

    ``log_b`` [G*B] (index g*B + b) is the prior; returns (posterior, n_skipped).
    """
    lib = _load()
    obs = np.ascontiguousarray(np.asarray(obs, dtype=np.float64).reshape(-1, 2))
    lb = np.ascontiguousarray(np.array(log_b, dtype=np.float64).reshape(-1))
    assert lb.size == model.G * model.B
    n_obs = obs.shape[0] - 1
    skipped = lib.orc_update_posterior(*model._args(), model.G, _ptr(model.goals, _dp), model.B,
                                       _ptr(model.beta, _dp), _ptr(obs, _dp), max(n_obs, 0),
                                       _ptr(lb, _dp))
    return lb, skipped


def sample_index(weights, u):
    """Inverse-CDF rule: smallest k with u*S < C_k (C_k running sum, S total)."""
    e = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    return _load().orc_sample_index(_ptr(e, _dp), e.size, float(u))


def draw_component(log_b, seed, human, i):
    lb = np.ascontiguousarray(np.asarray(log_b, dtype=np.float64).reshape(-1))
    return _load().orc_draw_component(lb.size, _ptr(lb, _dp), seed, human, i)


def inv_res(res):
    return _load().orc_inv_res(res)


def bin_point(x, y, grid):
    """Cell (cx, cy) of the FP32 point (x, y), or None if outside the grid."""
    lib = _load()
    cx = np.zeros(1, np.int32)
    cy = np.zeros(1, np.int32)
    x0, y0, res, W, H = grid
    ok = lib.orc_bin(np.float32(x), np.float32(y), np.float32(x0), np.float32(y0),
                     lib.orc_inv_res(np.float32(res)), int(W), int(H), _ptr(cx, _i32p), _ptr(cy, _i32p))
    return (int(cx[0]), int(cy[0])) if ok else None


def rollout(model: Model, log_b, z0, T, seed, human, i0, i1, grid=None, want_counts=True,
            want_headings=False, want_states32=False, want_states64=False, want_comp=False,
            decide_f32=False):
    """Algorithm 1 for particles [i0, i1) of stream (seed, human); ``headings``
    holds the drawn control index u = s*K + k.

    The particle state is carried in FP64 and, beside it, in FP32 (the same
    FP32 steps an FP32 implementation takes; the FP32 state is what is binned).
    ``decide_f32`` False evaluates the policy of each draw (Eq. 2) at the FP64
    state; True at the FP32 state, still in FP64 arithmetic: the particle
    state of Algorithm 1 held in the paper's FP32, so that a draw can differ
    from an FP32 implementation's only through that draw's own arithmetic.

    ``z0`` is taken as FP32 (the observed state handed to the GPU); ``log_b``
    is the belief b^{t'} (FP32 values from the GPU side are exact in FP64).
    ``grid`` = (x0, y0, res, W, H). Returns a dict of the requested arrays:
    counts [T, H, W] uint32, oob [T] uint32, headings [n, T] uint8,
    states32 [n, T, 2] float32, states64 [n, T, 2] float64, comp [n] int32.
    """
    lib = _load()
    lb = np.ascontiguousarray(np.asarray(log_b, dtype=np.float64).reshape(-1))
    n = int(i1) - int(i0)
    out = {}
    if grid is None:
        grid = (0.0, 0.0, 1.0, 1, 1)
        want_counts = False
    x0, y0, res, W, H = grid
    counts = np.zeros((T, H, W), np.uint32) if want_counts else None
    oob = np.zeros(T, np.uint32) if want_counts else None
    hd = np.zeros((n, T), np.uint8) if want_headings else None
    s32 = np.zeros((n, T, 2), np.float32) if want_states32 else None
    s64 = np.zeros((n, T, 2), np.float64) if want_states64 else None
    comp = np.zeros(n, np.int32) if want_comp else None
    lib.orc_rollout(*model._args(), model.G, _ptr(model.goals, _dp), model.B, _ptr(model.beta, _dp),
                    _ptr(lb, _dp), np.float32(z0[0]), np.float32(z0[1]), int(T), C.c_uint64(seed),
                    C.c_uint32(human), int(i0), int(i1), np.float32(x0), np.float32(y0),
                    np.float32(res), int(W), int(H), _ptr(counts, _u32p), _ptr(oob, _u32p),
                    _ptr(hd, _u8p), _ptr(s32, _fp), _ptr(s64, _dp), _ptr(comp, _i32p), int(bool(decide_f32)))
    if want_counts:
        out["counts"] = counts
        out["oob"] = oob
    if want_headings:
        out["headings"] = hd
    if want_states32:
        out["states32"] = s32
    if want_states64:
        out["states64"] = s64
    if want_comp:
        out["comp"] = comp
    return out


def bin_states(states32, grid):
    """Histogram [T, H, W] + oob [T] of FP32 states [n, T, 2] (emplacement step)."""
    lib = _load()
    s = np.ascontiguousarray(np.asarray(states32, dtype=np.float32))
    n, T = s.shape[0], s.shape[1]
    x0, y0, res, W, H = grid
    counts = np.zeros((T, H, W), np.uint32)
    oob = np.zeros(T, np.uint32)
    lib.orc_bin_states(_ptr(s, _fp), n, T, np.float32(x0), np.float32(y0), np.float32(res),
                       int(W), int(H), _ptr(counts, _u32p), _ptr(oob, _u32p))
    return counts, oob


def exact_occupancy(model: Model, log_b, z0, T, grid, edge_tol=1e-4):
    """Exact occupancy p(z_{t'+t} | z_{1:t'}) for t = 1..T by Eq. 4 / Eq. 5.

    Even K <= 8 only. Returns (p [T, H, W], p_oob [T], edge_mass [T]).
    """
    lib = _load()
    lb = np.ascontiguousarray(np.asarray(log_b, dtype=np.float64).reshape(-1))
    x0, y0, res, W, H = grid
    p = np.zeros((T, H, W), np.float64)
    po = np.zeros(T, np.float64)
    em = np.zeros(T, np.float64)
    rc = lib.orc_exact_occupancy(*model._args(), model.G, _ptr(model.goals, _dp), model.B,
                                 _ptr(model.beta, _dp), _ptr(lb, _dp), float(z0[0]), float(z0[1]),
                                 int(T), float(x0), float(y0), float(res), int(W), int(H),
                                 float(edge_tol), _ptr(p, _dp), _ptr(po, _dp), _ptr(em, _dp))
    if rc != 0:
        raise ValueError("exact_occupancy: unsupported K or out of memory")
    return p, po, em


def loglik_grad(model: Model, offsets, traj, log_prior):
    """Marginal log-likelihood L of trajectories and dL/d(goals, v, w1, w2).

    ``offsets`` [M+1] int32 point offsets into ``traj`` [P, 2].
    Returns (L, d_goals [G, 2], d_v, d_w [2]).
    """
    lib = _load()
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    tr = np.ascontiguousarray(np.asarray(traj, dtype=np.float64).reshape(-1, 2))
    lp = np.ascontiguousarray(np.asarray(log_prior, dtype=np.float64).reshape(-1))
    L = np.zeros(1)
    dg = np.zeros((model.G, 2))
    dv = np.zeros(1)
    dw = np.zeros(2)
    rc = lib.orc_loglik_grad(*model._args(), model.G, _ptr(model.goals, _dp), model.B,
                             _ptr(model.beta, _dp), off.size - 1, _ptr(off, _i32p), _ptr(tr, _dp),
                             _ptr(lp, _dp), _ptr(L, _dp), _ptr(dg, _dp), _ptr(dv, _dp), _ptr(dw, _dp))
    if rc != 0:
        raise ValueError("loglik_grad: unsupported sizes")
    return float(L[0]), dg, float(dv[0]), dw


def simulate(model: Model, true_j, z0, n_steps, seed, human, particle=0):
    """An observed trajectory drawn from the model (Eq. 1 discretised, Eq. 2).

    One particle of Algorithm 1 whose belief is a point mass on component
    ``true_j`` (= g*B + b). Returns FP64 states [n_steps+1, 2] (z0 first).
    """
    J = model.G * model.B
    lb = np.full(J, -np.inf)
    lb[true_j] = 0.0
    r = rollout(model, lb, z0, n_steps, seed, human, particle, particle + 1, grid=None,
                want_counts=False, want_states64=True)
    out = np.zeros((n_steps + 1, 2))
    out[0] = [np.float32(z0[0]), np.float32(z0[1])]
    out[1:] = r["states64"][0]
    return out
