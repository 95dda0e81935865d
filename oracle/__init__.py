"""ctypes front end of the FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg import this package.  The product path never does, and it shares
no code with the CUDA library (this module takes host numpy arrays, up-casts
them to float64 and calls liboracle.so).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")

_dp = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)
_i32p = C.POINTER(C.c_int32)


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ -O2 (no fast-math) and OpenMP."""
    stale = not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    if force or stale:
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", _SO, _SRC])
    return _SO


class ObParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("idm_amax", C.c_double), ("idm_b", C.c_double),
                ("idm_T", C.c_double), ("idm_s0", C.c_double), ("idm_dq", C.c_double),
                ("route_h", C.c_double), ("gap_min", C.c_double), ("band", C.c_double),
                ("idm_K", C.c_int32), ("pad_", C.c_int32),
                ("kin_amax", C.c_double), ("kin_kmax", C.c_double), ("kin_band_a", C.c_double),
                ("kin_band_th", C.c_double), ("route_max_dist", C.c_double), ("route_max_rel", C.c_double),
                ("disc_a_max", C.c_double), ("disc_k_max", C.c_double), ("disc_d_max", C.c_double),
                ("disc_t_max", C.c_double), ("disc_na", C.c_int32), ("disc_nk", C.c_int32), ("disc_nd", C.c_int32),
                ("disc_nt", C.c_int32)]


class ObBatch(C.Structure):
    _fields_ = [("S", C.c_int32), ("N_tot", C.c_int32), ("T_log", C.c_int32), ("pad_", C.c_int32),
                ("agent_off", _i32p), ("rg_off", _i32p),
                ("L", _dp), ("W", _dp), ("idm_v0", _dp),
                ("valid", _u8p), ("kind", _u8p),
                ("route_off", _i32p), ("route_x", _dp), ("route_y", _dp),
                ("rg_x", _dp), ("rg_y", _dp), ("rg_poly", _i32p), ("rg_type", _u8p), ("rg_valid", _u8p),
                ("log_x", _dp), ("log_y", _dp), ("log_th", _dp), ("log_vx", _dp), ("log_vy", _dp),
                ("path_off", _i32p), ("path_pt_off", _i32p), ("path_x", _dp), ("path_y", _dp), ("path_on", _u8p)]


class ObState(C.Structure):
    _fields_ = [(k, _dp) for k in ("x", "y", "th", "vx", "vy", "s")]


class ObMetrics(C.Structure):
    _fields_ = [("ov", _dp), ("off", _dp), ("logdiv", _dp), ("flags", _u8p), ("reward", _i32p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        _lib.oracle_transition.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, P(ObState), _dp,
                                           _u8p, C.c_int, P(ObState), _u8p, _i32p]
        _lib.oracle_metrics.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, P(ObState), P(ObState),
                                        C.c_int, P(ObMetrics)]
        _lib.oracle_rollout.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, P(ObState), _dp, _u8p,
                                        C.c_int, C.c_int, P(ObMetrics), C.c_int]
        _lib.oracle_inverse.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, P(ObState), P(ObState), _dp]
        _lib.oracle_discretize.argtypes = [P(ObParams), P(ObBatch), _dp, C.c_int, _i32p, _u8p]
        _lib.oracle_decode_actions.argtypes = [P(ObParams), P(ObBatch), _i32p, C.c_int, _dp]
        _lib.oracle_route.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, P(ObState), _dp, _u8p]
        _lib.oracle_observe.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, P(ObState), _u8p, C.c_int,
                                        C.c_int, _dp, _u8p, _dp, _i32p]
        _lib.oracle_expert_actions.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_int, C.c_int, C.c_int,
                                               _dp]
        _lib.oracle_box_depth.argtypes = [_dp, _dp]
        _lib.oracle_box_depth.restype = C.c_double
        _lib.oracle_point_sd.argtypes = [P(ObParams), P(ObBatch), C.c_int, C.c_double, C.c_double,
                                         P(C.c_int), _i32p]
        _lib.oracle_point_sd.restype = C.c_double
        _lib.oracle_loss.argtypes = [P(ObParams), P(ObBatch), C.c_int, P(ObState), _dp, C.c_int, C.c_int,
                                     C.c_double, C.c_double]
        _lib.oracle_loss.restype = C.c_double
        _lib.oracle_loss_grad.argtypes = [P(ObParams), P(ObBatch), C.c_int, P(ObState), _dp, C.c_int,
                                          C.c_int, C.c_double, C.c_double, C.c_int, _i32p, _i32p, _i32p, _dp]
        _lib.oracle_objective.argtypes = [P(ObParams), P(ObBatch), C.c_int, P(ObState), _dp, C.c_int, C.c_int,
                                          C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
        _lib.oracle_objective.restype = C.c_double
        _lib.oracle_objective_grad.argtypes = [P(ObParams), P(ObBatch), C.c_int, P(ObState), _dp, C.c_int,
                                               C.c_int, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp,
                                               C.c_int, _i32p, _i32p, _i32p, _i32p, _dp]
    return _lib


@dataclass
class Params:
    """Method constants (same meaning and defaults as the GPU library's)."""
    dt: float = 0.1
    idm_amax: float = 2.0
    idm_b: float = 3.0
    idm_T: float = 1.5
    idm_s0: float = 2.0
    idm_dq: float = 2.0
    route_h: float = 0.5
    gap_min: float = 0.1
    band: float = 1e-4
    idm_K: int = 32
    kin_amax: float = 6.0
    kin_kmax: float = 0.3
    kin_band_a: float = 1e-3
    kin_band_th: float = 1e-5
    route_max_dist: float = 5.0
    route_max_rel: float = 2.0
    disc_a_max: float = 6.0
    disc_k_max: float = 0.3
    disc_d_max: float = 6.0
    disc_t_max: float = 0.3
    disc_na: int = 13
    disc_nk: int = 31
    disc_nd: int = 25
    disc_nt: int = 13

    def c(self) -> ObParams:
        return ObParams(self.dt, self.idm_amax, self.idm_b, self.idm_T, self.idm_s0, self.idm_dq,
                        self.route_h, self.gap_min, self.band, self.idm_K, 0, self.kin_amax, self.kin_kmax,
                        self.kin_band_a, self.kin_band_th, self.route_max_dist, self.route_max_rel,
                        self.disc_a_max, self.disc_k_max, self.disc_d_max, self.disc_t_max, self.disc_na,
                        self.disc_nk, self.disc_nd, self.disc_nt)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


STATE_KEYS = ("x", "y", "th", "vx", "vy", "s")
CTRL_HOLD, CTRL_ACTION, CTRL_EXPERT, CTRL_LOG, CTRL_EXPERT_DISCRETE = 0, 1, 2, 3, 4


class Oracle:
    """FP64 view of a SceneBatch (arrays kept alive while the object lives)."""

    def __init__(self, batch, params: Optional[Params] = None):
        self.b = batch
        self.p = params or Params()
        self._cp = self.p.c()
        keep = {}

        def k(name, arr):
            keep[name] = arr
            return arr

        self._batch = ObBatch(
            batch.S, batch.N_tot, batch.log_x.shape[0], 0,
            _ptr(k("ao", np.ascontiguousarray(batch.agent_off, np.int32)), _i32p),
            _ptr(k("ro", np.ascontiguousarray(batch.rg_off, np.int32)), _i32p),
            _ptr(k("L", _f64(batch.L)), _dp), _ptr(k("W", _f64(batch.W)), _dp),
            _ptr(k("v0", _f64(batch.idm_v0)), _dp),
            _ptr(k("valid", np.ascontiguousarray(batch.valid, np.uint8)), _u8p),
            _ptr(k("kind", np.ascontiguousarray(batch.kind, np.uint8)), _u8p),
            _ptr(k("rto", np.ascontiguousarray(batch.route_off, np.int32)), _i32p),
            _ptr(k("rx", _f64(batch.route_x)), _dp), _ptr(k("ry", _f64(batch.route_y)), _dp),
            _ptr(k("gx", _f64(batch.rg_x)), _dp), _ptr(k("gy", _f64(batch.rg_y)), _dp),
            _ptr(k("gp", np.ascontiguousarray(batch.rg_poly, np.int32)), _i32p),
            _ptr(k("gt", np.ascontiguousarray(batch.rg_type, np.uint8)), _u8p),
            _ptr(k("gv", np.ascontiguousarray(batch.rg_valid, np.uint8)), _u8p),
            _ptr(k("lx", _f64(batch.log_x)), _dp), _ptr(k("ly", _f64(batch.log_y)), _dp),
            _ptr(k("lth", _f64(batch.log_th)), _dp), _ptr(k("lvx", _f64(batch.log_vx)), _dp),
            _ptr(k("lvy", _f64(batch.log_vy)), _dp),
            _ptr(k("po", np.ascontiguousarray(batch.path_off, np.int32)), _i32p),
            _ptr(k("ppo", np.ascontiguousarray(batch.path_pt_off, np.int32)), _i32p),
            _ptr(k("px", _f64(batch.path_x)), _dp), _ptr(k("py", _f64(batch.path_y)), _dp),
            _ptr(k("pon", np.ascontiguousarray(batch.path_on, np.uint8)), _u8p),
        )
        self._keep = keep

    # -- state helpers -------------------------------------------------------
    def initial_state(self) -> dict:
        b = self.b
        st = {k: _f64(getattr(b, k)).copy() for k in ("x", "y", "th", "vx", "vy")}
        st["s"] = np.zeros(b.N_tot)
        return st

    @staticmethod
    def _cstate(st: dict) -> ObState:
        for k in STATE_KEYS:
            assert st[k].dtype == np.float64 and st[k].flags.c_contiguous
        return ObState(*[_ptr(st[k], _dp) for k in STATE_KEYS])

    def _scenes(self, scenes):
        return (0, self.b.S) if scenes is None else scenes

    # -- calls ---------------------------------------------------------------
    def transition(self, st: dict, act: Optional[np.ndarray], ctrl=None, scenes=None, t_next: int = -1):
        """State t -> t+1 = t_next; act is [3][N_tot] (None: no agent takes
        CTRL_ACTION).  Returns (state, band_idm, lead)."""
        N = self.b.N_tot
        s0, s1 = self._scenes(scenes)
        st = {k: _f64(st[k]) for k in STATE_KEYS}
        out = {k: st[k].copy() for k in STATE_KEYS}
        act_p = None
        if act is not None:
            act = _f64(act).reshape(3, N)
            act_p = _ptr(act, _dp)
        band = np.zeros(N, np.uint8)
        lead = np.full(N, -1, np.int32)
        ctrl_a = None if ctrl is None else np.ascontiguousarray(ctrl, np.uint8)
        ctrl_p = None if ctrl_a is None else _ptr(ctrl_a, _u8p)
        rc = lib().oracle_transition(C.byref(self._cp), C.byref(self._batch), s0, s1, C.byref(self._cstate(st)),
                                     act_p, ctrl_p, t_next, C.byref(self._cstate(out)),
                                     _ptr(band, _u8p), _ptr(lead, _i32p))
        if rc:
            raise RuntimeError("oracle_transition failed")
        return out, band, lead

    def metrics(self, st: dict, t: int, scenes=None, prev: Optional[dict] = None) -> dict:
        """Metrics of state st against log row t; with prev (the state
        before) also the kinematic-infeasibility bits."""
        N, S = self.b.N_tot, self.b.S
        s0, s1 = self._scenes(scenes)
        st = {k: _f64(st[k]) for k in STATE_KEYS}
        m = dict(ov=np.zeros(N), off=np.zeros(N), logdiv=np.zeros(N), flags=np.zeros(N, np.uint8),
                 reward=np.zeros(S, np.int32))
        cm = ObMetrics(_ptr(m["ov"], _dp), _ptr(m["off"], _dp), _ptr(m["logdiv"], _dp),
                       _ptr(m["flags"], _u8p), _ptr(m["reward"], _i32p))
        pv = None
        if prev is not None:
            prev = {k: _f64(prev[k]) for k in STATE_KEYS}
            pv = C.byref(self._cstate(prev))
        rc = lib().oracle_metrics(C.byref(self._cp), C.byref(self._batch), s0, s1, C.byref(self._cstate(st)),
                                  pv, t, C.byref(cm))
        if rc:
            raise RuntimeError("oracle_metrics failed")
        return m

    def rollout(self, st: dict, act_seq: Optional[np.ndarray], t0: int, T: int, scenes=None, nthreads: int = 0,
                ctrl=None):
        """Free-running FP64 rollout; returns (final state, metrics [T][...])."""
        N, S = self.b.N_tot, self.b.S
        s0, s1 = self._scenes(scenes)
        st = {k: _f64(st[k]).copy() for k in STATE_KEYS}
        act_p = None
        if act_seq is not None:
            act = _f64(act_seq).reshape(-1, 3, N)
            act_p = _ptr(act, _dp)
        ctrl_a = None if ctrl is None else np.ascontiguousarray(ctrl, np.uint8)
        ctrl_p = None if ctrl_a is None else _ptr(ctrl_a, _u8p)
        m = dict(ov=np.zeros((T, N)), off=np.zeros((T, N)), logdiv=np.zeros((T, N)),
                 flags=np.zeros((T, N), np.uint8), reward=np.zeros((T, S), np.int32))
        cm = ObMetrics(_ptr(m["ov"], _dp), _ptr(m["off"], _dp), _ptr(m["logdiv"], _dp),
                       _ptr(m["flags"], _u8p), _ptr(m["reward"], _i32p))
        rc = lib().oracle_rollout(C.byref(self._cp), C.byref(self._batch), s0, s1, C.byref(self._cstate(st)),
                                  act_p, ctrl_p, t0, T, C.byref(cm), nthreads)
        if rc:
            raise RuntimeError("oracle_rollout failed")
        return st, m

    def inverse(self, prev: dict, nxt: dict, scenes=None) -> np.ndarray:
        """The action [3][N_tot] taking prev to nxt in each agent's action space."""
        N = self.b.N_tot
        s0, s1 = self._scenes(scenes)
        a = {k: _f64(prev[k]) for k in STATE_KEYS}
        c = {k: _f64(nxt[k]) for k in STATE_KEYS}
        out = np.zeros((3, N))
        rc = lib().oracle_inverse(C.byref(self._cp), C.byref(self._batch), s0, s1, C.byref(self._cstate(a)),
                                  C.byref(self._cstate(c)), _ptr(out, _dp))
        if rc:
            raise RuntimeError("oracle_inverse failed")
        return out

    def observe(self, st: dict, M: int, K: int, observers=None, scenes=None) -> dict:
        """Observation of state st (Sec. 3.2): agents [N_tot, M, 5] and
        agents_valid [N_tot, M]; rg [N_tot, K, 2] and rg_idx [N_tot, K]
        (rows of non-observers zero / -1)."""
        N = self.b.N_tot
        s0, s1 = self._scenes(scenes)
        st = {k: _f64(st[k]) for k in STATE_KEYS}
        out = dict(agents=np.zeros((N, M, 5)), agents_valid=np.zeros((N, M), np.uint8),
                   rg=np.zeros((N, K, 2)), rg_idx=np.full((N, K), -1, np.int32))
        obs = None if observers is None else np.ascontiguousarray(observers, np.uint8)
        rc = lib().oracle_observe(C.byref(self._cp), C.byref(self._batch), s0, s1, C.byref(self._cstate(st)),
                                  None if obs is None else _ptr(obs, _u8p), M, K, _ptr(out["agents"], _dp),
                                  _ptr(out["agents_valid"], _u8p), _ptr(out["rg"], _dp), _ptr(out["rg_idx"], _i32p))
        if rc:
            raise RuntimeError("oracle_observe failed")
        return out

    def discretize(self, act_seq: np.ndarray):
        """Discrete action indices [T][N_tot] of act_seq [T][3][N_tot] and
        the band flags (a component near a rounding boundary)."""
        act = _f64(act_seq).reshape(-1, 3, self.b.N_tot)
        T = act.shape[0]
        idx = np.zeros((T, self.b.N_tot), np.int32)
        band = np.zeros((T, self.b.N_tot), np.uint8)
        if lib().oracle_discretize(C.byref(self._cp), C.byref(self._batch), _ptr(act, _dp), T, _ptr(idx, _i32p),
                                   _ptr(band, _u8p)):
            raise RuntimeError("oracle_discretize failed")
        return idx, band

    def decode_actions(self, idx: np.ndarray) -> np.ndarray:
        idx = np.ascontiguousarray(idx, np.int32).reshape(-1, self.b.N_tot)
        act = np.zeros((idx.shape[0], 3, self.b.N_tot))
        if lib().oracle_decode_actions(C.byref(self._cp), C.byref(self._batch), _ptr(idx, _i32p), idx.shape[0],
                                       _ptr(act, _dp)):
            raise RuntimeError("oracle_decode_actions failed")
        return act

    def route(self, st: dict, scenes=None):
        """Route progress ratio [S] (NaN when undefined) and flags [S] (bit0
        off-route, bit1 band, bit2 progress ambiguous) of each scene's
        first agent."""
        S = self.b.S
        s0, s1 = self._scenes(scenes)
        st = {k: _f64(st[k]) for k in STATE_KEYS}
        prog = np.full(S, np.nan)
        flags = np.zeros(S, np.uint8)
        rc = lib().oracle_route(C.byref(self._cp), C.byref(self._batch), s0, s1, C.byref(self._cstate(st)),
                                _ptr(prog, _dp), _ptr(flags, _u8p))
        if rc:
            raise RuntimeError("oracle_route failed")
        return prog, flags

    def expert_actions(self, t0: int, T: int, scenes=None) -> np.ndarray:
        """Open-loop expert actions [T][3][N_tot] fitted to the log."""
        N = self.b.N_tot
        s0, s1 = self._scenes(scenes)
        out = np.zeros((T, 3, N))
        rc = lib().oracle_expert_actions(C.byref(self._cp), C.byref(self._batch), s0, s1, t0, T, _ptr(out, _dp))
        if rc:
            raise RuntimeError("oracle_expert_actions failed")
        return out

    def point_sd(self, scene: int, px: float, py: float) -> Tuple[float, int, int]:
        amb = C.c_int(0)
        seg = C.c_int32(-1)
        r = lib().oracle_point_sd(C.byref(self._cp), C.byref(self._batch), scene, px, py, C.byref(amb),
                                  C.byref(seg))
        return r, amb.value, seg.value

    def loss(self, scene: int, st0: dict, act_seq: np.ndarray, t0: int, T: int, lam: float = 1.0,
             tau: float = 0.25) -> float:
        st = {k: _f64(st0[k]) for k in STATE_KEYS}
        act = _f64(act_seq)
        return lib().oracle_loss(C.byref(self._cp), C.byref(self._batch), scene, C.byref(self._cstate(st)),
                                 _ptr(act, _dp), t0, T, lam, tau)

    def loss_grad(self, scene: int, st0: dict, act_seq: np.ndarray, t0: int, T: int, dirs,
                  lam: float = 1.0, tau: float = 0.25) -> np.ndarray:
        """dL/dact[t][c][g] for dirs = iterable of (t, c, g) (dual numbers)."""
        d = np.asarray(list(dirs), dtype=np.int32).reshape(-1, 3)
        dt_, dc, dg = (np.ascontiguousarray(d[:, i]) for i in range(3))
        out = np.zeros(len(d))
        st = {k: _f64(st0[k]) for k in STATE_KEYS}
        act = _f64(act_seq)
        rc = lib().oracle_loss_grad(C.byref(self._cp), C.byref(self._batch), scene, C.byref(self._cstate(st)),
                                    _ptr(act, _dp), t0, T, lam, tau, len(d), _ptr(dt_, _i32p), _ptr(dc, _i32p),
                                    _ptr(dg, _i32p), _ptr(out, _dp))
        if rc:
            raise RuntimeError("oracle_loss_grad failed")
        return out


    @staticmethod
    def _weights(w, T, N):
        if w is None:
            return None, None
        a = _f64(w).reshape(T, N)
        return a, _ptr(a, _dp)

    def objective(self, scene: int, st0: dict, act_seq: np.ndarray, t0: int, T: int, w_loss: float = 0.0,
                  g_logdiv=None, g_ov=None, g_off=None, lam: float = 1.0, tau: float = 0.25) -> float:
        """J = w_loss * loss + sum of the weighted per-step metrics (weights
        [T][N_tot] or None) of the scene's T-step rollout (oracle_objective)."""
        st = {k: _f64(st0[k]) for k in STATE_KEYS}
        act = _f64(act_seq)
        N = self.b.N_tot
        keep = [self._weights(w, T, N) for w in (g_logdiv, g_ov, g_off)]
        return lib().oracle_objective(C.byref(self._cp), C.byref(self._batch), scene, C.byref(self._cstate(st)),
                                      _ptr(act, _dp), t0, T, lam, tau, w_loss, *[k[1] for k in keep])

    def objective_grad(self, scene: int, st0: dict, act_seq: np.ndarray, t0: int, T: int, dirs,
                       w_loss: float = 0.0, g_logdiv=None, g_ov=None, g_off=None, lam: float = 1.0,
                       tau: float = 0.25) -> np.ndarray:
        """dJ/d(direction) by dual numbers for dirs = iterable of (kind, t, c,
        g): kind 0 = act_seq[t][c][g]; kind 1 = component c (x, y, theta, vx,
        vy) of agent g's initial state."""
        d = np.asarray(list(dirs), dtype=np.int32).reshape(-1, 4)
        dk, dt_, dc, dg = (np.ascontiguousarray(d[:, i]) for i in range(4))
        out = np.zeros(len(d))
        st = {k: _f64(st0[k]) for k in STATE_KEYS}
        act = _f64(act_seq)
        N = self.b.N_tot
        keep = [self._weights(w, T, N) for w in (g_logdiv, g_ov, g_off)]
        rc = lib().oracle_objective_grad(C.byref(self._cp), C.byref(self._batch), scene,
                                         C.byref(self._cstate(st)), _ptr(act, _dp), t0, T, lam, tau, w_loss,
                                         *[k[1] for k in keep], len(d), _ptr(dk, _i32p), _ptr(dt_, _i32p),
                                         _ptr(dc, _i32p), _ptr(dg, _i32p), _ptr(out, _dp))
        if rc:
            raise RuntimeError("oracle_objective_grad failed")
        return out


def box_depth(a, b) -> float:
    """SAT depth of boxes given as (x, y, theta, L, W)."""
    A, B = _f64(a), _f64(b)
    return lib().oracle_box_depth(_ptr(A, _dp), _ptr(B, _dp))
