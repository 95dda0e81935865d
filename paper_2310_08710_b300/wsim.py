"""Python binding of libwsim.so (include/wsim.h).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of the library.  PyTorch provides device memory (tensors) and
streams.  Importing this module loads libwsim.so and raises if it is missing;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwsim.so")

OK, EINVAL, ESIZE, ECUDA, ENONFINITE, ETIMEOUT, ENOMEM, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
MODE_GRAPH, MODE_STREAM, MODE_PLAIN, MODE_FUSED = 0, 1, 2, 3
GRAD_PLAIN = 1
MAX_AGENTS = 256
COUNTERS = 6  # wsim_counters: evals, tile tests, SAT pairs, IDM sample tests, pair bound tests, IDM circle tests
FLAG_COLLISION, FLAG_OFFROAD, FLAG_KININF = 1, 2, 4
CTRL_HOLD, CTRL_ACTION, CTRL_EXPERT, CTRL_LOG, CTRL_EXPERT_DISCRETE = 0, 1, 2, 3, 4

_fp = C.POINTER(C.c_float)
_u8p = C.POINTER(C.c_uint8)
_i32p = C.POINTER(C.c_int32)


class WsimConfig(C.Structure):
    _fields_ = [("dt", C.c_float), ("idm_amax", C.c_float), ("idm_b", C.c_float), ("idm_T", C.c_float),
                ("idm_s0", C.c_float), ("idm_dq", C.c_float), ("route_h", C.c_float), ("gap_min", C.c_float),
                ("loss_lambda", C.c_float), ("loss_tau", C.c_float), ("ckpt_every", C.c_int32),
                ("tile_segs", C.c_int32), ("kin_amax", C.c_float), ("kin_kmax", C.c_float),
                ("route_max_dist", C.c_float), ("route_max_rel", C.c_float),
                ("disc_a_max", C.c_float), ("disc_k_max", C.c_float), ("disc_d_max", C.c_float),
                ("disc_t_max", C.c_float), ("disc_na", C.c_int32), ("disc_nk", C.c_int32), ("disc_nd", C.c_int32),
                ("disc_nt", C.c_int32)]


class WsimBatch(C.Structure):
    _fields_ = [("S", C.c_int32), ("N_tot", C.c_int32), ("T_log", C.c_int32), ("pad_", C.c_int32),
                ("R_tot", C.c_int64), ("route_tot", C.c_int64),
                ("agent_off", C.c_void_p), ("rg_off", C.c_void_p),
                ("L", C.c_void_p), ("W", C.c_void_p), ("idm_v0", C.c_void_p),
                ("valid", C.c_void_p), ("kind", C.c_void_p), ("route_off", C.c_void_p),
                ("route_x", C.c_void_p), ("route_y", C.c_void_p), ("rg_x", C.c_void_p), ("rg_y", C.c_void_p),
                ("rg_poly", C.c_void_p), ("rg_type", C.c_void_p), ("rg_valid", C.c_void_p),
                ("log_x", C.c_void_p), ("log_y", C.c_void_p),
                ("log_th", C.c_void_p), ("log_vx", C.c_void_p), ("log_vy", C.c_void_p),
                ("path_off", C.c_void_p), ("path_pt_off", C.c_void_p), ("path_x", C.c_void_p),
                ("path_y", C.c_void_p), ("path_on", C.c_void_p)]


STATE_FIELDS = ("x", "y", "x_lo", "y_lo", "th", "th_lo", "vx", "vy", "s", "s_lo")


class WsimState(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in STATE_FIELDS]


ROLL_SHAPES, BUCKETS = 5, 3


class WsimTuning(C.Structure):
    _fields_ = [("split", C.c_int32), ("single_shape", C.c_int32), ("bucket_shape", C.c_int32 * BUCKETS),
                ("bucket_scenes", C.c_int32 * BUCKETS), ("ms_single", C.c_float * ROLL_SHAPES),
                ("ms_bucket", (C.c_float * ROLL_SHAPES) * BUCKETS), ("ms_split", C.c_float)]

    def as_dict(self) -> dict:
        return {"split": bool(self.split), "single_shape": self.single_shape,
                "bucket_shape": list(self.bucket_shape), "bucket_scenes": list(self.bucket_scenes),
                "ms_single": [round(v, 4) for v in self.ms_single],
                "ms_bucket": [[round(v, 4) for v in row] for row in self.ms_bucket],
                "ms_split": round(self.ms_split, 4)}


class WsimMetricBuf(C.Structure):
    _fields_ = [("ov", C.c_void_p), ("off", C.c_void_p), ("logdiv", C.c_void_p), ("flags", C.c_void_p),
                ("reward", C.c_void_p)]


class WsimMetricGrad(C.Structure):
    _fields_ = [("logdiv", C.c_void_p), ("ov", C.c_void_p), ("off", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libwsim.so is not built ({LIB_PATH}); run paper_2310_08710_b300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    lib.wsim_default_config.argtypes = [P(WsimConfig)]
    lib.wsim_default_config.restype = None
    lib.wsim_init.argtypes = [P(vp), P(WsimConfig), P(WsimBatch), vp]
    lib.wsim_step.argtypes = [vp, P(WsimState), vp, vp, P(WsimState), P(WsimMetricBuf), C.c_int, vp]
    lib.wsim_metrics.argtypes = [vp, P(WsimState), P(WsimMetricBuf), C.c_int, vp]
    lib.wsim_rollout.argtypes = [vp, P(WsimState), vp, vp, C.c_int, C.c_int, C.c_int, P(WsimMetricBuf),
                                 P(WsimState), vp]
    lib.wsim_status.argtypes = [vp, P(C.c_int), vp]
    lib.wsim_set_counting.argtypes = [vp, C.c_int]
    lib.wsim_counters.argtypes = [vp, P(C.c_int64), vp]
    lib.wsim_strerror.argtypes = [C.c_int]
    lib.wsim_strerror.restype = C.c_char_p
    lib.wsim_destroy.argtypes = [vp]
    lib.wsim_destroy.restype = None
    lib.wsim_autotune.argtypes = [vp, P(WsimState), vp, C.c_int, C.c_int, P(WsimTuning), vp]
    lib.wsim_set_tuning.argtypes = [vp, P(WsimTuning)]
    lib.wsim_get_tuning.argtypes = [vp, P(WsimTuning)]
    lib.wsim_loss_grad.argtypes = [vp, P(WsimState), vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp]
    lib.wsim_rollout_record.argtypes = [vp, P(WsimState), vp, C.c_int, C.c_int, C.c_int, P(WsimMetricBuf), vp,
                                        P(WsimState), vp]
    lib.wsim_rollout_backward.argtypes = [vp, vp, P(WsimMetricGrad), vp, vp, P(WsimState), vp]
    lib.wsim_metrics_static.argtypes = [P(WsimConfig), P(WsimBatch), P(WsimState), P(WsimMetricBuf), C.c_int, vp]
    lib.wsim_expert_actions.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    lib.wsim_discretize.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.wsim_decode_actions.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.wsim_route_metrics.argtypes = [vp, P(WsimState), vp, vp, vp]
    lib.wsim_observe.argtypes = [vp, P(WsimState), vp, C.c_int, C.c_int, vp, vp, vp, vp, vp]
    return lib


lib = _load()

EXPORTED = ("wsim_default_config", "wsim_init", "wsim_step", "wsim_metrics", "wsim_rollout", "wsim_status",
            "wsim_set_counting", "wsim_counters", "wsim_strerror", "wsim_destroy", "wsim_metrics_static",
            "wsim_autotune", "wsim_set_tuning", "wsim_get_tuning", "wsim_loss_grad", "wsim_rollout_record",
            "wsim_rollout_backward", "wsim_expert_actions", "wsim_observe",
            "wsim_route_metrics", "wsim_discretize", "wsim_decode_actions")


class WsimError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {lib.wsim_strerror(code).decode()} ({code})")
        self.code = code


def _check(rc: int, where: str):
    if rc != OK:
        raise WsimError(rc, where)


def default_config(**over) -> WsimConfig:
    c = WsimConfig()
    lib.wsim_default_config(C.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def _stream(stream: Optional[torch.cuda.Stream]) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


class DeviceBatch:
    """A SceneBatch copied into device tensors, plus its wsim_batch view."""

    def __init__(self, b, device="cuda"):
        dev = torch.device(device)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
        self.S, self.N_tot, self.T_log = b.S, b.N_tot, b.log_x.shape[0]
        self.agent_off = t(b.agent_off, torch.int32)
        self.rg_off = t(b.rg_off, torch.int32)
        self.L, self.W, self.idm_v0 = t(b.L, torch.float32), t(b.W, torch.float32), t(b.idm_v0, torch.float32)
        self.valid, self.kind = t(b.valid, torch.uint8), t(b.kind, torch.uint8)
        self.route_off = t(b.route_off, torch.int32)
        self.route_x, self.route_y = t(b.route_x, torch.float32), t(b.route_y, torch.float32)
        self.rg_x, self.rg_y = t(b.rg_x, torch.float32), t(b.rg_y, torch.float32)
        self.rg_poly = t(b.rg_poly, torch.int32)
        self.rg_type, self.rg_valid = t(b.rg_type, torch.uint8), t(b.rg_valid, torch.uint8)
        self.log_x, self.log_y = t(b.log_x, torch.float32), t(b.log_y, torch.float32)
        full = getattr(b, "log_th", None) is not None
        self.log_th = t(b.log_th, torch.float32) if full else None
        self.log_vx = t(b.log_vx, torch.float32) if full else None
        self.log_vy = t(b.log_vy, torch.float32) if full else None
        paths = getattr(b, "path_off", None) is not None and int(b.path_off[-1]) > 0
        self.path_off = t(b.path_off, torch.int32) if paths else None
        self.path_pt_off = t(b.path_pt_off, torch.int32) if paths else None
        self.path_x = t(b.path_x, torch.float32) if paths else None
        self.path_y = t(b.path_y, torch.float32) if paths else None
        self.path_on = t(b.path_on, torch.uint8) if paths else None
        self.c = WsimBatch(self.S, self.N_tot, self.T_log, 0, int(b.rg_off[-1]), int(b.route_off[-1]),
                           *[_ptr(getattr(self, k)) for k in (
                               "agent_off", "rg_off", "L", "W", "idm_v0", "valid", "kind", "route_off",
                               "route_x", "route_y", "rg_x", "rg_y", "rg_poly", "rg_type", "rg_valid",
                               "log_x", "log_y", "log_th", "log_vx", "log_vy",
                               "path_off", "path_pt_off", "path_x", "path_y", "path_on")])


class State:
    """Agent state in one [10, n_rows * N] float32 tensor (rows of N agents)."""

    def __init__(self, N: int, rows: int = 1, device="cuda", data: Optional[torch.Tensor] = None):
        self.N, self.rows = N, rows
        self.data = data if data is not None else torch.zeros((10, rows * N), dtype=torch.float32, device=device)

    @classmethod
    def from_batch(cls, b, device="cuda") -> "State":
        st = cls(b.N_tot, device=device)
        for k in ("x", "y", "th", "vx", "vy"):
            st.data[STATE_FIELDS.index(k)] = torch.as_tensor(getattr(b, k)).to(device)
        return st

    def field(self, k: str) -> torch.Tensor:
        return self.data[STATE_FIELDS.index(k)].view(self.rows, self.N)

    def c(self, row: int = 0) -> WsimState:
        base = row * self.N
        return WsimState(*[self.data[i, base:].data_ptr() for i in range(10)])

    def clone(self) -> "State":
        return State(self.N, self.rows, data=self.data.clone())


class Metrics:
    """Metric arrays for `rows` steps: [rows, N] (reward [rows, S])."""

    def __init__(self, N: int, S: int, rows: int = 1, device="cuda"):
        f = lambda: torch.zeros((rows, N), dtype=torch.float32, device=device)
        self.ov, self.off, self.logdiv = f(), f(), f()
        self.flags = torch.zeros((rows, N), dtype=torch.uint8, device=device)
        self.reward = torch.zeros((rows, S), dtype=torch.int32, device=device)

    def c(self) -> WsimMetricBuf:
        return WsimMetricBuf(self.ov.data_ptr(), self.off.data_ptr(), self.logdiv.data_ptr(),
                             self.flags.data_ptr(), self.reward.data_ptr())


class Sim:
    """A wsim context over one device batch."""

    def __init__(self, batch: DeviceBatch, cfg: Optional[WsimConfig] = None, stream=None):
        self.batch = batch
        self.cfg = cfg if cfg is not None else default_config()
        self._h = C.c_void_p()
        _check(lib.wsim_init(C.byref(self._h), C.byref(self.cfg), C.byref(batch.c), _stream(stream)), "wsim_init")

    def close(self):
        if self._h:
            lib.wsim_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, st_in: State, act: Optional[torch.Tensor], st_out: State, m: Optional[Metrics], t: int,
             ctrl: Optional[torch.Tensor] = None, stream=None):
        mc = m.c() if m is not None else None
        _check(lib.wsim_step(self._h, C.byref(st_in.c()), _ptr(act), _ptr(ctrl), C.byref(st_out.c()),
                             C.byref(mc) if mc is not None else None, t, _stream(stream)), "wsim_step")

    def metrics(self, st: State, m: Metrics, t: int, stream=None):
        _check(lib.wsim_metrics(self._h, C.byref(st.c()), C.byref(m.c()), t, _stream(stream)), "wsim_metrics")

    def rollout(self, st: State, act_seq: Optional[torch.Tensor], mseq: Metrics, t0: int, T: int,
                mode: int = MODE_GRAPH, ctrl: Optional[torch.Tensor] = None, traj: Optional[State] = None,
                stream=None):
        tc = traj.c() if traj is not None else None
        _check(lib.wsim_rollout(self._h, C.byref(st.c()), _ptr(act_seq), _ptr(ctrl), t0, T, mode,
                                C.byref(mseq.c()), C.byref(tc) if tc is not None else None, _stream(stream)),
               "wsim_rollout")

    def autotune(self, st: State, act_seq: torch.Tensor, t0: int = 10, T: int = 8, stream=None) -> dict:
        """Times the rollout launch configurations on this workload and keeps
        the fastest (see wsim_autotune)."""
        t = WsimTuning()
        _check(lib.wsim_autotune(self._h, C.byref(st.c()), act_seq.data_ptr(), t0, T, C.byref(t), _stream(stream)),
               "wsim_autotune")
        return t.as_dict()

    def set_tuning(self, split: bool = False, single_shape: int = 3, bucket_shape=(4, 0, 3)):
        t = WsimTuning()
        t.split, t.single_shape = int(split), single_shape
        for i, v in enumerate(bucket_shape):
            t.bucket_shape[i] = v
        _check(lib.wsim_set_tuning(self._h, C.byref(t)), "wsim_set_tuning")

    def get_tuning(self) -> dict:
        t = WsimTuning()
        _check(lib.wsim_get_tuning(self._h, C.byref(t)), "wsim_get_tuning")
        return t.as_dict()

    def loss_grad(self, st0: State, act_seq: torch.Tensor, t0: int = 10, T: Optional[int] = None,
                  ckpt_every: int = 10, grad: bool = True, plain: bool = False, stream=None):
        """BPTT loss of every scene (float64 [S]) and dL/dact ([T, 3, N_tot], or
        None when grad is False) of a T-step rollout from st0 (wsim_loss_grad)."""
        T = act_seq.shape[0] if T is None else T
        dev = act_seq.device
        loss = torch.empty(self.batch.S, dtype=torch.float64, device=dev)
        dact = torch.empty((T, 3, self.batch.N_tot), dtype=torch.float32, device=dev) if grad else None
        _check(lib.wsim_loss_grad(self._h, C.byref(st0.c()), act_seq.data_ptr(), t0, T, ckpt_every,
                                  GRAD_PLAIN if plain else 0, loss.data_ptr(), _ptr(dact), _stream(stream)),
               "wsim_loss_grad")
        return loss, dact

    def rollout_record(self, st0: State, act_seq: torch.Tensor, mseq: Optional[Metrics] = None, t0: int = 10,
                       T: Optional[int] = None, ckpt_every: int = 10, loss: bool = True,
                       st_T: Optional[State] = None, stream=None) -> Optional[torch.Tensor]:
        """Differentiable rollout, forward half (wsim_rollout_record): the
        T-step rollout from st0 with its checkpoints and, with mseq, its
        metric rows and their deciding indices kept in the context for
        rollout_backward.  Returns the scene losses (float64 [S]) or None."""
        T = act_seq.shape[0] if T is None else T
        out = torch.empty(self.batch.S, dtype=torch.float64, device=act_seq.device) if loss else None
        mc = mseq.c() if mseq is not None else None
        sc = st_T.c() if st_T is not None else None
        _check(lib.wsim_rollout_record(self._h, C.byref(st0.c()), act_seq.data_ptr(), t0, T, ckpt_every,
                                       C.byref(mc) if mc is not None else None, _ptr(out),
                                       C.byref(sc) if sc is not None else None, _stream(stream)),
               "wsim_rollout_record")
        self.record_id = getattr(self, "record_id", 0) + 1
        return out

    def rollout_backward(self, act_seq: torch.Tensor, g_logdiv: Optional[torch.Tensor] = None,
                         g_ov: Optional[torch.Tensor] = None, g_off: Optional[torch.Tensor] = None,
                         loss_w: Optional[torch.Tensor] = None, dact: bool = True, dst0: bool = True, stream=None):
        """Differentiable rollout, reverse half (wsim_rollout_backward): dJ/dact
        ([T, 3, N_tot]) and dJ/d(initial state) (a State) of J = sum loss_w *
        loss + the metric rows weighted by g_* ([T, N_tot] float32 each)."""
        T, dev = act_seq.shape[0], act_seq.device
        N = self.batch.N_tot
        f = lambda t: None if t is None else t.detach().to(torch.float32).contiguous()
        g_logdiv, g_ov, g_off = f(g_logdiv), f(g_ov), f(g_off)
        lw = None if loss_w is None else loss_w.detach().to(torch.float64).contiguous()
        gm = WsimMetricGrad(_ptr(g_logdiv), _ptr(g_ov), _ptr(g_off))
        da = torch.empty((T, 3, N), dtype=torch.float32, device=dev) if dact else None
        ds = State(N, device=dev) if dst0 else None
        dc = ds.c() if ds is not None else None
        _check(lib.wsim_rollout_backward(self._h, act_seq.data_ptr(), C.byref(gm), _ptr(lw), _ptr(da),
                                         C.byref(dc) if dc is not None else None, _stream(stream)),
               "wsim_rollout_backward")
        return da, ds

    def observe(self, st: State, M: int, K: int, observers: Optional[torch.Tensor] = None, out: Optional[dict] = None,
                stream=None) -> dict:
        """Observation (wsim_observe): agents [N_tot, M, 5], agents_valid
        [N_tot, M], rg [N_tot, K, 2], rg_idx [N_tot, K]; rows of agents that
        do not observe are left as they were in `out` (zeros / -1 when new)."""
        N, dev = self.batch.N_tot, self.batch.log_x.device
        if out is None:
            out = dict(agents=torch.zeros((N, M, 5), dtype=torch.float32, device=dev),
                       agents_valid=torch.zeros((N, M), dtype=torch.uint8, device=dev),
                       rg=torch.zeros((N, K, 2), dtype=torch.float32, device=dev),
                       rg_idx=torch.full((N, K), -1, dtype=torch.int32, device=dev))
        _check(lib.wsim_observe(self._h, C.byref(st.c()), _ptr(observers), M, K, out["agents"].data_ptr(),
                                out["agents_valid"].data_ptr(), out["rg"].data_ptr(), out["rg_idx"].data_ptr(),
                                _stream(stream)), "wsim_observe")
        return out

    def discretize(self, act_seq: torch.Tensor, stream=None) -> torch.Tensor:
        """Flat discrete action indices [T, N_tot] of act_seq [T, 3, N_tot]
        (wsim_discretize)."""
        T = act_seq.shape[0]
        idx = torch.empty((T, self.batch.N_tot), dtype=torch.int32, device=act_seq.device)
        _check(lib.wsim_discretize(self._h, act_seq.data_ptr(), T, idx.data_ptr(), _stream(stream)),
               "wsim_discretize")
        return idx

    def decode_actions(self, idx: torch.Tensor, stream=None) -> torch.Tensor:
        """Grid actions [T, 3, N_tot] of flat indices [T, N_tot]
        (wsim_decode_actions)."""
        T = idx.shape[0]
        act = torch.empty((T, 3, self.batch.N_tot), dtype=torch.float32, device=idx.device)
        _check(lib.wsim_decode_actions(self._h, idx.data_ptr(), T, act.data_ptr(), _stream(stream)),
               "wsim_decode_actions")
        return act

    def route_metrics(self, st: State, stream=None):
        """Route progress ratio (float32 [S], NaN when undefined) and
        off-route flag (uint8 [S]) of each scene's first agent
        (wsim_route_metrics)."""
        S, dev = self.batch.S, self.batch.log_x.device
        prog = torch.empty(S, dtype=torch.float32, device=dev)
        off = torch.empty(S, dtype=torch.uint8, device=dev)
        _check(lib.wsim_route_metrics(self._h, C.byref(st.c()), prog.data_ptr(), off.data_ptr(), _stream(stream)),
               "wsim_route_metrics")
        return prog, off

    def expert_actions(self, t0: int, T: int, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Open-loop expert actions [T, 3, N_tot] fitted to log rows t0 .. t0+T
        (wsim_expert_actions)."""
        if out is None:
            out = torch.empty((T, 3, self.batch.N_tot), dtype=torch.float32, device=self.batch.log_x.device)
        _check(lib.wsim_expert_actions(self._h, t0, T, out.data_ptr(), _stream(stream)), "wsim_expert_actions")
        return out

    def status(self, stream=None) -> int:
        v = C.c_int(0)
        _check(lib.wsim_status(self._h, C.byref(v), _stream(stream)), "wsim_status")
        return v.value

    def set_counting(self, on: bool):
        _check(lib.wsim_set_counting(self._h, int(on)), "wsim_set_counting")

    def counters(self, stream=None) -> np.ndarray:
        out = (C.c_int64 * COUNTERS)()
        _check(lib.wsim_counters(self._h, out, _stream(stream)), "wsim_counters")
        return np.array(out[:], dtype=np.int64)


def metrics_static(batch: DeviceBatch, st: State, m: Metrics, t: int, cfg: Optional[WsimConfig] = None,
                   stream=None):
    """wsim_metrics_static: the metrics of `st` at log row t with no context
    and no device allocation (for callers that cannot allocate; the library
    keeps the scratch in a fixed device array shared by all calls).
    Synchronises the stream."""
    cfg = cfg if cfg is not None else default_config()
    _check(lib.wsim_metrics_static(C.byref(cfg), C.byref(batch.c), C.byref(st.c()), C.byref(m.c()), t,
                                   _stream(stream)), "wsim_metrics_static")


class RolloutFn(torch.autograd.Function):
    """Differentiable rollout through the recorded forward and its backward:

        logdiv, ov, off, loss = RolloutFn.apply(actions, state0, sim, t0, ckpt_every)

    actions [T, 3, N_tot] and state0 (a State's [10, N_tot] data) are the
    differentiable inputs; the outputs are the metric rows [T, N_tot] of the
    T-step rollout (wsim_rollout's logdiv, ov, off) and the per-scene loss of
    wsim_loss_grad (float64 [S]).  The forward records the rollout in the
    context (wsim_rollout_record); backward runs wsim_rollout_backward with
    the incoming gradients as metric and loss weights.  A context holds one
    record: backward refuses a graph whose forward record was replaced.
    Entries of ov and off that are -inf (no other agent, no road edge) and
    the metrics of invalid agents carry no derivative."""

    @staticmethod
    def forward(ctx, actions: torch.Tensor, state0: torch.Tensor, sim: "Sim", t0: int = 10, ckpt_every: int = 10):
        act = actions.detach().contiguous()
        st0 = State(sim.batch.N_tot, data=state0.detach().contiguous())
        T = act.shape[0]
        m = Metrics(sim.batch.N_tot, sim.batch.S, rows=T, device=act.device)
        loss = sim.rollout_record(st0, act, m, t0, T, ckpt_every, loss=True)
        ctx.sim, ctx.record_id = sim, sim.record_id
        ctx.save_for_backward(act)
        return m.logdiv, m.ov, m.off, loss

    @staticmethod
    def backward(ctx, g_logdiv, g_ov, g_off, g_loss):
        (act,) = ctx.saved_tensors
        sim = ctx.sim
        if sim.record_id != ctx.record_id:
            raise RuntimeError("RolloutFn.backward: the context recorded another rollout since this forward")
        da, ds = sim.rollout_backward(act, g_logdiv, g_ov, g_off, g_loss, dact=ctx.needs_input_grad[0],
                                      dst0=ctx.needs_input_grad[1])
        return da, (ds.data if ds is not None else None), None, None, None


class RolloutLoss(torch.autograd.Function):
    """Differentiable rollout loss: forward returns the per-scene BPTT loss
    (float64 [S]) of a T-step rollout driven by `actions` ([T, 3, N_tot]) and
    records the rollout's checkpoints in the context (wsim_rollout_record,
    without metrics); backward runs the reverse sweep (wsim_rollout_backward)
    with grad_output as the scenes' loss weights.  A forward under no_grad is
    the recording forward alone."""

    @staticmethod
    def forward(ctx, actions: torch.Tensor, sim: "Sim", st0: State, t0: int = 10, ckpt_every: int = 10):
        act = actions.detach().contiguous()
        loss = sim.rollout_record(st0, act, None, t0, act.shape[0], ckpt_every, loss=True)
        ctx.sim, ctx.record_id = sim, sim.record_id
        ctx.save_for_backward(act)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (act,) = ctx.saved_tensors
        sim = ctx.sim
        if sim.record_id != ctx.record_id:
            raise RuntimeError("RolloutLoss.backward: the context recorded another rollout since this forward")
        da, _ = sim.rollout_backward(act, loss_w=grad_loss, dact=True, dst0=False)
        return da, None, None, None, None
