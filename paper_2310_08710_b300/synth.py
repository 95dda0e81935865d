"""Seeded synthetic scenes shaped like the Waymo Open Motion Dataset workloads.

The paper simulates WOMD scenes (Sec. 3.1: 9 s logs at 10 Hz, the first second
is history, up to 128 objects per scene; roadgraph = sampled road/lane
polylines, Sec. 3.2).  The dataset is not available here, so scenes are drawn
from seeded distributions of the same shape.  This module holds no arithmetic
of the simulated method: logs are integrated with the generator's own
continuous-time unicycle model, and delta actions are a random walk, so neither
side's dynamics is reused to make its own inputs.

Every scene s of a batch is drawn from its own counter-based seed
``splitmix64(base_seed ^ s)`` (SplitMix64 of Steele, Lea and Flood, 2014), so
any subset of scenes can be regenerated bit-identically on its own.

Arrays are float32 / int32 / uint8 in the layouts the C ABI takes:
agents and roadgraph points in CSR over scenes, logs time-major
``[T_log][N_tot]``, actions ``[T][3][N_tot]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Optional, Sequence, Tuple, Union

import numpy as np

KIND_BICYCLE, KIND_DELTA, KIND_IDM = 0, 1, 2
RG_EDGE, RG_LANE = 1, 2
T_LOG = 91          # 9.1 s at 10 Hz: 11 history steps + 80 simulated
T0 = 10             # index of the last history step (the simulation start)
T_ROLLOUT = 80
DT = 0.1
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of SplitMix64 for state x (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def scene_rng(base_seed: int, scene: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(splitmix64((base_seed ^ scene) & _M64)))


IntSpec = Union[int, Tuple[int, int]]


@dataclass(frozen=True)
class Workload:
    """Shape of one synthetic workload (the five used here are listed below)."""
    name: str
    S: int                      # scenes
    N: IntSpec                  # agents per scene, or inclusive range
    R: IntSpec                  # roadgraph points per scene, or inclusive range
    driver: str = "bicycle"     # "bicycle": all random bicycle; "idm": ego policy + IDM
    ego_delta_half: bool = False  # scenes < S/2 drive the ego with delta actions
    T: int = T_ROLLOUT


WORKLOADS: Dict[int, Workload] = {
    0: Workload("single scene 1x32x80, 2k roadgraph", 1, 32, 2000),
    1: Workload("batch 1024x128x80, 20k roadgraph, IDM sim agents", 1024, 128, 20000, driver="idm"),
    2: Workload("uneven 4096 x U{8..128} x80, U{1k..30k} roadgraph", 4096, (8, 128), (1000, 30000)),
    3: Workload("differentiable 256x64x80, 2k roadgraph", 256, 64, 2000),
    4: Workload("sweep 16384x128x80, 30k roadgraph, delta/bicycle ego + IDM", 16384, 128, 30000,
                driver="idm", ego_delta_half=True),
}


def _draw(rng: np.random.Generator, spec: IntSpec) -> int:
    if isinstance(spec, tuple):
        return int(rng.integers(spec[0], spec[1] + 1))
    return int(spec)


def _polylines(rng, n_pts, start, heading, arc, radius, turn, spacing=0.5):
    """Points of many polylines at fixed chord spacing: straight or circular arcs.

    Vectorised over all points: polyline p has n_pts[p] points starting at
    start[p] with initial heading heading[p]; arcs turn by 2*asin(spacing/2r)
    per point so every chord has length `spacing`.
    """
    n_pts = np.asarray(n_pts, dtype=np.int64)
    pid = np.repeat(np.arange(len(n_pts)), n_pts)
    first = np.concatenate([[0], np.cumsum(n_pts)[:-1]])
    k = np.arange(n_pts.sum()) - np.repeat(first, n_pts)
    h = heading[pid]
    x0, y0 = start[pid, 0], start[pid, 1]
    r = radius[pid]
    sg = turn[pid]
    dphi = 2.0 * np.arcsin(spacing / (2.0 * r))
    phi = h + sg * k * dphi
    cx = x0 - sg * r * np.sin(h)
    cy = y0 + sg * r * np.cos(h)
    ax = cx + sg * r * np.sin(phi)
    ay = cy - sg * r * np.cos(phi)
    sx = x0 + spacing * k * np.cos(h)
    sy = y0 + spacing * k * np.sin(h)
    a = arc[pid]
    px = np.where(k == 0, x0, np.where(a, ax, sx))
    py = np.where(k == 0, y0, np.where(a, ay, sy))
    return px, py, pid


def _roadgraph(rng, R):
    lens = []
    tot = 0
    while tot < R:
        n = int(rng.integers(20, 201))
        n = min(n, R - tot)
        lens.append(n)
        tot += n
    P = len(lens)
    start = rng.uniform(0.0, 200.0, size=(P, 2))
    heading = rng.uniform(-np.pi, np.pi, size=P)
    arc = rng.random(P) < 0.5
    radius = rng.uniform(10.0, 100.0, size=P)
    turn = np.where(rng.random(P) < 0.5, -1.0, 1.0)
    edge = rng.random(P) < 0.3
    x, y, pid = _polylines(rng, lens, start, heading, arc, radius, turn)
    rtype = np.where(edge[pid], RG_EDGE, RG_LANE).astype(np.uint8)
    return (x.astype(np.float32), y.astype(np.float32), pid.astype(np.int32), rtype,
            np.ones(R, dtype=np.uint8))


def _log_controls(rng, n):
    """Per-agent parameters of the smooth log controls (see _integrate_logs)."""
    return np.stack([rng.uniform(0.0, 2.0, n), rng.uniform(0.05, 0.2, n), rng.uniform(0.0, 2 * np.pi, n),
                     rng.uniform(0.0, 0.05, n), rng.uniform(0.05, 0.2, n), rng.uniform(0.0, 2 * np.pi, n)])


def _integrate_logs(ctl, x0, y0, th0, v0, T_log=T_LOG, t0=T0, sub=10):
    """Logged x, y, heading, vx, vy from a continuous unicycle with smooth
    seeded controls.

    speed' = A sin(2 pi f t + phi) (speed kept >= 0), heading' = K sin(2 pi fk
    t + phik) * speed, integrated with `sub` midpoint substeps per 0.1 s.  The
    logged velocity is the speed along the heading.  History steps before t0
    hold the t0 state.  This is the generator's own integrator, not either
    action space's dynamics, so fitted actions only approximate the log.
    """
    A, f, ph, K, fk, phk = ctl
    n = len(x0)
    lx, ly, lth, lvx, lvy = (np.empty((T_log, n), dtype=np.float32) for _ in range(5))
    x, y, th, v = (np.asarray(a, dtype=np.float64).copy() for a in (x0, y0, th0, v0))

    def record(t):
        lx[t], ly[t], lth[t] = x, y, th
        lvx[t], lvy[t] = v * np.cos(th), v * np.sin(th)

    for t in range(t0 + 1):
        record(t)
    h = DT / sub
    for t in range(t0 + 1, T_log):
        for j in range(sub):
            tm = (t - t0 - 1) * DT + (j + 0.5) * h
            acc = A * np.sin(2 * np.pi * f * tm + ph)
            kap = K * np.sin(2 * np.pi * fk * tm + phk)
            vm = np.maximum(0.0, v + 0.5 * h * acc)
            thm = th + 0.5 * h * kap * v
            x += h * vm * np.cos(thm)
            y += h * vm * np.sin(thm)
            th += h * kap * vm
            v = np.maximum(0.0, v + h * acc)
        record(t)
    return lx, ly, lth, lvx, lvy


def _scene(rng, wl: Workload, s: int, N: Optional[int], R: Optional[int]):
    N = _draw(rng, wl.N) if N is None else N
    R = _draw(rng, wl.R) if R is None else R
    T = wl.T
    # Agents at the simulation start (t0).
    x = rng.uniform(0.0, 200.0, N)
    y = rng.uniform(0.0, 200.0, N)
    th = rng.uniform(-np.pi, np.pi, N)
    sp = rng.uniform(0.0, 20.0, N)
    L = rng.uniform(4.0, 5.5, N)
    W = rng.uniform(1.8, 2.2, N)
    valid = (rng.random(N) >= 0.1).astype(np.uint8)
    valid[0] = 1  # the ego
    kind = np.full(N, KIND_BICYCLE, dtype=np.uint8)
    if wl.driver == "idm":
        kind[1:] = KIND_IDM
    if wl.ego_delta_half and s < wl.S // 2:
        kind[0] = KIND_DELTA
    v0 = rng.uniform(8.0, 15.0, N)
    # Positions are rounded to float32 first so that velocities, routes and
    # logs start from the exact pose both sides see.
    x = x.astype(np.float32).astype(np.float64)
    y = y.astype(np.float32).astype(np.float64)
    th = th.astype(np.float32).astype(np.float64)
    vx = sp * np.cos(th)
    vy = sp * np.sin(th)
    # Roadgraph.
    rg = _roadgraph(rng, R)
    # IDM routes: each IDM agent's own lane from its start pose, 320 points.
    idm = np.nonzero(kind == KIND_IDM)[0]
    n_route = np.zeros(N, dtype=np.int64)
    n_route[idm] = 320
    if len(idm):
        P = len(idm)
        arc = rng.random(P) < 0.5
        radius = rng.uniform(20.0, 200.0, P)
        turn = np.where(rng.random(P) < 0.5, -1.0, 1.0)
        rx, ry, _ = _polylines(rng, n_route[idm], np.stack([x[idm], y[idm]], 1), th[idm], arc, radius, turn)
    else:
        rx = ry = np.zeros(0)
    # Log controls (integrated for the whole batch at once).
    ctl = _log_controls(rng, N)
    # Actions: bicycle a ~ U[-4,4] m/s^2, kappa ~ U[-0.3,0.3] 1/m; delta
    # agents a random walk of displacements at speeds U[0,20] m/s.
    act = np.zeros((T, 3, N), dtype=np.float32)
    act[:, 0, :] = rng.uniform(-4.0, 4.0, (T, N))
    act[:, 1, :] = rng.uniform(-0.3, 0.3, (T, N))
    dl = np.nonzero(kind == KIND_DELTA)[0]
    if len(dl):
        psi = th[dl] + np.cumsum(rng.uniform(-0.05, 0.05, (T, len(dl))), axis=0)
        spd = rng.uniform(0.0, 20.0, (T, len(dl)))
        act[:, 0, dl] = spd * DT * np.cos(psi)
        act[:, 1, dl] = spd * DT * np.sin(psi)
        act[:, 2, dl] = rng.uniform(-0.05, 0.05, (T, len(dl)))
    # Route paths of the ego (built from its log in make_batch): where the two
    # off-route branches leave the on-route path, their turn and curvature.
    branch = np.stack([rng.uniform(0.05, 0.6, 2), rng.uniform(0.4, 1.0, 2) * np.where(rng.random(2) < 0.5, -1, 1),
                       rng.uniform(-0.02, 0.02, 2)])
    return dict(
        N=N, R=R, x=x, y=y, th=th, vx=vx, vy=vy, L=L, W=W, valid=valid, kind=kind, v0=v0,
        rg=rg, n_route=n_route, rx=rx, ry=ry, ctl=ctl, act=act, branch=branch,
    )


def _route_paths(lx, ly, th0, branch):
    """The ego's route paths (Sec. 3.2 on-/off-route paths, synthetic): one
    on-route polyline through its logged positions (t0 onwards, points closer
    than 0.25 m to the previous one dropped) extended 20 m before the start
    and 30 m past the end, and two off-route branches leaving it at the
    fractions branch[0] of its points, turning by branch[1] rad and then
    following curvature branch[2] for 60 m at 1 m spacing."""
    pts = [(lx[0], ly[0])]
    for x, y in zip(lx[1:], ly[1:]):
        if np.hypot(x - pts[-1][0], y - pts[-1][1]) >= 0.25:
            pts.append((x, y))
    pts = np.array(pts, dtype=np.float64)
    d0 = pts[1] - pts[0] if len(pts) > 1 else np.array([np.cos(th0), np.sin(th0)])
    d1 = pts[-1] - pts[-2] if len(pts) > 1 else d0
    d0, d1 = d0 / np.linalg.norm(d0), d1 / np.linalg.norm(d1)
    on = np.concatenate([[pts[0] - 20.0 * d0], pts, [pts[-1] + 30.0 * d1]])
    paths = [on]
    for frac, turn, kap in branch.T:
        k = min(len(on) - 2, max(1, int(frac * (len(on) - 1))))
        u = on[k + 1] - on[k]
        h = np.arctan2(u[1], u[0]) + turn + np.cumsum(np.full(60, kap))
        off = on[k] + np.concatenate([[[0.0, 0.0]], np.cumsum(np.stack([np.cos(h), np.sin(h)], 1), 0)])
        paths.append(off)
    return paths, np.array([1, 0, 0], np.uint8)


@dataclass
class SceneBatch:
    """A batch of scenes in the C ABI's layouts (host numpy arrays)."""
    cfg: int
    seed: int
    scenes: np.ndarray            # scene ids of the source workload
    S: int
    N_tot: int
    T: int
    agent_off: np.ndarray         # int32 [S+1]
    rg_off: np.ndarray            # int32 [S+1]
    L: np.ndarray                 # float32 [N_tot]
    W: np.ndarray
    valid: np.ndarray             # uint8
    kind: np.ndarray              # uint8
    idm_v0: np.ndarray            # float32
    route_off: np.ndarray         # int32 [N_tot+1]
    route_x: np.ndarray           # float32
    route_y: np.ndarray
    rg_x: np.ndarray              # float32 [R_tot]
    rg_y: np.ndarray
    rg_poly: np.ndarray           # int32
    rg_type: np.ndarray           # uint8
    rg_valid: np.ndarray          # uint8
    log_x: np.ndarray             # float32 [T_LOG][N_tot]
    log_y: np.ndarray
    x: np.ndarray                 # float32 [N_tot] state at t0
    y: np.ndarray
    th: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    actions: np.ndarray           # float32 [T][3][N_tot]
    log_th: Optional[np.ndarray] = None   # float32 [T_LOG][N_tot] logged heading (zeros if not given)
    log_vx: Optional[np.ndarray] = None   # logged velocity
    log_vy: Optional[np.ndarray] = None
    # Route paths of each scene's first agent: scene s owns paths
    # [path_off[s], path_off[s+1]); path p owns points [path_pt_off[p],
    # path_pt_off[p+1]); path_on[p] = 1 for an on-route path.
    path_off: Optional[np.ndarray] = None     # int32 [S+1] (no paths if not given)
    path_pt_off: Optional[np.ndarray] = None  # int32 [P+1]
    path_x: Optional[np.ndarray] = None       # float32 [path points]
    path_y: Optional[np.ndarray] = None
    path_on: Optional[np.ndarray] = None      # uint8 [P]
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        for k in ("log_th", "log_vx", "log_vy"):
            if getattr(self, k) is None:
                setattr(self, k, np.zeros_like(self.log_x))
        if self.path_off is None:
            self.path_off = np.zeros(self.S + 1, np.int32)
            self.path_pt_off = np.zeros(1, np.int32)
            self.path_x = np.zeros(0, np.float32)
            self.path_y = np.zeros(0, np.float32)
            self.path_on = np.zeros(0, np.uint8)

    @property
    def T_log(self) -> int:
        return self.log_x.shape[0]

    @property
    def R_tot(self) -> int:
        return int(self.rg_off[-1])

    def agent_steps(self) -> int:
        return self.N_tot * self.T

    def subset(self, idx: Sequence[int]) -> "SceneBatch":
        """The scenes at positions idx of this batch, as a batch of their own."""
        idx = np.asarray(idx, dtype=np.int64)
        a0, a1 = self.agent_off[idx], self.agent_off[idx + 1]
        r0, r1 = self.rg_off[idx], self.rg_off[idx + 1]
        ag = np.concatenate([np.arange(a, b) for a, b in zip(a0, a1)]).astype(np.int64)
        rg = np.concatenate([np.arange(a, b) for a, b in zip(r0, r1)]).astype(np.int64)
        ro0, ro1 = self.route_off[ag], self.route_off[ag + 1]
        rt = np.concatenate([np.arange(a, b) for a, b in zip(ro0, ro1)] + [np.zeros(0, np.int64)]).astype(np.int64)
        off = lambda n: np.concatenate([[0], np.cumsum(n)]).astype(np.int32)
        return SceneBatch(
            cfg=self.cfg, seed=self.seed, scenes=self.scenes[idx], S=len(idx), N_tot=len(ag), T=self.T,
            agent_off=off(a1 - a0), rg_off=off(r1 - r0),
            L=self.L[ag], W=self.W[ag], valid=self.valid[ag], kind=self.kind[ag], idm_v0=self.idm_v0[ag],
            route_off=off(ro1 - ro0), route_x=self.route_x[rt], route_y=self.route_y[rt],
            rg_x=self.rg_x[rg], rg_y=self.rg_y[rg], rg_poly=self.rg_poly[rg], rg_type=self.rg_type[rg],
            rg_valid=self.rg_valid[rg],
            log_x=np.ascontiguousarray(self.log_x[:, ag]), log_y=np.ascontiguousarray(self.log_y[:, ag]),
            log_th=np.ascontiguousarray(self.log_th[:, ag]), log_vx=np.ascontiguousarray(self.log_vx[:, ag]),
            log_vy=np.ascontiguousarray(self.log_vy[:, ag]),
            x=self.x[ag], y=self.y[ag], th=self.th[ag], vx=self.vx[ag], vy=self.vy[ag],
            actions=np.ascontiguousarray(self.actions[:, :, ag]),
            **self._path_subset(idx),
        )

    def _path_subset(self, idx) -> dict:
        p0, p1 = self.path_off[idx], self.path_off[idx + 1]
        pp = np.concatenate([np.arange(a, b) for a, b in zip(p0, p1)] + [np.zeros(0, np.int64)]).astype(np.int64)
        q0, q1 = self.path_pt_off[pp], self.path_pt_off[pp + 1]
        pts = np.concatenate([np.arange(a, b) for a, b in zip(q0, q1)] + [np.zeros(0, np.int64)]).astype(np.int64)
        off = lambda n: np.concatenate([[0], np.cumsum(n)]).astype(np.int32)
        return dict(path_off=off(p1 - p0), path_pt_off=off(q1 - q0), path_x=self.path_x[pts],
                    path_y=self.path_y[pts], path_on=self.path_on[pp])


def make_batch(cfg: int, seed: int = 0, scenes: Optional[Sequence[int]] = None,
               N: Optional[int] = None, R: Optional[int] = None, S: Optional[int] = None,
               T: Optional[int] = None, workers: int = 1) -> SceneBatch:
    """Scenes of workload `cfg` (0-4).

    scenes: ids of the workload's scenes to draw (default all S); a scene's
    content depends only on (seed, id), so subsets reproduce the full batch.
    N, R: override agents / roadgraph points per scene (tests use tiny scenes).
    S: override the scene count of the workload; T: rollout length.
    workers > 1 draws chunks of scenes in that many spawned processes and
    concatenates them (the same arrays as one process draws).
    """
    wl = WORKLOADS[cfg]
    if S is not None:
        wl = Workload(wl.name, S, wl.N, wl.R, wl.driver, wl.ego_delta_half, wl.T)
    if T is not None:
        wl = Workload(wl.name, wl.S, wl.N, wl.R, wl.driver, wl.ego_delta_half, T)
    ids = np.arange(wl.S) if scenes is None else np.asarray(scenes, dtype=np.int64)
    if workers > 1 and len(ids) > 1:
        import concurrent.futures
        import multiprocessing
        chunks = [c for c in np.array_split(ids, min(len(ids), 4 * workers)) if len(c)]
        ctx = multiprocessing.get_context("spawn")  # safe whatever the parent has initialised
        with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            got = list(ex.map(_build, [(cfg, seed, c, N, R, wl) for c in chunks]))
        return concat(got)
    return _build((cfg, seed, ids, N, R, wl))


def _build(job) -> SceneBatch:
    cfg, seed, ids, N, R, wl = job
    parts = [_scene(scene_rng(seed, int(s)), wl, int(s), N, R) for s in ids]
    Ns = np.array([p["N"] for p in parts], dtype=np.int64)
    Rs = np.array([p["R"] for p in parts], dtype=np.int64)
    agent_off = np.concatenate([[0], np.cumsum(Ns)]).astype(np.int32)
    rg_off = np.concatenate([[0], np.cumsum(Rs)]).astype(np.int32)
    cat = lambda k, dt: np.concatenate([p[k] for p in parts]).astype(dt)
    n_route = np.concatenate([p["n_route"] for p in parts])
    route_off = np.concatenate([[0], np.cumsum(n_route)]).astype(np.int32)
    x, y, th = cat("x", np.float32), cat("y", np.float32), cat("th", np.float32)
    vx, vy = cat("vx", np.float32), cat("vy", np.float32)
    ctl = np.concatenate([p["ctl"] for p in parts], axis=1)
    log_x, log_y, log_th, log_vx, log_vy = _integrate_logs(ctl, x, y, th,
                                                           np.hypot(vx.astype(np.float64), vy.astype(np.float64)))
    log_vx[: T0 + 1], log_vy[: T0 + 1] = vx, vy  # the history rows hold the start state exactly
    # route paths of each scene's ego (its first agent)
    px, py, pon, ppt, poff = [], [], [], [0], [0]
    for j, part in enumerate(parts):
        a = int(agent_off[j])
        if part["N"] == 0:
            poff.append(poff[-1])
            continue
        paths, on = _route_paths(log_x[T0:, a].astype(np.float64), log_y[T0:, a].astype(np.float64),
                                 float(th[a]), part["branch"])
        for q in paths:
            px.append(q[:, 0])
            py.append(q[:, 1])
            ppt.append(ppt[-1] + len(q))
        pon.append(on)
        poff.append(poff[-1] + len(paths))
    return SceneBatch(
        cfg=cfg, seed=seed, scenes=ids, S=len(ids), N_tot=int(Ns.sum()), T=wl.T,
        agent_off=agent_off, rg_off=rg_off,
        L=cat("L", np.float32), W=cat("W", np.float32), valid=cat("valid", np.uint8),
        kind=cat("kind", np.uint8), idm_v0=cat("v0", np.float32),
        route_off=route_off,
        route_x=np.concatenate([p["rx"] for p in parts]).astype(np.float32),
        route_y=np.concatenate([p["ry"] for p in parts]).astype(np.float32),
        rg_x=np.concatenate([p["rg"][0] for p in parts]),
        rg_y=np.concatenate([p["rg"][1] for p in parts]),
        rg_poly=np.concatenate([p["rg"][2] for p in parts]),
        rg_type=np.concatenate([p["rg"][3] for p in parts]),
        rg_valid=np.concatenate([p["rg"][4] for p in parts]),
        log_x=log_x, log_y=log_y, log_th=log_th, log_vx=log_vx, log_vy=log_vy, x=x, y=y, th=th, vx=vx, vy=vy,
        actions=np.ascontiguousarray(np.concatenate([p["act"] for p in parts], axis=2)),
        path_off=np.array(poff, np.int32), path_pt_off=np.array(ppt, np.int32),
        path_x=(np.concatenate(px) if px else np.zeros(0)).astype(np.float32),
        path_y=(np.concatenate(py) if py else np.zeros(0)).astype(np.float32),
        path_on=(np.concatenate(pon) if pon else np.zeros(0)).astype(np.uint8),
    )


def concat(batches: Sequence[SceneBatch]) -> SceneBatch:
    """One batch holding the scenes of `batches` in order (CSR offsets rebased)."""
    b0 = batches[0]

    def offs(name, base_of):
        out, base = [np.zeros(1, np.int64)], 0
        for b in batches:
            o = getattr(b, name).astype(np.int64)
            out.append(o[1:] + base)
            base += base_of(b)
        return np.concatenate(out).astype(np.int32)

    cat = lambda name, axis=0: np.concatenate([getattr(b, name) for b in batches], axis=axis)
    return SceneBatch(
        cfg=b0.cfg, seed=b0.seed, scenes=cat("scenes"), S=sum(b.S for b in batches),
        N_tot=sum(b.N_tot for b in batches), T=b0.T,
        agent_off=offs("agent_off", lambda b: b.N_tot), rg_off=offs("rg_off", lambda b: len(b.rg_x)),
        L=cat("L"), W=cat("W"), valid=cat("valid"), kind=cat("kind"), idm_v0=cat("idm_v0"),
        route_off=offs("route_off", lambda b: len(b.route_x)), route_x=cat("route_x"), route_y=cat("route_y"),
        rg_x=cat("rg_x"), rg_y=cat("rg_y"), rg_poly=cat("rg_poly"), rg_type=cat("rg_type"),
        rg_valid=cat("rg_valid"),
        log_x=cat("log_x", 1), log_y=cat("log_y", 1), log_th=cat("log_th", 1), log_vx=cat("log_vx", 1),
        log_vy=cat("log_vy", 1), x=cat("x"), y=cat("y"), th=cat("th"), vx=cat("vx"), vy=cat("vy"),
        actions=np.ascontiguousarray(cat("actions", 2)),
        path_off=offs("path_off", lambda b: len(b.path_on)),
        path_pt_off=offs("path_pt_off", lambda b: len(b.path_x)),
        path_x=cat("path_x"), path_y=cat("path_y"), path_on=cat("path_on"),
    )
