"""Hand-built tiny scenes for the oracle pins (host arrays, SceneBatch layout)."""
import numpy as np

from paper_2310_08710_b300 import synth


def tiny_batch(agents, roadgraph=None, routes=None, T=1, log=None):
    """One scene.

    agents: list of dicts with x, y, th, v (or vx, vy), L, W and optional
            kind (default bicycle), valid (default 1), v0 (IDM desired speed).
    roadgraph: list of (points [n][2], type) polylines (type 1 = road edge).
    routes: {agent index: points [n][2]} for IDM agents.
    log: optional [T_log][N][2] logged positions (default: zeros).
    """
    N = len(agents)
    f32 = lambda v: np.asarray(v, dtype=np.float32)
    x = f32([a["x"] for a in agents])
    y = f32([a["y"] for a in agents])
    th = f32([a.get("th", 0.0) for a in agents])
    vx = f32([a.get("vx", a.get("v", 0.0) * np.cos(a.get("th", 0.0))) for a in agents])
    vy = f32([a.get("vy", a.get("v", 0.0) * np.sin(a.get("th", 0.0))) for a in agents])
    roadgraph = roadgraph or []
    gx, gy, gp, gt = [], [], [], []
    for pid, (pts, typ) in enumerate(roadgraph):
        pts = np.asarray(pts, dtype=np.float64)
        gx.append(pts[:, 0]); gy.append(pts[:, 1])
        gp.append(np.full(len(pts), pid)); gt.append(np.full(len(pts), typ))
    cat = lambda l, dt: np.concatenate(l).astype(dt) if l else np.zeros(0, dt)
    rg_x, rg_y, rg_poly, rg_type = cat(gx, np.float32), cat(gy, np.float32), cat(gp, np.int32), cat(gt, np.uint8)
    routes = routes or {}
    n_route = np.array([len(routes.get(i, [])) for i in range(N)], dtype=np.int64)
    rx = [np.asarray(routes[i], np.float64)[:, 0] for i in range(N) if i in routes]
    ry = [np.asarray(routes[i], np.float64)[:, 1] for i in range(N) if i in routes]
    T_log = synth.T_LOG
    if log is None:
        log = np.zeros((T_log, N, 2))
    log = np.asarray(log, dtype=np.float32)
    return synth.SceneBatch(
        cfg=-1, seed=0, scenes=np.array([0]), S=1, N_tot=N, T=T,
        agent_off=np.array([0, N], np.int32), rg_off=np.array([0, len(rg_x)], np.int32),
        L=f32([a.get("L", 4.5) for a in agents]), W=f32([a.get("W", 2.0) for a in agents]),
        valid=np.array([a.get("valid", 1) for a in agents], np.uint8),
        kind=np.array([a.get("kind", 0) for a in agents], np.uint8),
        idm_v0=f32([a.get("v0", 10.0) for a in agents]),
        route_off=np.concatenate([[0], np.cumsum(n_route)]).astype(np.int32),
        route_x=cat(rx, np.float32), route_y=cat(ry, np.float32),
        rg_x=rg_x, rg_y=rg_y, rg_poly=rg_poly, rg_type=rg_type, rg_valid=np.ones(len(rg_x), np.uint8),
        log_x=np.ascontiguousarray(log[:, :, 0]), log_y=np.ascontiguousarray(log[:, :, 1]),
        x=x, y=y, th=th, vx=vx, vy=vy, actions=np.zeros((T, 3, N), np.float32),
    )


def straight_route(x0, y0, th, n=320, h=0.5):
    k = np.arange(n)
    return np.stack([x0 + h * k * np.cos(th), y0 + h * k * np.sin(th)], 1)
