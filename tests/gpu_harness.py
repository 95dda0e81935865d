"""Runs the CUDA path through the C ABI and compares it with the oracle.

Teacher-forced parity: for every checked step the oracle starts from the
GPU's own float32 state at t (hi + lo pairs summed exactly in float64),
computes t+1 and the metrics of the GPU's t+1 state, and the two are compared
per quantity.  Decisions inside the oracle's ambiguity bands (IDM lead
search, collision / off-road booleans) are excluded from the exact checks and
counted.
"""
import numpy as np
import torch

import oracle
from paper_2310_08710_b300 import synth

# Tolerances (float32 kernels against the float64 oracle).
TOL_POS = 1e-5      # m, positions per step
TOL_TH = 1e-6       # rad, heading
TOL_V = 1e-5        # m/s, velocity components
TOL_S = 1e-5        # m, IDM route parameter
TOL_LOGDIV = 1e-5   # m
TOL_DEPTH = 2e-5    # m, overlap depth and off-road distance
ULP_SLACK = 4       # float32 ulps of the value for large magnitudes


def run_rollout(b, mode=None, T=None, ctrl=None, cfg=None, tuning=None, no_actions=False, count=False):
    from paper_2310_08710_b300 import wsim
    mode = wsim.MODE_FUSED if mode is None else mode
    T = b.T if T is None else T
    db = wsim.DeviceBatch(b)
    sim = wsim.Sim(db, cfg)
    if tuning is not None:
        sim.set_tuning(**tuning)
    st = wsim.State.from_batch(b)
    act = None if no_actions else torch.as_tensor(b.actions[:T]).cuda().contiguous()
    traj = wsim.State(b.N_tot, rows=T)
    m = wsim.Metrics(b.N_tot, b.S, rows=T)
    ct = None if ctrl is None else torch.as_tensor(ctrl, dtype=torch.uint8).cuda()
    if count:
        sim.set_counting(True)
    sim.rollout(st, act, m, synth.T0, T, mode=mode, traj=traj, ctrl=ct)
    torch.cuda.synchronize()
    status = sim.status()
    counters = sim.counters() if count else None
    out = dict(
        traj=traj.data.cpu().numpy().reshape(10, T, b.N_tot),
        final=st.data.cpu().numpy(),
        ov=m.ov.cpu().numpy(), off=m.off.cpu().numpy(), logdiv=m.logdiv.cpu().numpy(),
        flags=m.flags.cpu().numpy(), reward=m.reward.cpu().numpy(), status=status, counters=counters,
    )
    sim.close()
    return out


def state64(rows, ag):
    """float64 state dict from a [10, N] float32 block (hi + lo exactly)."""
    f = lambda i: rows[i][ag].astype(np.float64)
    return dict(x=f(0) + f(2), y=f(1) + f(3), th=f(4) + f(5), vx=f(6), vy=f(7), s=f(8) + f(9))


def initial_rows(b):
    r = np.zeros((10, b.N_tot), np.float32)
    r[0], r[1], r[4], r[6], r[7] = b.x, b.y, b.th, b.vx, b.vy
    return r


def _ulp_tol(base, v):
    v = np.where(np.isfinite(v), np.abs(v), 0.0)
    return np.maximum(base, ULP_SLACK * np.spacing(v.astype(np.float32)).astype(np.float64))


def teacher_forced(b, gpu, scene_idx, steps, report=None, ctrl=None):
    """Checks the given steps of the given scenes; returns counters.  ctrl:
    the per-agent driver array the GPU rollout ran with (None: all actions)."""
    sub = b.subset(scene_idx)
    o = oracle.Oracle(sub)
    ag = np.concatenate([np.arange(b.agent_off[s], b.agent_off[s + 1]) for s in scene_idx]).astype(np.int64)
    valid = sub.valid.astype(bool)
    sub_ctrl = None if ctrl is None else np.ascontiguousarray(np.asarray(ctrl, np.uint8)[ag])
    c = dict(steps=0, agent_steps=0, band_idm=0, band_ov=0, band_off=0, band_kin=0, kin_flagged=0, max_pos=0.0,
             max_th=0.0, max_v=0.0, max_s=0.0, max_ov=0.0, max_off=0.0, max_logdiv=0.0, reward_checked=0)
    traj = gpu["traj"]
    for k in steps:
        prev = initial_rows(b) if k == 0 else traj[:, k - 1, :]
        st_t = state64(prev, ag)
        exp, band, _ = o.transition(st_t, sub.actions[k], ctrl=sub_ctrl, t_next=synth.T0 + k + 1)
        got = state64(traj[:, k, :], ag)
        keep = ~band.astype(bool)
        c["band_idm"] += int(band.sum())
        dpos = np.maximum(np.abs(got["x"] - exp["x"]), np.abs(got["y"] - exp["y"]))[keep]
        dth = np.abs(np.angle(np.exp(1j * (got["th"] - exp["th"]))))[keep]
        dv = np.maximum(np.abs(got["vx"] - exp["vx"]), np.abs(got["vy"] - exp["vy"]))[keep]
        ds = np.abs(got["s"] - exp["s"])[keep]
        assert dpos.max(initial=0) <= TOL_POS, ("position", k, dpos.max())
        assert dth.max(initial=0) <= TOL_TH, ("heading", k, dth.max())
        assert dv.max(initial=0) <= TOL_V, ("velocity", k, dv.max())
        assert ds.max(initial=0) <= TOL_S, ("route s", k, ds.max())
        c["max_pos"] = max(c["max_pos"], float(dpos.max(initial=0)))
        c["max_th"] = max(c["max_th"], float(dth.max(initial=0)))
        c["max_v"] = max(c["max_v"], float(dv.max(initial=0)))
        c["max_s"] = max(c["max_s"], float(ds.max(initial=0)))
        # Metrics of the GPU's own t+1 state.
        t = synth.T0 + k + 1
        me = o.metrics(got, t, prev=st_t)
        for key, tol, mk in (("ov", TOL_DEPTH, "max_ov"), ("off", TOL_DEPTH, "max_off"),
                             ("logdiv", TOL_LOGDIV, "max_logdiv")):
            gv = gpu[key][k][ag].astype(np.float64)
            ev = me[key]
            fin = np.isfinite(ev)
            assert np.array_equal(np.isfinite(gv), fin), (key, k)
            assert np.array_equal(gv[~fin], ev[~fin]), (key, k)
            d = np.abs(gv[fin] - ev[fin])
            bound = _ulp_tol(tol, ev[fin])
            assert (d <= bound).all(), (key, k, float((d - bound).max()))
            c[mk] = max(c[mk], float(d.max(initial=0)))
        gf = gpu["flags"][k][ag]
        ef = me["flags"]
        b_ov = (ef & 4) != 0
        b_off = (ef & 8) != 0
        assert np.array_equal((gf & 1)[~b_ov], (ef & 1)[~b_ov]), ("collision flag", k)
        assert np.array_equal((gf & 2)[~b_off], (ef & 2)[~b_off]), ("offroad flag", k)
        b_kin = (ef & 32) != 0
        assert np.array_equal(((gf & 4) != 0)[~b_kin], ((ef & 16) != 0)[~b_kin]), ("kinematic flag", k)
        c["band_ov"] += int((b_ov & valid).sum())
        c["band_off"] += int((b_off & valid).sum())
        c["band_kin"] += int((b_kin & valid).sum())
        c["kin_flagged"] += int(((gf & 4) != 0).sum())
        for j, s in enumerate(scene_idx):
            a0, a1 = sub.agent_off[j], sub.agent_off[j + 1]
            if not (ef[a0:a1] & 12).any():
                assert gpu["reward"][k][s] == me["reward"][j], ("reward", k, s)
                c["reward_checked"] += 1
        c["steps"] += 1
        c["agent_steps"] += int(valid.sum())
    if report is not None:
        report.update(c)
    return c
