"""Expert actor, log playback and kinematic infeasibility on the GPU against
the FP64 oracle (needs a B300).

Teacher-forced parity of rollouts whose agents take every driver (hold,
action, expert, log playback), element-by-element parity of the open-loop
expert actions, the expert's replay of logs written by an action space's own
forward model (the oracle writes them), bit-identical launch paths, and the
error statuses of impossible requests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth
from tests.gpu_harness import run_rollout, teacher_forced

pytestmark = pytest.mark.gpu
T0 = synth.T0
HOLD, ACTION, EXPERT, LOG = 0, 1, 2, 3


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def mixed_batch(seed=0, S=6, N=40, R=3000):
    """Workload-0-like scenes with bicycle, delta and IDM agents."""
    b = synth.make_batch(4, seed=seed, S=S, N=N, R=R)  # delta ego in the first half, IDM others
    rng = np.random.default_rng(seed)
    pol = rng.random(b.N_tot) < 0.5
    kinds = b.kind.copy()
    kinds[pol & (kinds == synth.KIND_IDM)] = rng.choice([synth.KIND_BICYCLE, synth.KIND_DELTA],
                                                        int((pol & (kinds == synth.KIND_IDM)).sum()))
    b.kind = kinds
    bic = b.kind == synth.KIND_BICYCLE
    b.actions[:, 0, bic] = np.float32(rng.uniform(-4, 4, (b.T, int(bic.sum()))))
    b.actions[:, 1, bic] = np.float32(rng.uniform(-0.3, 0.3, (b.T, int(bic.sum()))))
    delta = b.kind == synth.KIND_DELTA
    # delta actions in the regime of one bicycle step of a 10 m/s car
    b.actions[:, 0, delta] = np.float32(rng.uniform(-1.2, 1.2, (b.T, int(delta.sum()))))
    b.actions[:, 1, delta] = np.float32(rng.uniform(-1.2, 1.2, (b.T, int(delta.sum()))))
    b.actions[:, 2, delta] = np.float32(rng.uniform(-0.05, 0.05, (b.T, int(delta.sum()))))
    return b


def test_teacher_forced_parity_all_drivers(wsim):
    b = mixed_batch()
    rng = np.random.default_rng(1)
    ctrl = rng.choice([HOLD, ACTION, EXPERT, LOG], b.N_tot, p=[0.1, 0.3, 0.4, 0.2]).astype(np.uint8)
    g = run_rollout(b, ctrl=ctrl)
    assert g["status"] == 0
    rep = {}
    teacher_forced(b, g, list(range(b.S)), range(b.T), report=rep, ctrl=ctrl)
    print("all drivers:", rep)
    assert rep["kin_flagged"] > 0  # random bicycle / delta actions break the limits now and then
    assert rep["band_kin"] <= 0.01 * rep["agent_steps"]
    # log playback lands on the log exactly
    lg = (ctrl == LOG) & b.valid.astype(bool)
    assert (g["logdiv"][:, lg] == 0).all()


@pytest.mark.parametrize("mode_name", ["GRAPH", "STREAM", "PLAIN"])
def test_drivers_bit_identical_across_launch_paths(wsim, mode_name):
    b = mixed_batch(seed=2, S=4, N=24, R=2000)
    rng = np.random.default_rng(2)
    ctrl = rng.choice([HOLD, ACTION, EXPERT, LOG], b.N_tot).astype(np.uint8)
    ref = run_rollout(b, ctrl=ctrl, T=20)
    got = run_rollout(b, ctrl=ctrl, T=20, mode=getattr(wsim, "MODE_" + mode_name))
    for k in ("traj", "ov", "off", "logdiv", "flags", "reward"):
        assert np.array_equal(np.asarray(ref[k]).view(np.uint8), np.asarray(got[k]).view(np.uint8)), k


def _kappa_tol(b, ex_o, T):
    """Per-element tolerance of the fitted curvature kappa = turn / distance:
    float32 resolves the turn to 2e-6 rad and the distance v dt + a dt^2/2 to
    3e-7 m (dt^2/2 times the error of a), so kappa to (2e-6 + |kappa| 3e-7)
    over the oracle's distance, plus 1e-6 relative."""
    v = np.hypot(b.log_vx[T0:T0 + T].astype(np.float64), b.log_vy[T0:T0 + T].astype(np.float64))
    dist = v * 0.1 + 0.5 * ex_o[:, 0] * 0.01
    k = np.abs(ex_o[:, 1])
    with np.errstate(divide="ignore"):
        return np.where(dist > 0, (2e-6 + 3e-7 * k) / dist, 0.0) + 1e-6 * k


def _a_tol(b, T):
    """Per-element tolerance of the fitted acceleration (|v'| - |v|) / dt:
    three float32 ulps of the larger speed over dt."""
    sp = lambda t0: np.hypot(b.log_vx[t0:t0 + T].astype(np.float64), b.log_vy[t0:t0 + T].astype(np.float64))
    vmax = np.maximum(sp(T0), sp(T0 + 1)).astype(np.float32)
    return 3 * np.spacing(vmax).astype(np.float64) / 0.1 + 1e-6


def test_expert_actions_parity(wsim):
    b = mixed_batch(seed=3, S=8, N=64, R=2000)
    T = b.T
    sim = wsim.Sim(wsim.DeviceBatch(b))
    got = sim.expert_actions(T0, T).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert sim.status() == 0
    sim.close()
    ex = oracle.Oracle(b).expert_actions(T0, T)
    bic = (b.kind == synth.KIND_BICYCLE) & b.valid.astype(bool)
    dl = (b.kind == synth.KIND_DELTA) & b.valid.astype(bool)
    rest = ~(bic | dl)
    assert (got[:, :, rest] == 0).all() and (got[:, 2, bic] == 0).all()
    assert (np.abs(got[:, 0, bic] - ex[:, 0, bic]) <= _a_tol(b, T)[:, bic]).all()
    assert (np.abs(got[:, 1, bic] - ex[:, 1, bic]) <= _kappa_tol(b, ex, T)[:, bic]).all()
    d = np.abs(got[:, :, dl] - ex[:, :, dl])
    assert (d <= 1e-7 + 4 * np.spacing(np.abs(ex[:, :, dl]).astype(np.float32))).all()
    print("expert actions: max |da| %.2e, max |dkappa| %.2e, max |ddelta| %.2e" % (
        np.abs(got[:, 0, bic] - ex[:, 0, bic]).max(), np.abs(got[:, 1, bic] - ex[:, 1, bic]).max(), d.max()))


def test_expert_turn_in_every_direction(wsim):
    # The expert's turn comes from a float32 atan2 of its own (octant
    # reduction and a fitted polynomial): logged velocities in every
    # direction, on the octant boundaries and next to them, +-0 components,
    # speeds from 1 cm/s to 100 m/s and standing still; headings zero, so
    # the turn is the direction itself.
    b = mixed_batch(seed=5, S=2, N=64, R=1000)
    b.kind = np.full_like(b.kind, synth.KIND_BICYCLE)
    b.valid = np.ones_like(b.valid)
    rng = np.random.default_rng(5)
    rows, n = synth.T_LOG, b.N_tot
    base = np.arange(-4, 5) * (np.pi / 4)
    ang = np.concatenate([base, base + 1e-6, base - 1e-6, rng.uniform(-np.pi, np.pi, 64)])
    phi = rng.choice(ang, (rows, n))
    spd = 10.0 ** rng.uniform(-2, 2, (rows, n))
    spd[rng.random((rows, n)) < 0.05] = 0.0
    vx = (spd * np.cos(phi)).astype(np.float32)
    vy = (spd * np.sin(phi)).astype(np.float32)
    # exact axes and diagonals with signed zeros
    ex = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1),
          (-1, -0.0), (1, -0.0), (0.0, 1), (-0.0, -1)]
    for j, (a, c) in enumerate(ex):
        vx[T0 + 1 + j, :] = np.float32(a) * np.float32(3.0)
        vy[T0 + 1 + j, :] = np.float32(c) * np.float32(3.0)
    b.log_vx, b.log_vy = vx, vy
    b.log_th = np.zeros((rows, n), np.float32)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    got = sim.expert_actions(T0, b.T).cpu().numpy().astype(np.float64)
    assert sim.status() == 0
    sim.close()
    exo = oracle.Oracle(b).expert_actions(T0, b.T)
    assert (np.abs(got[:, 0] - exo[:, 0]) <= _a_tol(b, b.T)).all()
    assert (np.abs(got[:, 1] - exo[:, 1]) <= _kappa_tol(b, exo, b.T)).all()
    # the exact directions: turn = kappa * dist within 4e-7 rad of atan2
    v0 = np.hypot(vx[T0:T0 + 12].astype(np.float64), vy[T0:T0 + 12].astype(np.float64))
    v1 = np.hypot(vx[T0 + 1:T0 + 13].astype(np.float64), vy[T0 + 1:T0 + 13].astype(np.float64))
    turn = got[:12, 1] * 0.1 * 0.5 * (v0 + v1)
    want = np.arctan2(vy[T0 + 1:T0 + 13].astype(np.float64), vx[T0 + 1:T0 + 13].astype(np.float64))
    assert np.abs(turn - want).max() <= 4e-7 + 1e-6 * np.abs(want).max(), np.abs(turn - want).max()


def test_expert_actions_full_size_sampled(wsim):
    # 1024 scenes x 128 agents x 80 steps in one launch; every policy agent's
    # fitted actions checked on 16 sampled scenes, the others must be zero.
    b = synth.make_batch(1, seed=0)
    pol = b.valid.astype(bool) & (b.kind != synth.KIND_IDM)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    got = sim.expert_actions(T0, b.T).cpu().numpy().astype(np.float64)
    sim.close()
    assert (got[:, :, ~pol] == 0).all()
    scenes = list(range(0, b.S, b.S // 16))
    sub = b.subset(scenes)
    ag = np.concatenate([np.arange(b.agent_off[s], b.agent_off[s + 1]) for s in scenes])
    ex = oracle.Oracle(sub).expert_actions(T0, b.T)
    g = got[:, :, ag]
    p = pol[ag]
    assert (np.abs(g[:, 0, p] - ex[:, 0, p]) <= _a_tol(sub, b.T)[:, p]).all()
    assert (np.abs(g[:, 1, p] - ex[:, 1, p]) <= _kappa_tol(sub, ex, b.T)[:, p]).all()


def _self_written_logs(kind, seed, N=32, T=40):
    """Logs written by the oracle's forward model of one action space."""
    rng = np.random.default_rng(seed)
    b = synth.make_batch(0, seed=seed, N=N, T=T)
    b.kind[:] = kind
    b.valid[:] = 1
    sp = rng.uniform(5, 20, N)  # no agent comes to a stop within T steps
    b.vx = (sp * np.cos(b.th.astype(np.float64))).astype(np.float32)
    b.vy = (sp * np.sin(b.th.astype(np.float64))).astype(np.float32)
    acts = np.zeros((T, 3, N))
    acts[:, 0] = rng.uniform(-2, 2, (T, N))
    if kind == synth.KIND_BICYCLE:
        acts[:, 1] = rng.uniform(-0.2, 0.2, (T, N))
    else:
        acts[:, 1] = rng.uniform(-1, 1, (T, N))
        acts[:, 0] = rng.uniform(-1, 1, (T, N))
        acts[:, 2] = rng.uniform(-0.05, 0.05, (T, N))
    o = oracle.Oracle(b)
    st = o.initial_state()
    keys = ("x", "y", "th", "vx", "vy")
    logs = {k: np.repeat(st[k][None], synth.T_LOG, 0) for k in keys}
    for k in range(T):
        st, _, _ = o.transition(st, acts[k])
        for key in keys:
            logs[key][T0 + k + 1:] = st[key]
    b.log_x, b.log_y = logs["x"].astype(np.float32), logs["y"].astype(np.float32)
    b.log_th, b.log_vx, b.log_vy = (logs[k].astype(np.float32) for k in ("th", "vx", "vy"))
    return b


@pytest.mark.parametrize("kind", [synth.KIND_BICYCLE, synth.KIND_DELTA])
def test_expert_rollout_replays_self_written_logs(wsim, kind):
    # Sec. 5.2 expert ADE: on logs made by the agents' own action space the
    # closed-loop expert stays on the log to float32 rounding; no actions
    # are passed at all.
    b = _self_written_logs(kind, seed=5 + kind)
    g = run_rollout(b, ctrl=np.full(b.N_tot, EXPERT, np.uint8), no_actions=True)
    assert g["status"] == 0
    assert g["logdiv"].max() <= 5e-5, g["logdiv"].max()
    if kind == synth.KIND_BICYCLE:  # the fitted actions are inside the limits
        assert not (g["flags"] & 4).any()


def test_delta_expert_on_generator_logs_and_bicycle_expert_drift(wsim):
    b = synth.make_batch(0, seed=3)
    v = b.valid.astype(bool)
    ctrl = np.full(b.N_tot, EXPERT, np.uint8)
    b.kind[:] = synth.KIND_DELTA
    gd = run_rollout(b, ctrl=ctrl, no_actions=True)
    assert gd["logdiv"][:, v].max() <= 1e-5
    b.kind[:] = synth.KIND_BICYCLE
    gb = run_rollout(b, ctrl=ctrl, no_actions=True)
    o = oracle.Oracle(b)
    _, mo = o.rollout(o.initial_state(), None, T0, b.T, ctrl=ctrl)
    # free-running bicycle expert drift against the log, GPU and oracle alike
    ade_g = gb["logdiv"][:, v].mean(axis=0)
    ade_o = mo["logdiv"][:, v].mean(axis=0)
    assert np.abs(ade_g - ade_o).max() <= 1e-3, np.abs(ade_g - ade_o).max()
    rep = {}
    teacher_forced(b, gb, [0], range(b.T), report=rep, ctrl=ctrl)


def test_bad_driver_requests_set_status(wsim):
    b = synth.make_batch(0, seed=4, T=4)
    g = run_rollout(b, ctrl=np.full(b.N_tot, 7, np.uint8))  # no such driver
    assert g["status"] == wsim.EINVAL
    v = b.valid.astype(bool)
    assert np.array_equal(g["final"][0][v], b.x[v])  # held
    g = run_rollout(b, ctrl=np.full(b.N_tot, ACTION, np.uint8), no_actions=True)  # actions asked, none given
    assert g["status"] == wsim.EINVAL
    b.log_th = b.log_vx = b.log_vy = None  # no heading / velocity logs
    db = wsim.DeviceBatch(b)
    sim = wsim.Sim(db)
    with pytest.raises(wsim.WsimError):
        sim.expert_actions(T0, 4)
    st = wsim.State.from_batch(b)
    m = wsim.Metrics(b.N_tot, b.S, rows=4)
    sim.rollout(st, None, m, T0, 4, mode=wsim.MODE_FUSED,
                ctrl=torch.full((b.N_tot,), EXPERT, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    assert sim.status() == wsim.EINVAL
    sim.close()
