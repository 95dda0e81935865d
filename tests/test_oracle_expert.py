"""Pins of the oracle's inverse dynamics, expert actor, log playback and
kinematic-infeasibility metric (App. A.1 inverse kinematics, Sec. 3.4, Sec. 5.2).

Expected values come from hand-built states with a known motion (straight
driving with a known speed change, driving on a circle of known radius,
headings in every quadrant), from the forward dynamics (themselves pinned
against closed forms in test_oracle_dynamics.py) and from logs the test
writes itself, never from re-evaluating the inverse's own formulas.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch

DT = 0.1
EXPERT, LOG = oracle.CTRL_EXPERT, oracle.CTRL_LOG


def _st(x, y, th, vx, vy):
    n = len(x)
    return dict(x=np.asarray(x, float), y=np.asarray(y, float), th=np.asarray(th, float),
                vx=np.asarray(vx, float), vy=np.asarray(vy, float), s=np.zeros(n))


def _batch(n, kind=0):
    return tiny_batch([dict(x=0.0, y=0.0, kind=kind) for _ in range(n)])


def test_inverse_straight_line_and_circle_closed_forms():
    # Straight: heading th, speed v -> v + a dt along th: the inverse gives a
    # and zero curvature, in every quadrant.
    th = np.array([0.3, 2.0, -2.5, -1.0, 3.1])
    v = np.array([5.0, 12.0, 0.5, 20.0, 8.0])
    a = np.array([1.5, -3.0, 2.0, 0.0, -5.5])
    vn = v + a * DT
    o = oracle.Oracle(_batch(5))
    s0 = _st(np.zeros(5), np.zeros(5), th, v * np.cos(th), v * np.sin(th))
    s1 = _st(np.zeros(5), np.zeros(5), th, vn * np.cos(th), vn * np.sin(th))
    u = o.inverse(s0, s1)
    np.testing.assert_allclose(u[0], a, atol=1e-12)
    np.testing.assert_allclose(u[1], 0.0, atol=1e-12)
    # Circle of radius R at constant speed: the direction turns by v dt / R
    # over the distance v dt, so kappa = +-1/R, whatever the starting heading
    # (third-quadrant headings catch a lost quadrant in the direction).
    R = np.array([10.0, 25.0, 50.0, 200.0, 3.4])
    turn = np.array([1, -1, 1, -1, 1]) * v * DT / R
    thn = th + turn
    s2 = _st(np.zeros(5), np.zeros(5), thn, v * np.cos(thn), v * np.sin(thn))
    u = o.inverse(s0, s2)
    np.testing.assert_allclose(u[0], 0.0, atol=1e-11)
    np.testing.assert_allclose(u[1], np.sign(turn) / R, rtol=1e-12)


def test_inverse_of_unwrapped_heading_and_stopped_agent():
    o = oracle.Oracle(_batch(3))
    # Heading carried unwrapped at 4 pi + 0.2; the new velocity points at
    # 0.2 + 0.01: the turn is 0.01, not 0.01 - 4 pi.
    th = np.array([4 * np.pi + 0.2, -6 * np.pi - 1.0, 0.7])
    v = np.array([10.0, 10.0, 3.0])
    s0 = _st(np.zeros(3), np.zeros(3), th, v * np.cos(th), v * np.sin(th))
    d = np.array([0.01, -0.02, 0.0])
    vn = np.array([10.0, 10.0, 0.0])  # the third agent stops: no direction, no turn
    s1 = _st(np.zeros(3), np.zeros(3), th + d, vn * np.cos(th + d), vn * np.sin(th + d))
    u = o.inverse(s0, s1)
    np.testing.assert_allclose(u[1, :2], d[:2] / (v[:2] * DT), rtol=1e-9)
    assert u[0, 2] == pytest.approx(-30.0) and u[1, 2] == 0.0
    # No motion at all: zero distance, kappa = 0.
    z = _st(np.zeros(3), np.zeros(3), th, np.zeros(3), np.zeros(3))
    assert (o.inverse(z, z) == 0).all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bicycle_inverse_of_forward_is_identity(seed):
    # Random states (headings anywhere, unwrapped up to +-20 rad) and actions
    # inside the policy range, stepped by the forward model: the inverse
    # recovers (a, kappa) wherever the new speed stays positive.
    rng = np.random.default_rng(seed)
    N = 64
    th = rng.uniform(-20, 20, N)
    v = rng.uniform(0.5, 25, N)
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=th[i], v=v[i]) for i in range(N)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = np.zeros((3, N))
    act[0] = rng.uniform(-4, 4, N)
    act[1] = rng.uniform(-0.3, 0.3, N)
    nx, _, _ = o.transition(st, act)
    u = o.inverse(st, nx)
    ok = np.hypot(st["vx"], st["vy"]) + act[0] * DT > 0
    assert ok.sum() > N // 2
    np.testing.assert_allclose(u[0][ok], act[0][ok], atol=1e-9)
    np.testing.assert_allclose(u[1][ok], act[1][ok], atol=1e-9)
    assert (u[2] == 0).all()


def test_delta_inverse_replays_displacements():
    rng = np.random.default_rng(4)
    N = 16
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=rng.uniform(-3, 3), v=5.0, kind=1)
              for _ in range(N)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = rng.uniform(-2, 2, (3, N))
    nx, _, _ = o.transition(st, act)
    u = o.inverse(st, nx)
    np.testing.assert_allclose(u, act, atol=1e-12)


def _bicycle_log_batch(seed, N=12, T=30, kind=0):
    """A batch whose logs are a forward-model rollout of random actions
    (bicycle: kind 0, delta: kind 1), written by this test from
    oracle.transition; returns (batch, actions [T][3][N])."""
    rng = np.random.default_rng(seed)
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=rng.uniform(-3, 3),
                   v=rng.uniform(6, 20), kind=kind) for _ in range(N)]
    b = tiny_batch(agents, T=T)
    o = oracle.Oracle(b)
    st = o.initial_state()
    acts = np.zeros((T, 3, N))
    acts[:, 0] = rng.uniform(-2, 2, (T, N))
    acts[:, 1] = rng.uniform(-0.2, 0.2, (T, N)) if kind == 0 else rng.uniform(-2, 2, (T, N))
    if kind == 1:
        acts[:, 2] = rng.uniform(-0.1, 0.1, (T, N))
    logs = {k: np.zeros((synth.T_LOG, N)) for k in ("x", "y", "th", "vx", "vy")}
    for t in range(synth.T0 + 1):
        for k in logs:
            logs[k][t] = st[k]
    for k in range(T):
        st, _, _ = o.transition(st, acts[k])
        for key in logs:
            logs[key][synth.T0 + k + 1] = st[key]
    for t in range(synth.T0 + T + 1, synth.T_LOG):
        for key in logs:
            logs[key][t] = logs[key][synth.T0 + T]
    # float32 storage, as every batch array; the start state stays exact
    b.log_x, b.log_y = logs["x"].astype(np.float32), logs["y"].astype(np.float32)
    b.log_th, b.log_vx, b.log_vy = (logs[k].astype(np.float32) for k in ("th", "vx", "vy"))
    return b, acts


@pytest.mark.parametrize("kind", [0, 1])
def test_expert_reproduces_logs_written_by_its_own_action_space(kind):
    # Sec. 5.2 expert: on logs made by an action space's forward model, the
    # open-loop fitted actions are the actions that made them (to the log's
    # float32 rounding), and the closed-loop expert rollout follows the log
    # (log divergence at the float32 rounding of the logged positions).
    b, acts = _bicycle_log_batch(7 + kind, kind=kind)
    o = oracle.Oracle(b)
    T = acts.shape[0]
    ex = o.expert_actions(synth.T0, T)
    # float32 log rounding: speeds ~20 m/s (ulp 2e-6) differenced over 0.1 s,
    # positions ~300 m (ulp 3e-5), headings ~3 rad (ulp 2.4e-7)
    tol = [5e-5, 1e-6, 0.0] if kind == 0 else [5e-5, 5e-5, 1e-6]
    for c in range(3):
        np.testing.assert_allclose(ex[:, c], acts[:, c], atol=tol[c])
    ctrl = np.full(b.N_tot, EXPERT, np.uint8)
    _, m = o.rollout(o.initial_state(), None, synth.T0, T, ctrl=ctrl)
    assert m["logdiv"].max() < 3e-5, m["logdiv"].max()
    if kind == 1:  # delta: the positions are the log's, to rounding
        assert m["logdiv"].max() < 1e-9


def test_delta_expert_ade_zero_and_bicycle_expert_close_on_generator_logs():
    # The generator's logs come from its own continuous-time integrator (not
    # from either action space).  The delta expert still lands on every
    # logged position (Sec. 5.2 table: delta expert ADE 0.00); the bicycle
    # expert only fits speed and direction, so it drifts, but stays close.
    b = synth.make_batch(0, seed=3)
    o = oracle.Oracle(b)
    v = b.valid.astype(bool)
    ctrl = np.full(b.N_tot, EXPERT, np.uint8)
    b.kind[:] = synth.KIND_DELTA
    _, md = oracle.Oracle(b).rollout(o.initial_state(), None, synth.T0, b.T, ctrl=ctrl)
    assert md["logdiv"][:, v].max() < 1e-9
    b.kind[:] = synth.KIND_BICYCLE
    _, mb = oracle.Oracle(b).rollout(o.initial_state(), None, synth.T0, b.T, ctrl=ctrl)
    ade = mb["logdiv"][:, v].mean(axis=0)
    assert 0 < ade.max() < 2.0, ade.max()
    # The logs' controls stay far inside the limits (|a| <= 2, |kappa| <= 0.05),
    # so the fitted transitions are feasible, except where a stopped agent
    # starts again: the direction then has to turn over almost no distance.
    kin = (mb["flags"][:, v] & 16) != 0
    assert kin.mean() < 0.01, kin.mean()


def test_log_playback_and_ctrl_values():
    b, _ = _bicycle_log_batch(11, N=6, T=5)
    b.kind[4] = synth.KIND_IDM  # an IDM agent without a route may still replay the log
    o = oracle.Oracle(b)
    st = o.initial_state()
    ctrl = np.array([LOG, LOG, oracle.CTRL_HOLD, oracle.CTRL_ACTION, LOG, EXPERT], np.uint8)
    act = np.zeros((3, b.N_tot))
    nx, _, _ = o.transition(st, act, ctrl=ctrl, t_next=synth.T0 + 1)
    t1 = synth.T0 + 1
    for g in (0, 1, 4):
        assert nx["x"][g] == np.float64(b.log_x[t1, g]) and nx["th"][g] == np.float64(b.log_th[t1, g])
        assert nx["vx"][g] == np.float64(b.log_vx[t1, g])
    assert nx["x"][2] == st["x"][2] and nx["vx"][2] == st["vx"][2]
    m = o.metrics(nx, t1, prev=st)
    assert (m["logdiv"][[0, 1, 4]] == 0).all()
    with pytest.raises(RuntimeError):  # expert and playback need the log row
        o.transition(st, act, ctrl=ctrl)
    with pytest.raises(RuntimeError):  # ctrl values above 4 are rejected
        o.transition(st, act, ctrl=np.full(b.N_tot, 5, np.uint8), t_next=t1)


def _kin_flags(o, s0, s1):
    m = o.metrics(s1, synth.T0, prev=s0)
    return m["flags"]


def test_kinematic_infeasibility_limits():
    # Sec. 3.4: infeasible iff the inverse kinematics give |a| > 6 m/s^2 or
    # |kappa| > 0.3 1/m.  Hand-built transitions on both sides of each limit.
    th = 1.9
    v = 10.0
    cases = [  # (speed change, turn, expected flag)
        (0.65, 0.0, True), (-0.65, 0.0, True), (0.55, 0.0, False), (-0.55, 0.0, False),
        (0.0, 0.31 * v * DT, True), (0.0, -0.31 * v * DT, True), (0.0, 0.29 * v * DT, False),
        (0.0, 0.0, False),
    ]
    n = len(cases)
    o = oracle.Oracle(_batch(n))
    dv = np.array([c[0] for c in cases])
    tn = th + np.array([c[1] for c in cases])
    # distance travelled v dt + a dt^2/2 with a = dv/dt: for the turn cases dv = 0
    s0 = _st(np.zeros(n), np.zeros(n), np.full(n, th), np.full(n, v * np.cos(th)), np.full(n, v * np.sin(th)))
    s1 = _st(np.zeros(n), np.zeros(n), tn, (v + dv) * np.cos(tn), (v + dv) * np.sin(tn))
    f = _kin_flags(o, s0, s1)
    assert [bool(x & 16) for x in f] == [c[2] for c in cases]
    assert not (f & 32).any()
    # at the limit itself: inside the band
    s1b = _st(np.zeros(n), np.zeros(n), np.full(n, th), np.full(n, (v + 0.6) * np.cos(th)),
              np.full(n, (v + 0.6) * np.sin(th)))
    assert (_kin_flags(o, s0, s1b) & 32).all()
    tl = th + 0.3 * v * DT  # turn at the curvature limit over the distance v dt
    s1c = _st(np.zeros(n), np.zeros(n), np.full(n, tl), np.full(n, v * np.cos(tl)), np.full(n, v * np.sin(tl)))
    assert (_kin_flags(o, s0, s1c) & 32).all()
    # a stopped agent that stays stopped: no direction, exactly feasible, no band
    z = _st(np.zeros(n), np.zeros(n), np.full(n, th), np.zeros(n), np.zeros(n))
    assert (_kin_flags(o, z, z) & 48 == 0).all()


def test_reverse_motion_reads_as_infeasible():
    # Reading: the bicycle model has no speed clamp; a speed that crosses
    # zero flips the velocity, so the direction turns by pi and the step is
    # kinematically infeasible (and the fitted |a| is not the applied one).
    b = tiny_batch([dict(x=0.0, y=0.0, th=0.4, v=0.2)])
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = np.array([[-4.0], [0.0], [0.0]])
    nx, _, _ = o.transition(st, act)
    assert np.hypot(nx["vx"], nx["vy"])[0] == pytest.approx(0.2)
    assert _kin_flags(o, st, nx)[0] & 16


def test_rollout_flags_infeasible_policy_actions():
    # A rollout whose actions break the limits is flagged at those steps only.
    b = tiny_batch([dict(x=0.0, y=0.0, th=0.0, v=15.0), dict(x=50.0, y=50.0, th=1.0, v=15.0)], T=6)
    o = oracle.Oracle(b)
    acts = np.zeros((6, 3, 2))
    acts[2, 0, 0] = 7.0     # |a| > 6 at step 2 for agent 0
    acts[4, 1, 1] = 0.35    # |kappa| > 0.3 at step 4 for agent 1
    acts[1, 0, 1] = 5.0     # inside both limits
    _, m = o.rollout(o.initial_state(), acts, synth.T0, 6)
    got = (m["flags"] & 16) != 0
    want = np.zeros((6, 2), bool)
    want[2, 0] = want[4, 1] = True
    np.testing.assert_array_equal(got, want)
