"""Pins of the oracle's dynamics (App. A.1) against closed forms and invariants.

None of these re-evaluates the oracle's update equations: the expected values
are analytic trajectories of the discrete schemes (a telescoping sum for
straight driving, the arithmetic-progression cosine sum for constant
curvature), rigid-motion equivariance, and the delta model's exact replay of
another trajectory's displacements.
"""
import numpy as np
import pytest

import oracle
from tests.scenes import tiny_batch

DT = 0.1


def _run(o, st, act, n):
    """n transitions with the same action [3][N]; returns the list of states."""
    out = [st]
    for _ in range(n):
        st, _, _ = o.transition(st, act)
        out.append(st)
    return out


def _state(b):
    st = oracle.Oracle(b).initial_state()
    return st


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bicycle_straight_line_closed_form(seed):
    # kappa = 0, constant a, v0 + a t >= 0: x_n = x0 + cos(th)(v0 t + a t^2 / 2).
    rng = np.random.default_rng(seed)
    N = 16
    th = rng.uniform(-np.pi, np.pi, N)
    v0 = rng.uniform(0, 20, N)
    a = rng.uniform(-2, 4, N)
    a = np.where(v0 + a * 8.0 < 0, -v0 / 8.0, a)
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=th[i], v=v0[i]) for i in range(N)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    th64, v64 = st["th"], np.hypot(st["vx"], st["vy"])
    st["vx"], st["vy"] = v64 * np.cos(th64), v64 * np.sin(th64)  # velocity exactly along th
    a32 = a.astype(np.float32).astype(np.float64)
    act = np.zeros((3, N)); act[0] = a32
    traj = _run(o, st, act, 80)
    for n in (1, 7, 40, 80):
        t = n * DT
        ex = st["x"] + np.cos(th64) * (v64 * t + 0.5 * a32 * t * t)
        ey = st["y"] + np.sin(th64) * (v64 * t + 0.5 * a32 * t * t)
        np.testing.assert_allclose(traj[n]["x"], ex, atol=1e-9, rtol=0)
        np.testing.assert_allclose(traj[n]["y"], ey, atol=1e-9, rtol=0)
        np.testing.assert_allclose(np.hypot(traj[n]["vx"], traj[n]["vy"]), v64 + n * DT * a32, atol=1e-9)
        np.testing.assert_allclose(traj[n]["th"], th64, atol=0)


@pytest.mark.parametrize("seed", [0, 1])
def test_bicycle_constant_curvature_closed_form(seed):
    # a = 0, constant kappa: heading advances by phi = kappa v dt per step and
    # x_n = x0 + v dt sum_{k<n} cos(th0 + k phi) (arithmetic-progression sum).
    rng = np.random.default_rng(10 + seed)
    N = 12
    th0 = rng.uniform(-np.pi, np.pi, N)
    v = rng.uniform(1, 20, N)
    kap = rng.uniform(-0.3, 0.3, N)
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=th0[i], v=v[i]) for i in range(N)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    k32 = kap.astype(np.float32).astype(np.float64)
    act = np.zeros((3, N)); act[1] = k32
    traj = _run(o, st, act, 80)
    th = st["th"]
    sp = np.hypot(st["vx"], st["vy"])
    # The first step moves along the stored velocity; from then on along th_k.
    vx0, vy0 = st["vx"], st["vy"]
    phi = k32 * sp * DT
    for n in (1, 5, 33, 80):
        np.testing.assert_allclose(traj[n]["th"], th + n * phi, atol=1e-10)
        m = n - 1  # terms k = 1..n-1 of the cosine sum after the first step
        S_c = np.where(np.abs(phi) > 1e-12,
                       np.sin(m * phi / 2) / np.sin(phi / 2) * np.cos(th + phi + (m - 1) * phi / 2), m * np.cos(th))
        S_s = np.where(np.abs(phi) > 1e-12,
                       np.sin(m * phi / 2) / np.sin(phi / 2) * np.sin(th + phi + (m - 1) * phi / 2), m * np.sin(th))
        ex = st["x"] + vx0 * DT + sp * DT * S_c
        ey = st["y"] + vy0 * DT + sp * DT * S_s
        np.testing.assert_allclose(traj[n]["x"], ex, atol=1e-8)
        np.testing.assert_allclose(traj[n]["y"], ey, atol=1e-8)


def test_bicycle_negative_speed_not_clamped():
    # The forward equations have no clamp: braking past zero reverses along th'.
    b = tiny_batch([dict(x=10, y=5, th=0.3, v=0.2)])
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = np.zeros((3, 1)); act[0] = -4.0
    s1, _, _ = o.transition(st, act)
    v_exp = np.hypot(st["vx"], st["vy"])[0] - 0.4
    assert v_exp < 0
    assert np.isclose(s1["vx"][0], v_exp * np.cos(s1["th"][0]), atol=1e-12)
    assert np.isclose(s1["vy"][0], v_exp * np.sin(s1["th"][0]), atol=1e-12)


def test_bicycle_rigid_motion_equivariance():
    rng = np.random.default_rng(5)
    N = 10
    agents = [dict(x=rng.uniform(0, 50), y=rng.uniform(0, 50), th=rng.uniform(-3, 3), v=rng.uniform(0, 15))
              for _ in range(N)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    acts = [np.stack([rng.uniform(-4, 4, N), rng.uniform(-0.3, 0.3, N), np.zeros(N)]) for _ in range(20)]
    rot, tx, ty = 0.7, 13.0, -4.0
    c, s = np.cos(rot), np.sin(rot)
    st2 = dict(x=c * st["x"] - s * st["y"] + tx, y=s * st["x"] + c * st["y"] + ty, th=st["th"] + rot,
               vx=c * st["vx"] - s * st["vy"], vy=s * st["vx"] + c * st["vy"], s=st["s"].copy())
    a, b2 = st, st2
    for act in acts:
        a, _, _ = o.transition(a, act)
        b2, _, _ = o.transition(b2, act)
    np.testing.assert_allclose(b2["x"], c * a["x"] - s * a["y"] + tx, atol=1e-9)
    np.testing.assert_allclose(b2["y"], s * a["x"] + c * a["y"] + ty, atol=1e-9)
    np.testing.assert_allclose(b2["th"], a["th"] + rot, atol=1e-12)
    np.testing.assert_allclose(b2["vx"], c * a["vx"] - s * a["vy"], atol=1e-9)


def test_delta_replays_displacements_of_another_trajectory():
    # Delta agents fed the step displacements of a bicycle run land on its
    # positions and headings; their velocity is displacement / dt.
    rng = np.random.default_rng(7)
    N = 8
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=rng.uniform(-3, 3), v=rng.uniform(0, 20))
              for _ in range(N)]
    bb = tiny_batch(agents)
    ob = oracle.Oracle(bb)
    sb = ob.initial_state()
    traj = [sb]
    for _ in range(30):
        act = np.stack([rng.uniform(-4, 4, N), rng.uniform(-0.3, 0.3, N), np.zeros(N)])
        sb, _, _ = ob.transition(sb, act)
        traj.append(sb)
    bd = tiny_batch([dict(a, kind=1) for a in agents])
    od = oracle.Oracle(bd)
    sd = od.initial_state()
    for k in range(30):
        d = np.stack([traj[k + 1]["x"] - traj[k]["x"], traj[k + 1]["y"] - traj[k]["y"],
                      traj[k + 1]["th"] - traj[k]["th"]])
        sd, _, _ = od.transition(sd, d)
        np.testing.assert_allclose(sd["vx"], d[0] / DT, atol=1e-9)
        np.testing.assert_allclose(sd["vy"], d[1] / DT, atol=1e-9)
    np.testing.assert_allclose(sd["x"], traj[-1]["x"], atol=1e-9)
    np.testing.assert_allclose(sd["y"], traj[-1]["y"], atol=1e-9)
    np.testing.assert_allclose(sd["th"], traj[-1]["th"], atol=1e-12)


def test_delta_constant_displacement():
    b = tiny_batch([dict(x=1.0, y=2.0, th=0.5, kind=1)])
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = np.array([[0.3], [-0.2], [0.01]])
    traj = _run(o, st, act, 50)
    assert np.isclose(traj[50]["x"][0], 1.0 + 50 * 0.3, atol=1e-10)
    assert np.isclose(traj[50]["y"][0], 2.0 - 50 * 0.2, atol=1e-10)
    assert np.isclose(traj[50]["th"][0], np.float32(0.5) + 50 * 0.01, atol=1e-12)


def test_invalid_and_uncontrolled_agents_hold_state():
    agents = [dict(x=1, y=1, th=0.1, v=5), dict(x=9, y=3, th=1.0, v=7, valid=0), dict(x=20, y=3, th=2, v=3)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = np.ones((3, 3))
    ctrl = np.array([1, 1, 0], np.uint8)
    s1, _, _ = o.transition(st, act, ctrl=ctrl)
    for k in ("x", "y", "th", "vx", "vy"):
        assert s1[k][1] == st[k][1] and s1[k][2] == st[k][2]
        assert k in ("th",) or s1[k][0] != st[k][0]


@pytest.mark.parametrize("seed", [0, 1])
def test_bicycle_heading_change_is_curvature_times_distance(seed):
    # Constant a and kappa with speed kept >= 0: the scheme's steps telescope
    # to a distance v0 t + a t^2 / 2, and the heading turns by kappa times it.
    rng = np.random.default_rng(20 + seed)
    N = 10
    v0 = rng.uniform(2, 20, N)
    a = rng.uniform(-0.2, 3, N)
    kap = rng.uniform(-0.3, 0.3, N)
    agents = [dict(x=rng.uniform(0, 200), y=rng.uniform(0, 200), th=rng.uniform(-3, 3), v=v0[i]) for i in range(N)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    st = o.initial_state()
    sp = np.hypot(st["vx"], st["vy"])
    act = np.zeros((3, N)); act[0] = a.astype(np.float32); act[1] = kap.astype(np.float32)
    traj = _run(o, st, act, 40)
    for n in (1, 13, 40):
        t = n * DT
        dist = sp * t + 0.5 * act[0] * t * t
        np.testing.assert_allclose(traj[n]["th"] - st["th"], act[1] * dist, atol=1e-10)
        np.testing.assert_allclose(np.hypot(traj[n]["vx"], traj[n]["vy"]), sp + act[0] * t, atol=1e-10)
