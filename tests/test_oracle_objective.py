"""Pins of the oracle's differentiable objective and its dual-number gradient.

The objective weighs the smooth BPTT loss and the per-step metrics of a
rollout (log divergence, overlap depth, off-road distance: Sec. 3.4); its
gradient with respect to the actions and the initial state is what the
differentiable rollout returns (the differentiable simulation of Sec. 6).
Pins: the objective's values against the oracle's own metrics and loss,
closed forms of its derivative on trajectories known analytically (straight
driving beside a straight road edge, two boxes overlapping along one axis,
the distance to fixed logged points), and central finite differences in
FP64 for random weights on random scenes.  The step is h = 1e-5: the metric
terms (distances that can be short, corners whose nearest point sits near a
segment end) curve enough that h = 1e-3 leaves a truncation error of 1e-5
relative, while at 1e-5 both truncation and rounding stay below 1e-7.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch

H = 1e-5
DT = 0.1


def _straight(x0, y0, th, v):
    return dict(x=x0, y=y0, th=th, vx=v * np.cos(th), vy=v * np.sin(th))


def _state(agents):
    keys = ("x", "y", "th", "vx", "vy")
    st = {k: np.array([a[k] for a in agents], dtype=np.float64) for k in keys}
    st["s"] = np.zeros(len(agents))
    return st


def test_objective_values_are_the_weighted_metrics_and_loss():
    b = synth.make_batch(3, seed=3, scenes=range(2), N=8, T=12)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    rng = np.random.default_rng(3)
    w = {k: rng.normal(size=(b.T, b.N_tot)) for k in ("logdiv", "ov", "off")}
    _, m = o.rollout(st, b.actions, 10, b.T, nthreads=1)
    for s in range(b.S):
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        valid = b.valid[a0:a1].astype(bool)
        exp = 0.0
        for k in ("logdiv", "ov", "off"):
            v = m[k][:, a0:a1][:, valid]
            ww = w[k][:, a0:a1][:, valid]
            exp += float(np.sum(np.where(np.isfinite(v), ww * v, 0.0)))
        got = o.objective(s, st, act, 10, b.T, 0.0, w["logdiv"], w["ov"], w["off"])
        assert abs(got - exp) <= 1e-9 * max(1.0, abs(exp)), (s, got, exp)
        lo = o.loss(s, st, act, 10, b.T)
        got2 = o.objective(s, st, act, 10, b.T, 0.5, w["logdiv"], w["ov"], w["off"])
        assert abs(got2 - (exp + 0.5 * lo)) <= 1e-9 * max(1.0, abs(got2))
        # the loss alone: the same gradient as oracle_loss_grad
        dirs = [(t, c, g) for t in (0, 5, 11) for c in (0, 1) for g in range(a0, a1) if b.valid[g]]
        g1 = o.loss_grad(s, st, act, 10, b.T, dirs)
        g2 = o.objective_grad(s, st, act, 10, b.T, [(0, t, c, g) for t, c, g in dirs], w_loss=1.0)
        assert np.array_equal(g1, g2)


def test_offroad_gradient_closed_form_beside_a_straight_edge():
    # One agent driving straight (a = kappa = 0) at heading th0 in (0, pi/2)
    # above a road edge along +x (the road on its left, y > 0): every corner
    # is on road, the lowest corner is nearest, off = -(y - hl sin th - hw
    # cos th).  After step 1 the velocity lies along th0, so y_k = y0 + vy0
    # dt + (k-1) v sin(th0) dt and dy_k/dth0 = (k-1) v cos(th0) dt.
    th0, v, L, W, T = 0.3, 2.0, 4.5, 2.0, 10
    edge = np.stack([np.arange(-200.0, 200.5, 0.5), np.zeros(801)], 1)
    a = _straight(0.0, 5.0, th0, v)
    b = tiny_batch([dict(a, L=L, W=W)], roadgraph=[(edge, 1)])
    o = oracle.Oracle(b)
    st = _state([a])
    act = np.zeros((T, 3, 1))
    rng = np.random.default_rng(0)
    g = rng.uniform(0.5, 1.5, size=(T, 1))
    k = np.arange(1, T + 1)
    y = 5.0 + k * v * np.sin(th0) * DT
    off = -(y - 0.5 * L * np.sin(th0) - 0.5 * W * np.cos(th0))
    assert abs(o.objective(0, st, act, 10, T, g_off=g) - np.sum(g[:, 0] * off)) < 1e-9
    d_y0, d_x0, d_th0 = o.objective_grad(0, st, act, 10, T, [(1, 0, 1, 0), (1, 0, 0, 0), (1, 0, 2, 0)], g_off=g)
    assert abs(d_y0 - (-g.sum())) < 1e-12
    assert abs(d_x0) < 1e-12
    dth = -(k - 1) * v * np.cos(th0) * DT + 0.5 * L * np.cos(th0) - 0.5 * W * np.sin(th0)
    assert abs(d_th0 - np.sum(g[:, 0] * dth)) < 1e-9
    # reversing the edge puts the agent off road: the signs flip
    b2 = tiny_batch([dict(a, L=L, W=W)], roadgraph=[(edge[::-1].copy(), 1)])
    o2 = oracle.Oracle(b2)
    assert abs(o2.objective_grad(0, st, act, 10, T, [(1, 0, 1, 0)], g_off=g)[0] - g.sum()) < 1e-12


def test_overlap_gradient_closed_form_two_boxes():
    # Two axis-aligned boxes moving together along +x: the x axis is the
    # shallowest (depth hlA + hlB - |dx| = 0.5 m against 1.5 m along y), so
    # d ov / d xB = -1 and d ov / d xA = +1 for both agents' metric, and the
    # y position does not enter.
    T, v = 6, 3.0
    A, B = _straight(0.0, 0.0, 0.0, v), _straight(4.0, 0.5, 0.0, v)
    b = tiny_batch([dict(A, L=4.5, W=2.0), dict(B, L=4.5, W=2.0)])
    o = oracle.Oracle(b)
    st = _state([A, B])
    act = np.zeros((T, 3, 2))
    g = np.random.default_rng(1).uniform(0.5, 1.5, size=(T, 2))
    assert abs(o.objective(0, st, act, 10, T, g_ov=g) - 0.5 * g.sum()) < 1e-9
    dxa, dxb, dyb = o.objective_grad(0, st, act, 10, T, [(1, 0, 0, 0), (1, 0, 0, 1), (1, 0, 1, 1)], g_ov=g)
    assert abs(dxa - g.sum()) < 1e-12 and abs(dxb + g.sum()) < 1e-12 and abs(dyb) < 1e-12


def test_logdiv_gradient_closed_form():
    # Straight driving from (x0, y0) with velocity (vx0, vy0): x_k = x0 + k
    # vx0 dt.  With v = |(vx0, vy0)| the velocity after step 1 is v (cos th0,
    # sin th0), so dx_k/dvx0 = dt + (k-1) dt cos(th0) vx0 / v.
    th0, v, T = 0.7, 6.0, 9
    a = _straight(1.0, -2.0, th0, v)
    log = np.zeros((91, 1, 2)); log[:, 0, 0] = 30.0; log[:, 0, 1] = 12.0
    b = tiny_batch([a], log=log)
    o = oracle.Oracle(b)
    st = _state([a])
    act = np.zeros((T, 3, 1))
    g = np.random.default_rng(2).uniform(0.5, 1.5, size=(T, 1))
    k = np.arange(1, T + 1)
    x = 1.0 + k * a["vx"] * DT
    y = -2.0 + k * a["vy"] * DT
    ld = np.hypot(x - 30.0, y - 12.0)
    assert abs(o.objective(0, st, act, 10, T, g_logdiv=g) - np.sum(g[:, 0] * ld)) < 1e-9
    dx0, dvx0 = o.objective_grad(0, st, act, 10, T, [(1, 0, 0, 0), (1, 0, 3, 0)], g_logdiv=g)
    assert abs(dx0 - np.sum(g[:, 0] * (x - 30.0) / ld)) < 1e-12
    dxk = DT + (k - 1) * DT * np.cos(th0) * a["vx"] / v
    dyk = (k - 1) * DT * np.sin(th0) * a["vx"] / v
    exp = np.sum(g[:, 0] * ((x - 30.0) * dxk + (y - 12.0) * dyk) / ld)
    assert abs(dvx0 - exp) < 1e-10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_objective_gradient_matches_central_differences(seed):
    # Random weights on every metric and the loss; directions over actions
    # and initial-state components of the policy agents.
    b = synth.make_batch(3, seed=seed, scenes=range(2), N=8, T=16)
    o = oracle.Oracle(b)
    st0 = o.initial_state()
    act = b.actions.astype(np.float64)
    rng = np.random.default_rng(seed)
    w = {k: rng.normal(size=(b.T, b.N_tot)) for k in ("g_logdiv", "g_ov", "g_off")}
    checked = skipped = 0
    for s in range(b.S):
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        agents = [g for g in range(a0, a1) if b.valid[g]]
        dirs = [(0, int(rng.integers(0, b.T)), int(rng.integers(0, 2)), int(rng.choice(agents))) for _ in range(16)]
        dirs += [(1, 0, int(rng.integers(0, 5)), int(rng.choice(agents))) for _ in range(10)]
        gd = o.objective_grad(s, st0, act, 10, b.T, dirs, w_loss=0.3, **w)

        def J(kind, t, c, g, d):
            a, st = act, st0
            if kind == 0:
                a = act.copy(); a[t, c, g] += d
            else:
                st = {k: v.copy() for k, v in st0.items()}
                st[("x", "y", "th", "vx", "vy")[c]][g] += d
            return o.objective(s, st, a, 10, b.T, 0.3, **w)
        for dr, gv in zip(dirs, gd):
            fd = (J(*dr, H) - J(*dr, -H)) / (2 * H)
            fd2 = (J(*dr, 2 * H) - J(*dr, -2 * H)) / (4 * H)
            if abs(fd - fd2) > 1e-5 * max(1.0, abs(fd)):  # a max switch or kink inside [-2h, 2h]
                skipped += 1
                continue
            checked += 1
            assert abs(gv - fd) <= 1e-6 * max(1.0, abs(fd)), (s, dr, gv, fd)
    assert checked >= 36 and skipped <= checked // 3


def test_idm_initial_state_is_a_constant():
    b = synth.make_batch(1, seed=7, S=1, N=6, R=800, T=8)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    w = np.ones((b.T, b.N_tot))
    idm = [g for g in range(b.N_tot) if b.kind[g] == synth.KIND_IDM and b.valid[g]]
    g = o.objective_grad(0, st, act, 10, b.T, [(1, 0, c, i) for i in idm for c in range(5)], w_loss=1.0,
                         g_logdiv=w, g_ov=w, g_off=w)
    assert (g == 0).all()
