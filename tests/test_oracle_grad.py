"""Pins of the oracle's differentiable loss and its dual-number gradient.

The loss is the BPTT objective of the differentiable rollout (squared log
divergence, Sec. 3.4, plus a softplus-smoothed overlap penalty); the paper
names differentiable simulation as its future work (Sec. 6).  Pins: central
finite differences (h = 1e-3, FP64) of the oracle's own FP64 loss, closed
forms of the loss on trajectories that are known analytically, and the
penalty of far-apart boxes vanishing.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch

H = 1e-3


def _grad_case(seed, n_scenes=2, n_agents=8, T=20):
    b = synth.make_batch(3, seed=seed, scenes=range(n_scenes), N=n_agents, T=T)
    return b, oracle.Oracle(b)


@pytest.mark.parametrize("seed", [0, 1])
def test_dual_gradient_matches_central_differences(seed):
    b, o = _grad_case(seed)
    st0 = o.initial_state()
    act = b.actions.astype(np.float64)
    rng = np.random.default_rng(seed)
    checked = skipped = 0
    for s in range(b.S):
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        dirs = [(int(rng.integers(0, b.T)), int(rng.integers(0, 2)), int(rng.integers(a0, a1))) for _ in range(24)]
        g = o.loss_grad(s, st0, act, 10, b.T, dirs)
        for (t, c, gi), gd in zip(dirs, g):
            def L(delta):
                a = act.copy(); a[t, c, gi] += delta
                return o.loss(s, st0, a, 10, b.T)
            fd = (L(H) - L(-H)) / (2 * H)
            fd2 = (L(H / 2) - L(-H / 2)) / H
            # a kink (active SAT axis or softplus branch switch) inside [-h, h]
            # shows as disagreement between the two step sizes: skip, count
            if abs(fd - fd2) > 1e-4 * max(1.0, abs(fd)):
                skipped += 1
                continue
            checked += 1
            assert abs(gd - fd) <= 1e-5 * max(1.0, abs(fd)), (s, t, c, gi, gd, fd)
    assert checked >= 40 and skipped <= checked // 4


def test_loss_closed_form_straight_line():
    # One agent driving straight with constant a, log = the analytic path
    # shifted sideways by 3 m: loss = sum_t 9 (no pairs).
    N, T = 1, 30
    th, v0, a = 0.4, 10.0, 1.5
    t = np.arange(91) * 0.1
    tt = np.clip(t - 1.0, 0, None)
    path = np.stack([np.cos(th) * (v0 * tt + 0.5 * a * tt ** 2), np.sin(th) * (v0 * tt + 0.5 * a * tt ** 2)], 1)
    shift = 3.0 * np.array([-np.sin(th), np.cos(th)])
    log = (path + shift)[:, None, :]
    b = tiny_batch([dict(x=0.0, y=0.0, th=th, v=v0)], log=log)
    o = oracle.Oracle(b)
    st = dict(x=np.zeros(1), y=np.zeros(1), th=np.array([th]), vx=np.array([v0 * np.cos(th)]),
              vy=np.array([v0 * np.sin(th)]), s=np.zeros(1))
    act = np.zeros((T, 3, 1)); act[:, 0, 0] = a
    # the log is float32: compare against the float32 log's own distances
    lx, ly = b.log_x.astype(np.float64)[11:11 + T, 0], b.log_y.astype(np.float64)[11:11 + T, 0]
    k = np.arange(1, T + 1) * 0.1
    px, py = np.cos(th) * (v0 * k + 0.5 * a * k ** 2), np.sin(th) * (v0 * k + 0.5 * a * k ** 2)
    exp = np.sum((px - lx) ** 2 + (py - ly) ** 2)
    assert abs(o.loss(0, st, act, 10, T) - exp) < 1e-8
    assert abs(exp - 9.0 * T) < 1e-3


def test_overlap_penalty_softplus_values():
    # Two agents at rest, log at their own positions: loss = T * lam * tau *
    # softplus(d / tau) with d the overlap depth (axis-aligned: closed form).
    T, lam, tau = 5, 1.0, 0.25
    for dx, d in ((3.0, 1.0), (4.5, -0.5), (40.0, -36.0)):
        log = np.zeros((91, 2, 2)); log[:, 1, 0] = dx
        b = tiny_batch([dict(x=0.0, y=0.0, L=4.0, W=2.0), dict(x=dx, y=0.0, L=4.0, W=2.0)], log=log)
        o = oracle.Oracle(b)
        st = o.initial_state()
        act = np.zeros((T, 3, 2))
        exp = T * lam * tau * np.log1p(np.exp(d / tau))
        assert abs(o.loss(0, st, act, 10, T, lam, tau) - exp) < 1e-12 * max(1, exp) + 1e-300


def test_gradient_of_log_term_closed_form():
    # No pairs, one agent: dL/da_0 for the straight-line case equals
    # sum_t 2 (p_t - log_t) . dp_t/da_0 with dp_t/da_0 = dir * (dt^2/2 + (t-1) dt^2).
    th, v0 = 0.2, 8.0
    log = np.zeros((91, 1, 2)); log[:, 0, 0] = 50.0; log[:, 0, 1] = -7.0
    b = tiny_batch([dict(x=0.0, y=0.0, th=th, v=v0)], log=log)
    o = oracle.Oracle(b)
    st = dict(x=np.zeros(1), y=np.zeros(1), th=np.array([th]), vx=np.array([v0 * np.cos(th)]),
              vy=np.array([v0 * np.sin(th)]), s=np.zeros(1))
    T = 12
    act = np.zeros((T, 3, 1))
    g = o.loss_grad(0, st, act, 10, T, [(0, 0, 0)])[0]
    dt = 0.1
    k = np.arange(1, T + 1)
    pos = np.stack([np.cos(th) * v0 * k * dt, np.sin(th) * v0 * k * dt], 1)
    dpos = (dt * dt / 2 + (k - 1) * dt * dt)[:, None] * np.array([np.cos(th), np.sin(th)])
    exp = np.sum(2 * (pos - np.array([50.0, -7.0])) * dpos)
    assert abs(g - exp) < 1e-9


def test_loss_with_idm_agents_matches_rollout_log_divergence():
    # With lambda = 0 the loss is sum_t sum_i d_i(t)^2 of the same closed-loop
    # rollout (IDM agents included) that oracle_rollout produces.
    b = synth.make_batch(1, seed=4, S=2, R=3000, T=15)
    o = oracle.Oracle(b)
    st = o.initial_state()
    _, m = o.rollout(st, b.actions, 10, b.T, nthreads=1)
    for s in range(b.S):
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        exp = float(np.sum(m["logdiv"][:, a0:a1] ** 2))
        got = o.loss(s, st, b.actions.astype(np.float64), 10, b.T, lam=0.0)
        assert abs(got - exp) <= 1e-9 * max(1.0, exp)


def test_idm_stop_gradient_equals_fd_when_out_of_reach():
    # An ego far from every IDM agent: nothing it does changes their motion,
    # so the stop-gradient derivative equals the finite difference.
    b = synth.make_batch(1, seed=6, S=1, N=6, R=500, T=12)
    b.x[0] += 5000.0
    b.log_x[:, 0] += 5000.0
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    dirs = [(t, c, 0) for t in (0, 3, 11) for c in (0, 1)]
    g = o.loss_grad(0, st, act, 10, b.T, dirs)
    for (t, c, gi), gd in zip(dirs, g):
        a1, a2 = act.copy(), act.copy()
        a1[t, c, gi] += H
        a2[t, c, gi] -= H
        fd = (o.loss(0, st, a1, 10, b.T) - o.loss(0, st, a2, 10, b.T)) / (2 * H)
        assert abs(gd - fd) <= 1e-5 * max(1.0, abs(fd))
