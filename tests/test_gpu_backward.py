"""Differentiable rollout with caller-supplied metric gradients (needs a B300).

wsim_rollout_record / wsim_rollout_backward give the gradient of any weighted
sum of the per-step metrics (log divergence, overlap depth, off-road distance:
Sec. 3.4) and of the smooth loss, with respect to the actions and the initial
state (the differentiable simulation of Sec. 6).  Checked against the FP64
oracle's dual numbers (oracle_objective_grad, itself pinned by closed forms
and central differences): relative L2 error <= 1e-3 per scene.  The recorded
forward's metric rows and loss must equal wsim_rollout's and wsim_loss_grad's
bit for bit, and the gradient must not depend on the checkpoint interval.

Overlap depth and off-road distance are maxima (over partners, over corners
and nearest segments).  Where the float32 and float64 trajectories could pick
different maximisers (a second partner, corner or non-adjacent segment within
1e-4 m of the best) the metric's weight is set to 0 for that agent-step; the
count is printed.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth
from tests import gpu_harness as H

pytestmark = pytest.mark.gpu
T0 = synth.T0
TOL_GRAD = 1e-3
BAND = 1e-4


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def _segments(b, s):
    """Road-edge segments of scene s: start, vector, global point index."""
    r0, r1 = b.rg_off[s], b.rg_off[s + 1]
    k = np.arange(r0, r1 - 1)
    ok = ((b.rg_valid[k] != 0) & (b.rg_valid[k + 1] != 0) & (b.rg_type[k] == 1) & (b.rg_type[k + 1] == 1)
          & (b.rg_poly[k] == b.rg_poly[k + 1]))
    k = k[ok]
    a = np.stack([b.rg_x[k], b.rg_y[k]], 1).astype(np.float64)
    u = np.stack([b.rg_x[k + 1], b.rg_y[k + 1]], 1).astype(np.float64) - a
    return a, u, k


def _near_ties(b, traj):
    """Agent-steps whose overlap or off-road maximiser is not decided by more
    than BAND: (ov_tie, off_tie) boolean [T, N_tot] arrays."""
    T = traj.shape[1]
    ov_tie = np.zeros((T, b.N_tot), bool)
    off_tie = np.zeros((T, b.N_tot), bool)
    o = oracle.Oracle(b)
    corners = ((1, 1), (1, -1), (-1, -1), (-1, 1))
    for s in range(b.S):
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        ag = np.arange(a0, a1)
        va = ag[b.valid[a0:a1] != 0]
        A, U, K = _segments(b, s)
        for k in range(T):
            st = H.state64(traj[:, k, :], ag)
            x, y, th = st["x"], st["y"], st["th"]

            def box(q):
                return (x[q], y[q], th[q], b.L[a0 + q], b.W[a0 + q])
            for g in va:
                i = g - a0
                ds = sorted(oracle.box_depth(box(min(i, j - a0)), box(max(i, j - a0))) for j in va if j != g)
                if len(ds) >= 2 and ds[-1] - ds[-2] < BAND:
                    ov_tie[k, g] = True
                if len(A) == 0:
                    continue
                c, sn = np.cos(th[i]), np.sin(th[i])
                hl, hw = 0.5 * b.L[g], 0.5 * b.W[g]
                sds = []
                for sl, sw in corners:
                    px = x[i] + sl * hl * c - sw * hw * sn
                    py = y[i] + sl * hl * sn + sw * hw * c
                    w = np.stack([px - A[:, 0], py - A[:, 1]], 1)
                    t = np.clip((w * U).sum(1) / (U * U).sum(1), 0, 1)
                    d = np.hypot(w[:, 0] - t * U[:, 0], w[:, 1] - t * U[:, 1])
                    e = int(np.argmin(d))
                    far = np.abs(K - K[e]) > 1  # neither the winner nor a segment sharing one of its vertices
                    if far.any() and d[far].min() - d[e] < BAND:
                        off_tie[k, g] = True
                    sds.append(o.point_sd(s, px, py)[0])
                sds.sort()
                if sds[-1] - sds[-2] < BAND:
                    off_tie[k, g] = True
    return ov_tie, off_tie


def _weights(b, T, seed, ties=None):
    """Random metric weights [T, N_tot] (0 for invalid agents and near-tied
    maxima) and per-scene loss weights."""
    rng = np.random.default_rng(seed)
    w = {k: rng.normal(size=(T, b.N_tot)).astype(np.float32) for k in ("logdiv", "ov", "off")}
    inval = b.valid == 0
    for v in w.values():
        v[:, inval] = 0
    if ties is not None:
        w["ov"][ties[0]] = 0
        w["off"][ties[1]] = 0
    return w, rng.uniform(0.5, 1.5, b.S)


def _gpu(w, b, weights, loss_w, ck=10, T=None):
    """Record + backward on the GPU: (metric rows, loss, dact, dst0 rows)."""
    T = b.T if T is None else T
    sim = w.Sim(w.DeviceBatch(b))
    st = w.State.from_batch(b)
    act = torch.as_tensor(b.actions[:T]).cuda().contiguous()
    m = w.Metrics(b.N_tot, b.S, rows=T)
    loss = sim.rollout_record(st, act, m, T0, T, ck)
    g = {k: torch.as_tensor(v).cuda() for k, v in weights.items()}
    da, ds = sim.rollout_backward(act, g["logdiv"], g["ov"], g["off"],
                                  None if loss_w is None else torch.as_tensor(loss_w).cuda())
    torch.cuda.synchronize()
    assert sim.status() == 0
    out = dict(m={k: getattr(m, k).cpu().numpy() for k in ("ov", "off", "logdiv", "flags", "reward")},
               loss=loss.cpu().numpy(), dact=da.cpu().numpy(), dst0=ds.data.cpu().numpy())
    sim.close()
    return out


def _oracle_check(b, T, weights, loss_w, got, n_act=160, seed=0):
    """Relative L2 error per scene of the GPU gradient against the oracle's
    duals (sampled action directions and every initial-state component of
    the valid policy agents); returns the worst."""
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions[:T].astype(np.float64)
    rng = np.random.default_rng(seed)
    wf = {("g_" + k): v.astype(np.float64) for k, v in weights.items()}
    worst = 0.0
    for s in range(b.S):
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        pol = [g for g in range(a0, a1) if b.valid[g] and b.kind[g] != synth.KIND_IDM]
        if not pol:
            continue
        adirs = [(0, t, c, g) for g in pol for t in range(T)
                 for c in ((0, 1) if b.kind[g] == synth.KIND_BICYCLE else (0, 1, 2))]
        if len(adirs) > n_act:
            adirs = [adirs[k] for k in rng.choice(len(adirs), n_act, replace=False)]
        sdirs = [(1, 0, c, g) for g in pol for c in range(5)]
        dirs = adirs + sdirs
        ref = o.objective_grad(s, st, act, T0, T, dirs, w_loss=float(loss_w[s]) if loss_w is not None else 0.0,
                               **wf)
        rows = {0: 0, 1: 1, 2: 4, 3: 6, 4: 7}  # state component -> row of the [10, N] state block
        g = np.array([got["dact"][t, c, gg] if k == 0 else got["dst0"][rows[c], gg] for k, t, c, gg in dirs])
        e = float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30))
        assert e <= TOL_GRAD, (s, e)
        worst = max(worst, e)
    return worst


def test_record_forward_bit_identical_to_rollout_and_loss_grad(wsim):
    for b in (synth.make_batch(1, seed=31, S=6, R=4000, T=24), synth.make_batch(3, seed=31, S=12)):
        ref = H.run_rollout(b, mode=wsim.MODE_FUSED)
        sim = wsim.Sim(wsim.DeviceBatch(b))
        st = wsim.State.from_batch(b)
        act = torch.as_tensor(b.actions).cuda().contiguous()
        m = wsim.Metrics(b.N_tot, b.S, rows=b.T)
        stT = wsim.State(b.N_tot)
        loss = sim.rollout_record(st, act, m, T0, b.T, 10, st_T=stT)
        l2, _ = sim.loss_grad(st, act, T0, b.T, 10, grad=False)
        torch.cuda.synchronize()
        assert sim.status() == 0
        for k in ("ov", "off", "logdiv", "flags", "reward"):
            assert np.array_equal(getattr(m, k).cpu().numpy().view(np.uint8), ref[k].view(np.uint8)), k
        assert np.array_equal(stT.data.cpu().numpy().view(np.uint8), ref["final"].view(np.uint8))
        assert torch.equal(loss, l2)
        sim.close()


def test_loss_weights_reproduce_loss_grad_bit_for_bit(wsim):
    b = synth.make_batch(3, seed=32, S=10, T=40)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().contiguous()
    _, ref = sim.loss_grad(st, act, T0, b.T, 10)
    sim.rollout_record(st, act, None, T0, b.T, 10)
    da, _ = sim.rollout_backward(act, loss_w=torch.ones(b.S, dtype=torch.float64, device="cuda"), dst0=False)
    torch.cuda.synchronize()
    assert torch.equal(da, ref)
    # metric weights need a record with metrics
    with pytest.raises(wsim.WsimError) as e:
        sim.rollout_backward(act, g_ov=torch.ones((b.T, b.N_tot), device="cuda"))
    assert e.value.code == wsim.ESTATE
    sim.close()
    sim = wsim.Sim(wsim.DeviceBatch(b))
    with pytest.raises(wsim.WsimError) as e:
        sim.rollout_backward(act, loss_w=torch.ones(b.S, dtype=torch.float64, device="cuda"))
    assert e.value.code == wsim.ESTATE
    sim.close()


def test_metric_gradient_matches_oracle_duals_8x8(wsim):
    b = synth.make_batch(3, seed=33, S=8, N=8)
    traj = H.run_rollout(b)["traj"]
    ties = _near_ties(b, traj)
    weights, loss_w = _weights(b, b.T, 33, ties)
    got = _gpu(wsim, b, weights, loss_w)
    worst = _oracle_check(b, b.T, weights, loss_w, got, n_act=480)
    print("metric gradient rel err (8 scenes x 8 agents, 480 action + all initial-state directions each):", worst,
          "tied agent-steps excluded: ov", int(ties[0].sum()), "off", int(ties[1].sum()))


def test_each_metric_alone_matches_oracle(wsim):
    b = synth.make_batch(3, seed=34, S=4, N=10, T=30)
    traj = H.run_rollout(b)["traj"]
    ties = _near_ties(b, traj)
    for only in ("logdiv", "ov", "off"):
        weights, _ = _weights(b, b.T, 34, ties)
        for k in weights:
            if k != only:
                weights[k][:] = 0
        got = _gpu(wsim, b, weights, None)
        e = _oracle_check(b, b.T, weights, None, got)
        print(only, "alone: rel err", e)


def test_checkpoint_interval_bit_identical(wsim):
    b = synth.make_batch(3, seed=35, S=12, T=37)
    weights, loss_w = _weights(b, b.T, 35)
    ref = _gpu(wsim, b, weights, loss_w, ck=10)
    for ck in (1, 7, 37):
        g = _gpu(wsim, b, weights, loss_w, ck=ck)
        for k in ("dact", "dst0", "loss"):
            assert np.array_equal(g[k].view(np.uint8), ref[k].view(np.uint8)), (ck, k)


def test_delta_ego_idm_agents_and_roadgraph_scenes(wsim):
    # delta ego in scene 0, bicycle ego in scene 1, IDM agents (constants for
    # the derivative) around them, 3000-point roadgraphs
    b = synth.make_batch(4, seed=36, S=2, N=12, R=3000, T=20)
    traj = H.run_rollout(b)["traj"]
    ties = _near_ties(b, traj)
    weights, loss_w = _weights(b, b.T, 36, ties)
    got = _gpu(wsim, b, weights, loss_w)
    idm = b.kind == synth.KIND_IDM
    assert (got["dact"][:, :, idm] == 0).all() and (got["dst0"][:, idm] == 0).all()
    e = _oracle_check(b, b.T, weights, loss_w, got, n_act=10 ** 9)
    print("delta/bicycle egos with IDM agents: rel err", e)


def test_full_size_256x64_sampled(wsim):
    # the differentiable workload at full size (256 scenes x 64 agents x 80
    # steps), three scenes checked against the oracle
    b = synth.make_batch(3, seed=37)
    weights, loss_w = _weights(b, b.T, 37)
    got = _gpu(wsim, b, weights, loss_w)
    assert np.isfinite(got["dact"]).all() and np.isfinite(got["dst0"]).all()
    sub_idx = [0, 101, 255]
    sub = b.subset(sub_idx)
    ag = np.concatenate([np.arange(b.agent_off[s], b.agent_off[s + 1]) for s in sub_idx])
    ties = _near_ties(sub, H.run_rollout(sub)["traj"])
    wsub = {k: v[:, ag].copy() for k, v in weights.items()}
    wsub["ov"][ties[0]] = 0
    wsub["off"][ties[1]] = 0
    # the sub-batch's gradient from the full batch's run, where no tie was masked
    keep = ~(ties[0] | ties[1])
    got_sub = _gpu(wsim, sub, wsub, loss_w[sub_idx])
    full = dict(dact=got["dact"][:, :, ag], dst0=got["dst0"][:, ag])
    if keep.all():
        assert np.array_equal(full["dact"].view(np.uint8), got_sub["dact"].view(np.uint8))
    e = _oracle_check(sub, b.T, wsub, loss_w[sub_idx], got_sub, n_act=120)
    print("256x64 sampled scenes: rel err", e)


def test_rollout_fn_autograd(wsim):
    b = synth.make_batch(3, seed=38, S=4, N=8, T=16)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().requires_grad_(True)
    s0 = st.data.clone().requires_grad_(True)
    logdiv, ov, off, loss = wsim.RolloutFn.apply(act, s0, sim, T0, 4)
    weights, loss_w = _weights(b, b.T, 38)
    g = {k: torch.as_tensor(v).cuda() for k, v in weights.items()}
    lw = torch.as_tensor(loss_w).cuda()
    J = ((g["logdiv"] * logdiv).sum() + (g["ov"] * torch.where(torch.isfinite(ov), ov, 0)).sum()
         + (g["off"] * torch.where(torch.isfinite(off), off, 0)).sum() + (lw * loss).sum())
    J.backward()
    sim.rollout_record(st, act.detach(), wsim.Metrics(b.N_tot, b.S, rows=b.T), T0, b.T, 4)
    gm = {k: torch.where(torch.isfinite(v), g[k], torch.zeros_like(g[k])) for k, v in
          (("logdiv", logdiv), ("ov", ov), ("off", off))}
    da, ds = sim.rollout_backward(act.detach(), gm["logdiv"], gm["ov"], gm["off"], lw)
    assert torch.allclose(act.grad, da, rtol=1e-6, atol=1e-6)
    assert torch.allclose(s0.grad, ds.data, rtol=1e-6, atol=1e-6)
    # a second forward replaces the record: the first graph cannot go back
    out1 = wsim.RolloutFn.apply(act, s0, sim, T0, 4)
    wsim.RolloutFn.apply(act, s0, sim, T0, 4)
    with pytest.raises(RuntimeError):
        out1[0].sum().backward()
    sim.close()
