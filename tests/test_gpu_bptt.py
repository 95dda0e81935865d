"""BPTT adjoint on the GPU against the FP64 oracle (needs a B300).

The oracle's gradient comes from forward-mode dual numbers over its own FP64
rollout (independent of the hand adjoint); it is itself pinned against
central differences on the CPU.  Gates: relative L2 error of the gradient
<= 1e-3 per scene, loss relative error <= 1e-5, checkpoint interval and
launch path bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth

pytestmark = pytest.mark.gpu
T0 = synth.T0
TOL_GRAD = 1e-3
TOL_LOSS = 1e-5


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def gpu_grad(w, b, ckpt=10, plain=False, T=None):
    T = b.T if T is None else T
    sim = w.Sim(w.DeviceBatch(b))
    st = w.State.from_batch(b)
    act = torch.as_tensor(b.actions[:T]).cuda().contiguous()
    loss, dact = sim.loss_grad(st, act, T0, T, ckpt_every=ckpt, plain=plain)
    torch.cuda.synchronize()
    assert sim.status() == 0
    sim.close()
    return loss.cpu().numpy(), dact.cpu().numpy()


def policy_dirs(b, s, T):
    """All action components of the scene's policy agents."""
    a0, a1 = b.agent_off[s], b.agent_off[s + 1]
    out = []
    for g in range(a0, a1):
        if not b.valid[g] or b.kind[g] == synth.KIND_IDM:
            continue
        comps = (0, 1) if b.kind[g] == synth.KIND_BICYCLE else (0, 1, 2)
        out += [(t, c, g) for t in range(T) for c in comps]
    return out


def rel_err(g, ref):
    return float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30))


def test_gradient_matches_oracle_duals_8x8(wsim):
    b = synth.make_batch(3, seed=0, S=8, N=8)
    loss, dact = gpu_grad(wsim, b)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    worst = 0.0
    for s in range(b.S):
        lo = o.loss(s, st, act, T0, b.T)
        assert abs(loss[s] - lo) <= TOL_LOSS * abs(lo), (s, loss[s], lo)
        dirs = policy_dirs(b, s, b.T)
        ref = o.loss_grad(s, st, act, T0, b.T, dirs)
        got = np.array([dact[t, c, g] for t, c, g in dirs], dtype=np.float64)
        e = rel_err(got, ref)
        worst = max(worst, e)
        assert e <= TOL_GRAD, (s, e)
    print("grad rel err (8 scenes x 8 agents, all components):", worst)


@pytest.mark.parametrize("tau", [0.05, 0.25, 2.0])
def test_pair_culling_exact_at_every_tau(wsim, tau):
    # Pairs whose SAT depth bound lies below -120 tau are skipped (their
    # softplus and sigmoid are exactly 0 in float32).  Agents packed into a
    # 30 m square (overlapping and near pairs) and spread over 200 m, at a
    # tau that culls almost nothing (2 m), the default and a small one:
    # loss and gradient against the oracle's FP64 sum over every pair.
    b = synth.make_batch(3, seed=6, S=4, N=24, T=30)
    for s in range(2):  # the first two scenes packed, the others as drawn
        a0, a1 = b.agent_off[s], b.agent_off[s + 1]
        for k in ("x", "y"):
            v = getattr(b, k)
            v[a0:a1] = (100.0 + 0.15 * (v[a0:a1].astype(np.float64) - 100.0)).astype(np.float32)
            lg = getattr(b, "log_" + k)
            lg[:, a0:a1] = (100.0 + 0.15 * (lg[:, a0:a1].astype(np.float64) - 100.0)).astype(np.float32)
    cfg = wsim.default_config(loss_tau=tau)
    sim = wsim.Sim(wsim.DeviceBatch(b), cfg)
    loss, dact = sim.loss_grad(wsim.State.from_batch(b), torch.as_tensor(b.actions).cuda().contiguous(), T0, b.T)
    torch.cuda.synchronize()
    assert sim.status() == 0
    sim.close()
    loss, dact = loss.cpu().numpy(), dact.cpu().numpy()
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    for s in range(b.S):
        lo = o.loss(s, st, act, T0, b.T, tau=tau)
        assert abs(loss[s] - lo) <= TOL_LOSS * abs(lo), (s, loss[s], lo)
        dirs = policy_dirs(b, s, b.T)
        ref = o.loss_grad(s, st, act, T0, b.T, dirs, tau=tau)
        got = np.array([dact[t, c, g] for t, c, g in dirs], dtype=np.float64)
        assert rel_err(got, ref) <= TOL_GRAD, (s, tau, rel_err(got, ref))


def test_gradient_matches_central_differences(wsim):
    b = synth.make_batch(3, seed=1, S=8, N=8)
    _, dact = gpu_grad(wsim, b)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    rng = np.random.default_rng(1)
    h = 1e-3
    got, ref, skipped = [], [], 0
    for s in range(b.S):
        dirs = policy_dirs(b, s, b.T)
        for k in rng.choice(len(dirs), 6, replace=False):
            t, c, g = dirs[k]

            def L(d):
                a = act.copy()
                a[t, c, g] += d
                return o.loss(s, st, a, T0, b.T)
            fd = (L(h) - L(-h)) / (2 * h)
            fd2 = (L(h / 2) - L(-h / 2)) / h
            if abs(fd - fd2) > 1e-4 * max(1.0, abs(fd)):  # a kink inside [-h, h]
                skipped += 1
                continue
            got.append(dact[t, c, g])
            ref.append(fd)
    e = rel_err(np.array(got), np.array(ref))
    print("grad vs central differences: rel err", e, "checked", len(got), "kinks skipped", skipped)
    assert len(got) >= 36 and e <= TOL_GRAD


def test_checkpoint_interval_and_launch_path_bit_identical(wsim):
    b = synth.make_batch(3, seed=2, S=12)
    ref_l, ref_g = gpu_grad(wsim, b, ckpt=10)
    for ck, plain in ((1, False), (7, False), (80, False), (10, True)):
        l, g = gpu_grad(wsim, b, ckpt=ck, plain=plain)
        assert np.array_equal(l.view(np.uint8), ref_l.view(np.uint8)), (ck, plain)
        assert np.array_equal(g.view(np.uint8), ref_g.view(np.uint8)), (ck, plain)


def test_differentiable_256x64_full_size_sampled(wsim):
    b = synth.make_batch(3, seed=0)
    loss, dact = gpu_grad(wsim, b)
    assert np.isfinite(loss).all() and np.isfinite(dact).all()
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    rng = np.random.default_rng(3)
    for s in (0, 101, 255):
        lo = o.loss(s, st, act, T0, b.T)
        assert abs(loss[s] - lo) <= TOL_LOSS * abs(lo)
        dirs = policy_dirs(b, s, b.T)
        pick = [dirs[k] for k in rng.choice(len(dirs), 24, replace=False)]
        ref = o.loss_grad(s, st, act, T0, b.T, pick)
        got = np.array([dact[t, c, g] for t, c, g in pick], dtype=np.float64)
        assert rel_err(got, ref) <= TOL_GRAD, s


def test_max_agents_per_scene(wsim):
    # 256 agents: every warp owns rows and the per-warp pair buffers are full;
    # sampled directions against the oracle, and the checkpoint interval and
    # launch path still bit-identical
    b = synth.make_batch(3, seed=9, S=2, N=256, T=12)
    loss, dact = gpu_grad(wsim, b)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    rng = np.random.default_rng(4)
    for s in range(b.S):
        lo = o.loss(s, st, act, T0, b.T)
        assert abs(loss[s] - lo) <= TOL_LOSS * abs(lo), (s, loss[s], lo)
        dirs = policy_dirs(b, s, b.T)
        pick = [dirs[k] for k in rng.choice(len(dirs), 32, replace=False)]
        ref = o.loss_grad(s, st, act, T0, b.T, pick)
        got = np.array([dact[t, c, g] for t, c, g in pick], dtype=np.float64)
        assert rel_err(got, ref) <= TOL_GRAD, (s, rel_err(got, ref))
    for ck, plain in ((1, False), (10, True)):
        l, g = gpu_grad(wsim, b, ckpt=ck, plain=plain)
        assert np.array_equal(l.view(np.uint8), loss.view(np.uint8)), (ck, plain)
        assert np.array_equal(g.view(np.uint8), dact.view(np.uint8)), (ck, plain)


def test_delta_ego_and_idm_stop_gradient(wsim):
    # scene 0: delta ego, scene 1: bicycle ego; the other agents are IDM
    # (moving, constant for the derivative)
    b = synth.make_batch(4, seed=5, S=2, N=12, R=3000, T=20)
    assert b.kind[0] == synth.KIND_DELTA and b.kind[b.agent_off[1]] == synth.KIND_BICYCLE
    loss, dact = gpu_grad(wsim, b, ckpt=6)
    o = oracle.Oracle(b)
    st = o.initial_state()
    act = b.actions.astype(np.float64)
    for s in range(b.S):
        lo = o.loss(s, st, act, T0, b.T)
        assert abs(loss[s] - lo) <= TOL_LOSS * abs(lo)
        dirs = policy_dirs(b, s, b.T)
        ref = o.loss_grad(s, st, act, T0, b.T, dirs)
        got = np.array([dact[t, c, g] for t, c, g in dirs], dtype=np.float64)
        assert rel_err(got, ref) <= TOL_GRAD, s
        idm = [g for g in range(b.agent_off[s], b.agent_off[s + 1]) if b.kind[g] == synth.KIND_IDM]
        assert (dact[:, :, idm] == 0).all()


def test_autograd_function(wsim):
    b = synth.make_batch(3, seed=6, S=4, N=8, T=16)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().requires_grad_(True)
    loss = wsim.RolloutLoss.apply(act, sim, st, T0, 4)
    weights = torch.arange(1, b.S + 1, dtype=torch.float64, device="cuda")
    (loss * weights).sum().backward()
    ref_l, ref_g = sim.loss_grad(st, act.detach(), T0, b.T, 4)
    assert torch.equal(loss.detach(), ref_l)
    w_agent = torch.repeat_interleave(weights, torch.as_tensor(np.diff(b.agent_off), device="cuda").long())
    assert torch.allclose(act.grad, ref_g * w_agent.float()[None, None, :])
    sim.close()
