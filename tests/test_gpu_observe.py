"""Observation function on the GPU against the FP64 oracle (needs a B300).

Agents in the observer's frame within float32 tolerances; the K nearest
roadgraph point indices bit-exact (both sides rank by the same float32 key,
ties to the lower index) and their coordinates in the observer's frame
within tolerance; every agent observing and an observer subset; K above a
scene's point count; the 1024-scene batch sampled; batches with more
observers than the warp-per-observer kernel has resident warps (that kernel
then observes them), with a dense cluster of tied points beyond a warp's
point list and more candidate tiles than a warp lists.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth
from tests.gpu_harness import run_rollout, state64

pytestmark = pytest.mark.gpu
TOL = 1e-5       # m, m/s absolute ...
REL = 3e-7       # ... plus this fraction of the vector's length: a float32
                 # rotation (cos, sin within 1 ulp, two rounded products) of a
                 # vector of length r errs by up to ~2.4e-7 r
TOL_YAW = 1e-6   # rad


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def _tol(r):
    """Tolerance of a rotated vector's components, r its length."""
    return TOL + REL * r


def _check(g, o, obs_rows, M, K):
    av, ov = g["agents_valid"][obs_rows], o["agents_valid"][obs_rows]
    assert np.array_equal(av, ov)
    ga, oa = g["agents"][obs_rows].astype(np.float64), o["agents"][obs_rows]
    m = ov.astype(bool)
    for c0 in (0, 3):  # position, velocity
        r = np.hypot(oa[..., c0], oa[..., c0 + 1])[m]
        for c in (c0, c0 + 1):
            d = np.abs(ga[..., c] - oa[..., c])[m]
            assert (d <= _tol(r)).all(), (c, d.max())
    dyaw = np.abs(np.angle(np.exp(1j * (ga[..., 2] - oa[..., 2]))))[m]
    assert dyaw.max(initial=0) <= TOL_YAW
    assert np.array_equal(g["rg_idx"][obs_rows], o["rg_idx"][obs_rows])
    ok = o["rg_idx"][obs_rows] >= 0
    orr = o["rg"][obs_rows]
    d = np.abs(g["rg"][obs_rows].astype(np.float64) - orr)[ok]
    r = np.hypot(orr[..., 0], orr[..., 1])[ok][:, None]
    assert (d <= _tol(r)).all(), d.max()
    return float(d.max(initial=0))


def _gpu_observe(wsim, b, rows, M, K, observers=None):
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State(b.N_tot, data=torch.as_tensor(rows).cuda().contiguous())
    ob = None if observers is None else torch.as_tensor(observers, dtype=torch.uint8).cuda()
    out = sim.observe(st, M, K, observers=ob)
    torch.cuda.synchronize()
    assert sim.status() == 0
    sim.close()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_every_agent_observes_after_a_rollout(wsim):
    # state after 40 steps of a rollout (compensated positions, unwrapped headings)
    b = synth.make_batch(0, seed=3, T=40)
    g = run_rollout(b, T=40)
    rows = g["final"]
    ag = np.arange(b.N_tot)
    st = state64(rows, ag)
    for K in (16, 500, 2500):  # 2500 > the scene's 2000 points: padding
        go = _gpu_observe(wsim, b, rows, 32, K)
        oo = oracle.Oracle(b).observe(st, 32, K)
        obs = np.nonzero(b.valid)[0]
        err = _check(go, oo, obs, 32, K)
        print("K", K, "max point error", err)
        assert (go["rg_idx"][b.valid == 0] == -1).all()  # invalid agents do not observe


def test_observer_subset_and_untouched_rows(wsim):
    b = synth.make_batch(3, seed=2, S=6, N=20, R=3000)
    rows = np.zeros((10, b.N_tot), np.float32)
    rows[0], rows[1], rows[4], rows[6], rows[7] = b.x, b.y, b.th, b.vx, b.vy
    observers = np.zeros(b.N_tot, np.uint8)
    observers[b.agent_off[:-1]] = 1  # the first agent of every scene
    go = _gpu_observe(wsim, b, rows, 24, 64, observers)
    oo = oracle.Oracle(b).observe(state64(rows, np.arange(b.N_tot)), 24, 64, observers)
    _check(go, oo, np.nonzero(observers)[0], 24, 64)
    others = observers == 0
    assert (go["rg_idx"][others] == -1).all() and (go["agents_valid"][others] == 0).all()


def test_batch_1024x128_sampled_observers(wsim):
    # the ego of every scene observes; 16 scenes checked against the oracle
    b = synth.make_batch(1, seed=0)
    rows = np.zeros((10, b.N_tot), np.float32)
    rows[0], rows[1], rows[4], rows[6], rows[7] = b.x, b.y, b.th, b.vx, b.vy
    observers = np.zeros(b.N_tot, np.uint8)
    observers[b.agent_off[:-1]] = 1
    go = _gpu_observe(wsim, b, rows, 128, 256, observers)
    scenes = list(range(0, b.S, b.S // 16))
    sub = b.subset(scenes)
    ag = np.concatenate([np.arange(b.agent_off[s], b.agent_off[s + 1]) for s in scenes])
    sub_obs = observers[ag]
    oo = oracle.Oracle(sub).observe(state64(rows, ag), 128, 256, sub_obs)
    # global roadgraph indices of the subset are renumbered: map back
    rg_map = np.concatenate([np.arange(b.rg_off[s], b.rg_off[s + 1]) for s in scenes])
    oo["rg_idx"] = np.where(oo["rg_idx"] >= 0, rg_map[np.maximum(oo["rg_idx"], 0)], -1)
    go_sub = {k: v[ag] for k, v in go.items()}
    _check(go_sub, oo, np.nonzero(sub_obs)[0], 128, 256)


def _sampled_check(go, b, rows, scenes, M, K, observers=None):
    sub = b.subset(scenes)
    ag = np.concatenate([np.arange(b.agent_off[s], b.agent_off[s + 1]) for s in scenes])
    sub_obs = None if observers is None else observers[ag]
    oo = oracle.Oracle(sub).observe(state64(rows, ag), M, K, sub_obs)
    rg_map = np.concatenate([np.arange(b.rg_off[s], b.rg_off[s + 1]) for s in scenes])
    oo["rg_idx"] = np.where(oo["rg_idx"] >= 0, rg_map[np.maximum(oo["rg_idx"], 0)], -1)
    go_sub = {k: v[ag] for k, v in go.items()}
    obs = np.nonzero(sub.valid if sub_obs is None else sub_obs)[0]
    return _check(go_sub, oo, obs, M, K)


def test_every_agent_of_640_scenes_warp_per_observer(wsim):
    # 640 scenes x 128 agents, 20k-point roadgraphs: ~74,000 observers, well
    # above the warp kernel's threshold (one observer per resident warp, 5 x 8
    # warps per SM).  Scene 0: 600 points stacked
    # 0.5 m ahead of its ego (the K-th key shared by more points than a warp
    # gathers: that observer goes to the block kernel).  Scene 1: one point of
    # each of 200 tiles within 0.3-0.5 m of its ego (more candidate tiles than a
    # warp lists: every tile re-tested).  Scenes 2 and 3: no valid point, and
    # fewer valid points than K.
    b = synth.make_batch(1, seed=7, scenes=range(640))
    for s in (0, 1):
        assert b.valid[b.agent_off[s]]
    xe, ye = float(b.x[b.agent_off[0]]), float(b.y[b.agent_off[0]])
    r0 = int(b.rg_off[0])
    b.rg_x[r0 + 100:r0 + 700] = np.float32(xe + 0.5)
    b.rg_y[r0 + 100:r0 + 700] = np.float32(ye)
    b.rg_valid[r0 + 100:r0 + 700] = 1
    xe1, ye1 = float(b.x[b.agent_off[1]]), float(b.y[b.agent_off[1]])
    r1 = int(b.rg_off[1])
    for t in range(200):
        ang, rad = 2 * np.pi * t / 200, 0.3 + 0.001 * t
        b.rg_x[r1 + 32 * t] = np.float32(xe1 + rad * np.cos(ang))
        b.rg_y[r1 + 32 * t] = np.float32(ye1 + rad * np.sin(ang))
        b.rg_valid[r1 + 32 * t] = 1
    # Scene 2: no valid roadgraph point (every slot -1).  Scene 3: 40 valid
    # points, fewer than K (the rest of the slots -1).
    b.rg_valid[b.rg_off[2]:b.rg_off[3]] = 0
    r3 = int(b.rg_off[3])
    b.rg_valid[r3 + 40:b.rg_off[4]] = 0
    b.rg_valid[r3:r3 + 40] = 1
    rows = np.zeros((10, b.N_tot), np.float32)
    rows[0], rows[1], rows[4], rows[6], rows[7] = b.x, b.y, b.th, b.vx, b.vy
    assert b.valid.sum() > 148 * 40 * 11
    for K in (64, 256):
        go = _gpu_observe(wsim, b, rows, 128, K)
        # the ego of scene 0 sees the first K of the 600 tied points
        assert np.array_equal(go["rg_idx"][b.agent_off[0]][:K], np.arange(r0 + 100, r0 + 100 + K))
        obs2 = np.arange(b.agent_off[2], b.agent_off[3])[b.valid[b.agent_off[2]:b.agent_off[3]] != 0]
        assert (go["rg_idx"][obs2] == -1).all()
        obs3 = np.arange(b.agent_off[3], b.agent_off[4])[b.valid[b.agent_off[3]:b.agent_off[4]] != 0]
        assert (np.sort(go["rg_idx"][obs3][:, :40], axis=1) == np.arange(r3, r3 + 40)).all()
        assert (go["rg_idx"][obs3][:, 40:] == -1).all()
        err = _sampled_check(go, b, rows, [0, 1, 2, 3, 17, 639], 128, K)
        print("K", K, "max point error", err)
        assert (go["rg_idx"][b.valid == 0] == -1).all()


def test_observe_argument_limits(wsim):
    b = synth.make_batch(0, seed=1)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State.from_batch(b)
    with pytest.raises(wsim.WsimError):
        sim.observe(st, 16, 8)  # M below the scene's 32 agents
    with pytest.raises(wsim.WsimError):
        sim.observe(st, 32, 5000)  # K above the limit
    sim.close()
