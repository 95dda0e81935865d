"""CUDA path against the FP64 oracle, through the C ABI (needs a B300).

Teacher-forced parity per step and per quantity (positions 1e-5 m, heading
1e-6 rad, velocity 1e-5 m/s, log divergence 1e-5 m, overlap depth and
off-road distance 2e-5 m, or 4 float32 ulps of larger values); collision and
off-road booleans and the reward bit-exact outside the oracle's ambiguity
bands.  The four rollout modes must agree bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2310_08710_b300 import synth
from tests import gpu_harness as H
from tests.scenes import straight_route, tiny_batch

pytestmark = pytest.mark.gpu
SHAPES = 5  # launch shapes of the scene-resident rollout


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def test_single_scene_32_agents_every_step(wsim):
    b = synth.make_batch(0, seed=1)
    g = H.run_rollout(b)
    assert g["status"] == 0
    c = H.teacher_forced(b, g, [0], range(b.T))
    assert c["steps"] == 80
    print("single scene", c)


def test_single_scene_modes_bit_identical_and_deterministic(wsim):
    b = synth.make_batch(0, seed=2)
    ref = H.run_rollout(b, mode=wsim.MODE_FUSED)
    for mode in (wsim.MODE_FUSED, wsim.MODE_GRAPH, wsim.MODE_STREAM, wsim.MODE_PLAIN):
        g = H.run_rollout(b, mode=mode)
        for k in ("traj", "final", "ov", "off", "logdiv", "flags", "reward"):
            assert np.array_equal(g[k].view(np.uint8), ref[k].view(np.uint8)), (mode, k)


def test_batch_1024x128_idm_full_size_sampled_scenes(wsim):
    # Full 1024-scene batch in the benchmark's launch configuration (the
    # scene-resident rollout); the oracle checks a spread of scenes at every
    # step, and the per-step graph path must agree bit for bit.
    b = synth.make_batch(1, seed=0)
    g = H.run_rollout(b, mode=wsim.MODE_FUSED)
    gg = H.run_rollout(b, mode=wsim.MODE_GRAPH)
    for k in ("traj", "final", "ov", "off", "logdiv", "flags", "reward"):
        assert np.array_equal(g[k].view(np.uint8), gg[k].view(np.uint8)), k
    assert g["status"] == 0
    scenes = [0, 333, 700, 1023]
    c = H.teacher_forced(b, g, scenes, range(b.T))
    print("1024x128 IDM batch", c)
    assert c["band_idm"] <= 0.02 * c["agent_steps"]


def test_uneven_batch_against_plain_and_oracle(wsim):
    # Scenes of 1k-30k roadgraph points: the largest do not fit the
    # shared-memory stage and read their segments from global memory.
    b = synth.make_batch(2, seed=0, S=512)
    g = H.run_rollout(b, mode=wsim.MODE_FUSED)
    for mode in (wsim.MODE_GRAPH, wsim.MODE_PLAIN):
        p = H.run_rollout(b, mode=mode)
        for k in ("traj", "ov", "off", "logdiv", "flags", "reward"):
            assert np.array_equal(g[k].view(np.uint8), p[k].view(np.uint8)), (mode, k)
    rng = np.random.default_rng(0)
    scenes = sorted(rng.choice(b.S, 8, replace=False).tolist())
    big = int(np.argmax(np.diff(b.rg_off)))
    c = H.teacher_forced(b, g, sorted(set(scenes + [big])), [0, 1, 2, 17, 40, 79])
    print("uneven batch", c)


def test_roadgraph_gaps_and_short_runs(wsim):
    # Invalid points and type changes inside polylines split the road edges
    # into many runs of 1 to a few segments; every run starts its own culling
    # tile, with padding in between.  All launch shapes and the oracle agree.
    b = synth.make_batch(0, seed=5, S=1, R=4000)
    rng = np.random.default_rng(5)
    b.rg_valid = (rng.random(b.R_tot) > 0.12).astype(np.uint8)
    flip = rng.random(b.R_tot) < 0.05
    b.rg_type = np.where(flip, 1 - b.rg_type, b.rg_type).astype(np.uint8)
    g = H.run_rollout(b)
    assert g["status"] == 0
    for shape in range(SHAPES):
        p = H.run_rollout(b, tuning=dict(single_shape=shape))
        for k in ("traj", "off", "flags", "reward"):
            assert np.array_equal(g[k].view(np.uint8), p[k].view(np.uint8)), (shape, k)
    p = H.run_rollout(b, mode=wsim.MODE_PLAIN)
    assert np.array_equal(g["off"].view(np.uint8), p["off"].view(np.uint8))
    c = H.teacher_forced(b, g, [0], range(b.T))
    print("gaps and short runs", c)


def _fan_scene(seed, fans=60, T=4):
    """Road edges in fans: three polylines start at one point P and leave it
    at angles a, a + 45, a + 90 degrees; the polylines of all fans are
    shuffled, so their index order has nothing to do with where they lie.
    One parked agent per fan sits in the quadrant behind the fan, where
    every corner's nearest point on all three polylines is P itself: exact
    ties between segments of different polylines, whose sides differ
    (the lowest index decides, Sec. 3.4 road-edge side)."""
    rng = np.random.default_rng(seed)
    polys, agents = [], []
    side = int(np.ceil(np.sqrt(fans)))
    for f in range(fans):
        P = np.array([25.0 * (f % side), 25.0 * (f // side)]) + rng.uniform(-3, 3, 2)
        a = rng.uniform(-np.pi, np.pi)
        for d in (0.0, np.pi / 4, np.pi / 2):
            n = int(rng.integers(17, 41))
            k = np.arange(n)[:, None]
            polys.append((P + 0.5 * k * np.array([np.cos(a + d), np.sin(a + d)]), 1))
        phi = a + 1.25 * np.pi
        c = P + 3.6 * np.array([np.cos(phi), np.sin(phi)])
        agents.append(dict(x=c[0], y=c[1], th=phi, v=0.0, L=4.5, W=2.0))
    order = rng.permutation(len(polys))
    return tiny_batch(agents, roadgraph=[polys[i] for i in order], T=T)


def _tied_corners(b):
    """Corners (float64, at t0) whose nearest distance to the road edges is
    reached by segments of two or more polylines."""
    e = (b.rg_type == 1)
    same = e[:-1] & e[1:] & (b.rg_poly[:-1] == b.rg_poly[1:])
    a = np.stack([b.rg_x[:-1], b.rg_y[:-1]], 1)[same].astype(np.float64)
    z = np.stack([b.rg_x[1:], b.rg_y[1:]], 1)[same].astype(np.float64)
    pid = b.rg_poly[:-1][same]
    n = 0
    for i in range(b.N_tot):
        c, s = np.cos(float(b.th[i])), np.sin(float(b.th[i]))
        for u, v in ((1, 1), (1, -1), (-1, -1), (-1, 1)):
            px = float(b.x[i]) + u * 0.5 * float(b.L[i]) * c - v * 0.5 * float(b.W[i]) * s
            py = float(b.y[i]) + u * 0.5 * float(b.L[i]) * s + v * 0.5 * float(b.W[i]) * c
            d = z - a
            t = np.clip(((px - a[:, 0]) * d[:, 0] + (py - a[:, 1]) * d[:, 1]) / (d * d).sum(1), 0, 1)
            dist = np.hypot(a[:, 0] + t * d[:, 0] - px, a[:, 1] + t * d[:, 1] - py)
            n += len(set(pid[dist == dist.min()].tolist())) > 1
    return n


def test_ties_across_polylines_go_to_the_lower_index(wsim):
    # The off-road search visits super-tiles in spatial order, not index
    # order; equal distances must still resolve to the lowest segment index
    # in every launch path, as in the oracle's exhaustive scan.
    b = _fan_scene(3)
    assert _tied_corners(b) >= 200
    g = H.run_rollout(b)
    assert g["status"] == 0
    off = g["off"][0]
    assert (off > 0).sum() >= 10 and (off < 0).sum() >= 10  # both sides won ties
    for shape in range(SHAPES):
        p = H.run_rollout(b, tuning=dict(single_shape=shape))
        assert np.array_equal(g["off"].view(np.uint8), p["off"].view(np.uint8)), shape
    for mode in (wsim.MODE_GRAPH, wsim.MODE_PLAIN):
        p = H.run_rollout(b, mode=mode)
        assert np.array_equal(g["off"].view(np.uint8), p["off"].view(np.uint8)), mode
    c = H.teacher_forced(b, g, [0], range(b.T))
    print("ties across polylines", c)


def test_idm_far_from_origin_scene_resident_equals_per_step(wsim):
    # Far from the origin (float32 spacing 2-4 mm) the culling bounds of the
    # off-road, overlap and IDM searches work with large coordinates; the
    # scene-resident rollout and the per-step kernels must still give the
    # same bits.
    import copy
    b = copy.copy(synth.make_batch(1, seed=4, S=48, R=3000, T=24))
    for k, d in (("x", 3.1e4), ("y", -2.3e4)):
        for f in (k, "rg_" + k, "route_" + k, "log_" + k):
            setattr(b, f, (getattr(b, f).astype(np.float64) + d).astype(np.float32))
    g = H.run_rollout(b, mode=wsim.MODE_FUSED)
    assert g["status"] == 0
    gg = H.run_rollout(b, mode=wsim.MODE_GRAPH)
    for k in ("traj", "final", "ov", "off", "logdiv", "flags", "reward"):
        assert np.array_equal(g[k].view(np.uint8), gg[k].view(np.uint8)), k


def test_scene_beyond_the_tile_order_limit(wsim):
    # A scene of more than 4,096 culling tiles (70,000 road-edge points in
    # short polylines) keeps its tiles in index order for the super-tiles;
    # its neighbour scene is ordered.  Both against the oracle, and the
    # scene-resident rollout against the per-step kernels bit for bit.
    rng = np.random.default_rng(12)
    polys = []
    for p in range(3500):
        n = 20
        start = rng.uniform(0.0, 400.0, 2)
        h = rng.uniform(-np.pi, np.pi)
        k = np.arange(n)[:, None]
        polys.append((start + 0.5 * k * np.array([np.cos(h), np.sin(h)]), 1))
    agents = [dict(x=float(x), y=float(y), th=float(t), v=float(v))
              for x, y, t, v in zip(rng.uniform(50, 350, 12), rng.uniform(50, 350, 12),
                                   rng.uniform(-np.pi, np.pi, 12), rng.uniform(0, 10, 12))]
    big = tiny_batch(agents, roadgraph=polys, T=6)
    small = synth.make_batch(0, seed=12, S=1, N=12, R=3000, T=6)
    b = _concat([big, small], 6)
    g = H.run_rollout(b)
    assert g["status"] == 0
    gg = H.run_rollout(b, mode=wsim.MODE_GRAPH)
    for k in ("traj", "ov", "off", "flags", "reward"):
        assert np.array_equal(g[k].view(np.uint8), gg[k].view(np.uint8)), k
    c = H.teacher_forced(b, g, [0, 1], range(b.T))
    print("scene beyond the tile order limit", c)


def test_every_launch_configuration_bit_identical(wsim):
    # Uneven scenes span the three size buckets; every single launch shape
    # and every split configuration of the scene-resident rollout must give
    # the same bits as the per-step graph path.
    b = synth.make_batch(2, seed=7, S=96, T=12)
    sim = wsim.Sim(wsim.DeviceBatch(b))
    info = sim.get_tuning()
    sim.close()
    print("buckets", info)
    assert sum(info["bucket_scenes"]) == b.S and min(info["bucket_scenes"][:2]) > 0
    ref = H.run_rollout(b, mode=wsim.MODE_GRAPH)
    configs = [dict(split=False, single_shape=sh) for sh in range(SHAPES)]
    configs += [dict(split=True, bucket_shape=(sh, (sh + 1) % SHAPES, (sh + 2) % SHAPES)) for sh in range(SHAPES)]
    for tun in configs:
        g = H.run_rollout(b, mode=wsim.MODE_FUSED, tuning=tun)
        for k in ("traj", "final", "ov", "off", "logdiv", "flags", "reward"):
            assert np.array_equal(g[k].view(np.uint8), ref[k].view(np.uint8)), (tun, k)


def test_lean_and_full_kernels_bit_identical(wsim):
    # The rollout and step kernels are compiled twice: without the driver
    # array and without work counting (the benchmark's launches), and with
    # every driver and counting.  Both must give the same bits; the counted
    # run must count work in every category an IDM batch exercises.
    b = synth.make_batch(1, seed=11, S=24, R=4000, T=16)
    ctrl = np.full(b.N_tot, wsim.CTRL_ACTION, np.uint8)
    for mode in (wsim.MODE_FUSED, wsim.MODE_GRAPH):
        lean = H.run_rollout(b, mode=mode)
        counted = H.run_rollout(b, mode=mode, count=True)
        driven = H.run_rollout(b, mode=mode, ctrl=ctrl)
        for k in ("traj", "final", "ov", "off", "logdiv", "flags", "reward"):
            assert np.array_equal(lean[k].view(np.uint8), counted[k].view(np.uint8)), (mode, k)
            assert np.array_equal(lean[k].view(np.uint8), driven[k].view(np.uint8)), (mode, k)
        c = counted["counters"]
        print(mode, c)
        assert c[0] > 0 and c[1] > 0 and c[3] > 0 and c[4] > 0 and c[5] > 0, c


def test_autotune_keeps_results(wsim):
    import torch
    b = synth.make_batch(2, seed=8, S=64, T=10)
    db = wsim.DeviceBatch(b)
    sim = wsim.Sim(db)
    st = wsim.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().contiguous()
    res = sim.autotune(st, act, 10, 6)
    print("autotune", res)
    assert torch.equal(st.data, wsim.State.from_batch(b).data)  # input state untouched
    singles = [v for v in res["ms_single"] if v >= 0]
    chosen = res["ms_split"] if res["split"] else res["ms_single"][res["single_shape"]]
    assert len(singles) == SHAPES and chosen <= min(singles + ([res["ms_split"]] if res["ms_split"] >= 0 else []))
    tun = dict(split=res["split"], single_shape=res["single_shape"], bucket_shape=res["bucket_shape"])
    sim.close()
    g1 = H.run_rollout(b)
    g2 = H.run_rollout(b, tuning=tun)
    for k in ("traj", "ov", "off", "flags", "reward"):
        assert np.array_equal(g1[k].view(np.uint8), g2[k].view(np.uint8)), k


def test_large_scene_workload_delta_and_bicycle_egos_with_idm(wsim):
    # Scenes of the 16384 x 128 sweep workload (30k-point roadgraphs, delta
    # ego in the first half, bicycle ego in the second, 127 IDM agents); many
    # exceed the shared-memory stage and read their segments from L2.
    b = synth.make_batch(4, seed=0, S=256)
    g = H.run_rollout(b)
    assert g["status"] == 0
    big = int(np.argmax(np.diff(b.rg_off)))
    c = H.teacher_forced(b, g, sorted({0, 127, 128, 255, big}), [0, 1, 2, 39, 79])
    print("large-scene workload", c)
    assert c["band_idm"] <= 0.02 * c["agent_steps"]


def test_edge_cases_tiny_scenes(wsim):
    # scenes with 1 agent, 2 agents, no road edges, all agents invalid, an
    # empty scene, and a box touching an edge
    edge = np.stack([np.arange(-20, 20.5, 0.5), np.zeros(81)], 1)
    scenes = [
        tiny_batch([dict(x=0.0, y=1.0, th=0.2, v=3.0)], roadgraph=[(edge, 1)]),
        tiny_batch([dict(x=0.0, y=3.0, v=5.0), dict(x=3.0, y=3.5, th=0.3, v=1.0)], roadgraph=[(edge, 2)]),
        tiny_batch([dict(x=0.0, y=1.0, valid=0), dict(x=3.0, y=1.0, valid=0)], roadgraph=[(edge, 1)]),
    ]
    b = _concat(scenes + [_empty_scene()], T=20)
    g = H.run_rollout(b)
    assert g["status"] == 0
    H.teacher_forced(b, g, list(range(b.S)), range(b.T))
    assert np.isneginf(g["ov"][0][0])                    # a lone agent has no pair
    assert np.isneginf(g["off"][0][1]) and np.isneginf(g["off"][0][2])  # no road edge
    assert (g["ov"][:, 3:5] == 0).all() and (g["flags"][:, 3:5] == 0).all()  # invalid agents


def test_max_agents_per_scene(wsim):
    b = synth.make_batch(0, seed=4, N=256, S=2, R=3000)
    g = H.run_rollout(b, T=12)
    H.teacher_forced(b, g, [0, 1], range(12))
    bad = synth.make_batch(0, seed=4, N=257, S=1, R=100)
    with pytest.raises(wsim.WsimError) as e:
        wsim.Sim(wsim.DeviceBatch(bad))
    assert e.value.code == wsim.ESIZE


def test_max_road_edge_segments_per_scene(wsim):
    # one straight road edge: n points give n - 1 segments in one run, padded
    # to a multiple of 16; 2^20 packed positions is the limit of a scene
    # (16-bit tile indexes in the candidate-tile lists)
    for n_seg, ok in ((1 << 20, True), ((1 << 20) + 1, False)):
        xs = np.arange(n_seg + 1, dtype=np.float64) * 0.01
        b = tiny_batch([dict(x=5.0, y=1.0, th=0.0, v=1.0), dict(x=9000.0, y=-2.0, th=0.5, v=2.0)],
                       roadgraph=[(np.stack([xs, np.zeros_like(xs)], 1), 1)], T=4)
        if ok:
            g = H.run_rollout(b, T=4)
            H.teacher_forced(b, g, [0], range(4))
        else:
            with pytest.raises(wsim.WsimError) as e:
                wsim.Sim(wsim.DeviceBatch(b))
            assert e.value.code == wsim.ESIZE


def test_idm_scene_with_routes_every_step(wsim):
    b = synth.make_batch(1, seed=3, S=6, R=4000)
    g = H.run_rollout(b)
    c = H.teacher_forced(b, g, list(range(6)), range(b.T))
    print("idm", c)
    assert c["band_idm"] <= 0.02 * c["agent_steps"]


def test_idm_routes_with_uneven_point_spacing(wsim):
    # The lead search bounds each group of look-ahead samples by the route's
    # largest segment length per route parameter (computed at init): routes
    # whose segments are stretched 0.4x to 4x (the parameter still counts
    # 0.5 m per segment) must give the oracle's leads.
    b = synth.make_batch(1, seed=8, S=6, R=4000)
    rng = np.random.default_rng(8)
    for g in range(b.N_tot):
        r0, r1 = b.route_off[g], b.route_off[g + 1]
        if r1 - r0 < 2:
            continue
        x = b.route_x[r0:r1].astype(np.float64)
        y = b.route_y[r0:r1].astype(np.float64)
        f = rng.uniform(0.4, 4.0, r1 - r0 - 1)
        b.route_x[r0 + 1:r1] = (x[0] + np.cumsum(np.diff(x) * f)).astype(np.float32)
        b.route_y[r0 + 1:r1] = (y[0] + np.cumsum(np.diff(y) * f)).astype(np.float32)
    g = H.run_rollout(b)
    assert g["status"] == 0
    gg = H.run_rollout(b, mode=wsim.MODE_GRAPH)
    for k in ("traj", "ov", "off", "flags"):
        assert np.array_equal(g[k].view(np.uint8), gg[k].view(np.uint8)), k
    c = H.teacher_forced(b, g, list(range(b.S)), range(b.T))
    print("idm, stretched routes", c)
    assert c["band_idm"] <= 0.02 * c["agent_steps"]


def test_ctrl_mask_and_nonfinite_status(wsim):
    b = synth.make_batch(0, seed=5)
    ctrl = (np.arange(b.N_tot) % 3 != 0).astype(np.uint8)
    g = H.run_rollout(b, ctrl=ctrl, T=5)
    r0 = H.initial_rows(b)
    held = ctrl == 0
    assert np.array_equal(g["traj"][:, 4, held], r0[:, held])
    b.actions[2, 0, 5] = np.nan
    g = H.run_rollout(b, T=5)
    assert g["status"] == wsim.ENONFINITE


def _empty_scene():
    b = tiny_batch([dict(x=0.0, y=0.0)])
    return synth.SceneBatch(**{**b.__dict__, "N_tot": 0, "agent_off": np.array([0, 0], np.int32),
                               "L": b.L[:0], "W": b.W[:0], "valid": b.valid[:0], "kind": b.kind[:0],
                               "idm_v0": b.idm_v0[:0], "route_off": np.zeros(1, np.int32),
                               "log_x": b.log_x[:, :0], "log_y": b.log_y[:, :0], "x": b.x[:0], "y": b.y[:0],
                               "th": b.th[:0], "vx": b.vx[:0], "vy": b.vy[:0], "actions": b.actions[:, :, :0]})


def _concat(bs, T):
    """Concatenate single-scene batches; random actions for T steps."""
    rng = np.random.default_rng(0)
    cat = lambda k: np.concatenate([getattr(x, k) for x in bs])
    off = lambda n: np.concatenate([[0], np.cumsum(n)]).astype(np.int32)
    N = [x.N_tot for x in bs]
    R = [x.R_tot for x in bs]
    rt = [int(x.route_off[-1]) for x in bs]
    route_off = np.concatenate([[0]] + [x.route_off[1:] + sum(rt[:i]) for i, x in enumerate(bs)]).astype(np.int32)
    polys = np.concatenate([x.rg_poly + 1000 * i for i, x in enumerate(bs)]).astype(np.int32)
    act = np.stack([rng.uniform(-4, 4, (T, sum(N))), rng.uniform(-0.3, 0.3, (T, sum(N))),
                    np.zeros((T, sum(N)))], 1).astype(np.float32)
    return synth.SceneBatch(
        cfg=-1, seed=0, scenes=np.arange(len(bs)), S=len(bs), N_tot=sum(N), T=T,
        agent_off=off(N), rg_off=off(R), L=cat("L"), W=cat("W"), valid=cat("valid"), kind=cat("kind"),
        idm_v0=cat("idm_v0"), route_off=route_off, route_x=cat("route_x"), route_y=cat("route_y"),
        rg_x=cat("rg_x"), rg_y=cat("rg_y"), rg_poly=polys, rg_type=cat("rg_type"), rg_valid=cat("rg_valid"),
        log_x=np.concatenate([x.log_x for x in bs], 1), log_y=np.concatenate([x.log_y for x in bs], 1),
        x=cat("x"), y=cat("y"), th=cat("th"), vx=cat("vx"), vy=cat("vy"), actions=act)
