"""Pins of the oracle's observation function (Sec. 3.2: other agents in the
agent's own frame, the roadgraph subsampled by distance).

Expected values come from hand-placed agents and points with known
coordinates in the observer's frame, from rigid motions of a whole scene,
from a round trip back to world coordinates, and from a brute-force float64
nearest-point ranking on point sets without near ties.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch


def _obs(b, M, K, observers=None, st=None):
    o = oracle.Oracle(b)
    return o.observe(o.initial_state() if st is None else st, M, K, observers)


def test_agents_in_frame_of_a_rotated_observer():
    # observer at (10, 5) heading +90 deg: world +y is its forward (+x),
    # world -x is its left... (+y in its frame is world -x)
    agents = [dict(x=10.0, y=5.0, th=np.pi / 2, v=2.0),
              dict(x=10.0, y=9.0, th=np.pi / 2, v=3.0),    # 4 m ahead
              dict(x=7.0, y=5.0, th=0.0, v=1.0),           # 3 m to its left, driving world +x
              dict(x=0.0, y=0.0, valid=0),
              dict(x=10.0, y=0.0, th=-3.0, v=0.0)]        # heading difference -3 - pi/2 wraps to pi/2 - 3 + pi
    b = tiny_batch(agents)
    out = _obs(b, M=5, K=1)
    a, v = out["agents"][0], out["agents_valid"][0]
    assert list(v) == [0, 1, 1, 0, 1]  # itself and the invalid agent are not observed
    assert a[4][2] == pytest.approx(-3.0 - np.pi / 2 + 2 * np.pi)
    np.testing.assert_allclose(a[4][:2], [-5.0, 0.0], atol=1e-6)
    np.testing.assert_allclose(a[1], [4.0, 0.0, 0.0, 3.0, 0.0], atol=1e-6)
    # world +x velocity is the observer's -y; heading 0 - pi/2
    np.testing.assert_allclose(a[2], [0.0, 3.0, -np.pi / 2, 0.0, -1.0], atol=1e-6)
    assert (a[0] == 0).all() and (a[3] == 0).all()


def test_round_trip_to_world_and_rigid_motion():
    rng = np.random.default_rng(0)
    b = synth.make_batch(0, seed=4, N=12, R=600)
    o = oracle.Oracle(b)
    st = o.initial_state()
    out = o.observe(st, 12, 32)
    for g in np.nonzero(b.valid)[0]:
        c, s = np.cos(st["th"][g]), np.sin(st["th"][g])
        for j in np.nonzero(out["agents_valid"][g])[0]:
            x, y = out["agents"][g, j, :2]
            np.testing.assert_allclose([st["x"][g] + c * x - s * y, st["y"][g] + s * x + c * y],
                                       [st["x"][j], st["y"][j]], atol=1e-9)
        for k, r in enumerate(out["rg_idx"][g]):
            x, y = out["rg"][g, k]
            np.testing.assert_allclose([st["x"][g] + c * x - s * y, st["y"][g] + s * x + c * y],
                                       [b.rg_x[r], b.rg_y[r]], atol=1e-9)
    # translate and rotate the whole scene: frames move with it
    ang, tx, ty = 0.7, 30.0, -12.0
    R = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
    b2 = synth.make_batch(0, seed=4, N=12, R=600)
    xy = R @ np.stack([b.x, b.y]).astype(np.float64) + [[tx], [ty]]
    st2 = dict(st, x=xy[0], y=xy[1], th=st["th"] + ang)
    vv = R @ np.stack([st["vx"], st["vy"]])
    st2["vx"], st2["vy"] = vv[0], vv[1]
    rxy = R @ np.stack([b.rg_x, b.rg_y]).astype(np.float64) + [[tx], [ty]]
    b2.rg_x, b2.rg_y = rxy[0], rxy[1]  # float64 arrays: the oracle takes them as is
    o2 = oracle.Oracle(b2)
    out2 = o2.observe(st2, 12, 32)
    np.testing.assert_allclose(out2["agents"], out["agents"], atol=1e-9)
    assert (out2["agents_valid"] == out["agents_valid"]).all()
    np.testing.assert_allclose(out2["rg"][b.valid != 0], out["rg"][b.valid != 0], atol=2e-5)


def test_nearest_points_against_brute_force_and_padding():
    # random points (no near ties): the oracle's K nearest equal a float64
    # argsort of the distances; with K beyond the valid points the rest is -1
    rng = np.random.default_rng(1)
    n = 300
    pts = rng.uniform(-50, 50, (n, 2))
    valid = rng.random(n) > 0.2
    b = tiny_batch([dict(x=1.5, y=-2.0, th=0.3, v=1.0)], roadgraph=[(pts, 2)])
    b.rg_valid = valid.astype(np.uint8)
    K = 40
    out = _obs(b, 1, K)
    d = np.hypot(pts[:, 0] - np.float32(1.5), pts[:, 1] - np.float32(-2.0))
    d[~valid] = np.inf
    order = np.argsort(d, kind="stable")[:K]
    gap = np.sort(d)[K] - np.sort(d)[K - 1]
    assert gap > 1e-3  # no near tie at the boundary
    assert list(out["rg_idx"][0]) == list(order)
    big = _obs(b, 1, n + 5)
    idx = big["rg_idx"][0]
    assert (idx[: valid.sum()] >= 0).all() and (idx[valid.sum():] == -1).all()
    assert set(idx[: valid.sum()]) == set(np.nonzero(valid)[0])


def test_ties_go_to_the_lower_index_and_observer_mask():
    # four points at the same distance around the observer: index order
    pts = np.array([[0.0, 5.0], [5.0, 0.0], [0.0, -5.0], [-5.0, 0.0], [9.0, 0.0]])
    b = tiny_batch([dict(x=0.0, y=0.0, th=0.0, v=0.0), dict(x=1.0, y=1.0, th=0.0, v=0.0)],
                   roadgraph=[(pts, 1)])
    out = _obs(b, 2, 3)
    assert list(out["rg_idx"][0]) == [0, 1, 2]
    only = _obs(b, 2, 3, observers=np.array([0, 1], np.uint8))
    assert (only["rg_idx"][0] == -1).all() and (only["agents_valid"][0] == 0).all()  # not an observer
    assert only["rg_idx"][1][0] >= 0
