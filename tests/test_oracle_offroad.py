"""Pins of the oracle's off-road signed distance (Sec. 3.4, off-road).

Expected values: closed-form distances to a straight edge, to a circle and
to a square; point-in-polygon for the sign; a dense sampling of every
road-edge segment for the distance; orientation reversal and rigid motion.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch


def _o(polylines):
    b = tiny_batch([dict(x=0, y=0)], roadgraph=[(p, 1) for p in polylines])
    return oracle.Oracle(b)


def test_straight_edge_along_x():
    pts = np.stack([np.arange(0, 50.5, 0.5), np.zeros(101)], 1)
    o = _o([pts])
    rng = np.random.default_rng(0)
    for _ in range(200):
        px, py = rng.uniform(1, 49), rng.uniform(-10, 10)
        sd, amb, _ = o.point_sd(0, px, py)
        assert abs(sd - (-py)) < 1e-12 and not amb


def test_open_end_uses_segment_side():
    pts = np.array([[0.0, 0.0], [1.0, 0.0]])
    o = _o([pts])
    sd, _, _ = o.point_sd(0, 3.0, 4.0)  # beyond the end: distance to the end point
    assert abs(sd - (-np.hypot(2.0, 4.0))) < 1e-12
    sd, _, _ = o.point_sd(0, 3.0, -4.0)
    assert abs(sd - np.hypot(2.0, 4.0)) < 1e-12


@pytest.mark.parametrize("r", [10.0, 37.0, 100.0])
def test_arc_edge_matches_circle(r):
    # counter-clockwise circle: the left side (the road) is the inside
    n = int(np.ceil(2 * np.pi * r / 0.5))
    dphi = 2 * np.arcsin(0.25 / r)
    k = np.arange(int(np.pi / dphi))  # half circle
    pts = np.stack([r * np.cos(k * dphi), r * np.sin(k * dphi)], 1)
    o = _o([pts.astype(np.float32)])
    sag = 0.5 ** 2 / (8 * r)
    rng = np.random.default_rng(1)
    for _ in range(200):
        ang = rng.uniform(0.2, np.pi - 0.2)
        rad = rng.uniform(r - 5, r + 5)
        sd, amb, _ = o.point_sd(0, rad * np.cos(ang), rad * np.sin(ang))
        assert abs(sd - (rad - r)) < sag + 1e-5


def _square(ccw=True, s=1.0):
    # start in the middle of the bottom side so that the open ends are collinear
    p = [(0, -s), (s, -s), (s, s), (-s, s), (-s, -s), (0, -s)]
    p = np.array(p, dtype=np.float64)
    return p if ccw else p[::-1].copy()


@pytest.mark.parametrize("ccw", [True, False])
def test_square_vertices_sign_and_distance(ccw):
    # Road on the left: inside of a CCW square, outside of a CW one.  Covers
    # left-turn (convex) and right-turn (reflex) vertices.
    o = _o([_square(ccw, 2.0)])
    rng = np.random.default_rng(2)
    for _ in range(2000):
        x, y = rng.uniform(-4, 4, 2)
        if abs(x) < 0.2 and y < -1.5:
            continue  # near the collinear open ends
        dx, dy = abs(x) - 2, abs(y) - 2
        inside = dx < 0 and dy < 0
        dist = -max(dx, dy) if inside else np.hypot(max(dx, 0), max(dy, 0))
        if dist < 1e-6:
            continue
        exp = (-dist if inside else dist) * (1 if ccw else -1)
        sd, amb, _ = o.point_sd(0, x, y)
        assert abs(sd - exp) < 1e-12, (x, y, sd, exp)


def test_reversal_flips_sign_and_rigid_motion():
    b = synth.make_batch(0, seed=3)
    o = oracle.Oracle(b)
    # reverse every road-edge polyline
    rx, ry = b.rg_x.copy(), b.rg_y.copy()
    for pid in np.unique(b.rg_poly):
        idx = np.nonzero(b.rg_poly == pid)[0]
        rx[idx], ry[idx] = rx[idx][::-1], ry[idx][::-1]
    br = synth.SceneBatch(**{**b.__dict__, "rg_x": rx, "rg_y": ry})
    orv = oracle.Oracle(br)
    rot, tx, ty = 1.1, -50.0, 20.0
    c, s = np.cos(rot), np.sin(rot)
    gx = (c * b.rg_x.astype(np.float64) - s * b.rg_y + tx)
    gy = (s * b.rg_x.astype(np.float64) + c * b.rg_y + ty)
    # keep the moved roadgraph in float64 by bypassing the float32 fields
    bm = synth.SceneBatch(**{**b.__dict__, "rg_x": gx, "rg_y": gy})
    om = oracle.Oracle(bm)
    rng = np.random.default_rng(4)
    n = 0
    for _ in range(300):
        px, py = rng.uniform(0, 200, 2)
        sd, amb, _ = o.point_sd(0, px, py)
        sdr, ambr, _ = orv.point_sd(0, px, py)
        sdm, ambm, _ = om.point_sd(0, c * px - s * py + tx, s * px + c * py + ty)
        if amb or ambr or abs(sd) < 1e-6:
            continue
        n += 1
        assert abs(sd + sdr) < 1e-9
        assert abs(sd - sdm) < 1e-9
    assert n > 250


def test_distance_matches_dense_sampling():
    # |sd| equals the distance to the nearest of many points sampled on every
    # road-edge segment, within the sampling resolution.
    b = synth.make_batch(0, seed=5)
    o = oracle.Oracle(b)
    x, y, p, t = (b.rg_x.astype(np.float64), b.rg_y.astype(np.float64), b.rg_poly, b.rg_type)
    seg = np.nonzero((t[:-1] == 1) & (t[1:] == 1) & (p[:-1] == p[1:]))[0]
    u = np.linspace(0, 1, 65)
    sx = (x[seg, None] + u[None] * (x[seg + 1] - x[seg])[:, None]).ravel()
    sy = (y[seg, None] + u[None] * (y[seg + 1] - y[seg])[:, None]).ravel()
    rng = np.random.default_rng(6)
    for _ in range(100):
        px, py = rng.uniform(0, 200, 2)
        sd, _, _ = o.point_sd(0, px, py)
        dense = np.min(np.hypot(sx - px, sy - py))
        assert abs(sd) <= dense + 1e-9
        assert dense - abs(sd) <= 0.5 / 64 / 2 + 1e-9


def test_no_edges_gives_minus_inf_and_metrics_corners():
    o = _o([])
    sd, amb, seg = o.point_sd(0, 1.0, 1.0)
    assert sd == -np.inf and seg == -1
    # agent metrics: off = max over the four corners (box across a straight edge)
    pts = np.stack([np.arange(-20, 20.5, 0.5), np.zeros(81)], 1)
    b = tiny_batch([dict(x=0.0, y=0.5, th=0.0, L=4.0, W=2.0)], roadgraph=[(pts, 1)])
    ob = oracle.Oracle(b)
    m = ob.metrics(ob.initial_state(), 10)
    assert abs(m["off"][0] - 0.5) < 1e-9  # lowest corners at y = -0.5
    assert m["flags"][0] & 2
    # lane polylines (type 2) are not road edges
    b2 = tiny_batch([dict(x=0.0, y=0.5)], roadgraph=[(pts, 2)])
    o2 = oracle.Oracle(b2)
    assert o2.metrics(o2.initial_state(), 10)["off"][0] == -np.inf


def _tri_truth(P, x, y):
    """Signed distance to a triangle boundary (inside negative), independently."""
    from tests.test_oracle_overlap import seg_point_dist
    d = min(seg_point_dist((x, y), P[i], P[(i + 1) % 3]) for i in range(3))
    def cr(u, w):
        return u[0] * w[1] - u[1] * w[0]
    s = [cr(np.subtract(P[(i + 1) % 3], P[i]), np.subtract((x, y), P[i])) for i in range(3)]
    inside = all(v > 0 for v in s) or all(v < 0 for v in s)
    return -d if inside else d


@pytest.mark.parametrize("ccw", [True, False])
def test_acute_triangle_sharp_turns(ccw):
    # Turns sharper than 90 degrees: vertex regions where exactly one adjacent
    # segment has the point on its left.  Start mid-edge so the open ends are
    # collinear.
    A, B, Cc = (0.0, 0.0), (10.0, 1.0), (1.0, 3.0)
    M = (0.5 * (A[0] + B[0]), 0.5 * (A[1] + B[1]))
    poly = np.array([M, B, Cc, A, M])
    if not ccw:
        poly = poly[::-1].copy()
    o = _o([poly])
    rng = np.random.default_rng(8)
    n = 0
    for _ in range(3000):
        x, y = rng.uniform(-3, 13), rng.uniform(-3, 6)
        if np.hypot(x - M[0], y - M[1]) < 0.3:
            continue
        tr = _tri_truth([A, B, Cc], x, y)
        if abs(tr) < 1e-6:
            continue
        exp = tr if ccw else -tr
        sd, _, _ = o.point_sd(0, x, y)
        assert abs(sd - exp) < 1e-9, (x, y, sd, exp)
        n += 1
    assert n > 2900


def test_tie_goes_to_lower_index_and_opposite_signs_are_ambiguous():
    # Two parallel edges 2 m apart, both oriented +x: a point midway is on
    # the left (road) of the lower one and on the right of the upper one.
    xs = np.arange(0, 10.5, 0.5)
    low = np.stack([xs, -np.ones_like(xs)], 1)
    high = np.stack([xs, np.ones_like(xs)], 1)
    o = _o([low, high])
    sd, amb, seg = o.point_sd(0, 5.25, 0.0)
    assert seg == 10 and abs(sd + 1.0) < 1e-12 and amb
    o2 = _o([high, low])  # same geometry, other index order
    sd2, amb2, seg2 = o2.point_sd(0, 5.25, 0.0)
    assert seg2 == 10 and abs(sd2 - 1.0) < 1e-12 and amb2
    # clearly nearer to one edge: no ambiguity
    sd3, amb3, _ = o.point_sd(0, 5.25, 0.3)
    assert not amb3 and abs(sd3 - 0.7) < 1e-12
