"""Pins of the oracle's box overlap (Sec. 3.4, collision) against brute force.

Expected values come from an independent polygon-clipping routine
(Sutherland-Hodgman, 1974) and polygon distances written here, from the
interval closed form for axis-aligned boxes, and from symmetries of the
definition.
"""
import numpy as np
import pytest

import oracle
from tests.scenes import tiny_batch


def corners(b):
    x, y, th, L, W = b
    c, s = np.cos(th), np.sin(th)
    pts = []
    for sl, sw in ((1, 1), (-1, 1), (-1, -1), (1, -1)):  # counter-clockwise
        pts.append((x + sl * L / 2 * c - sw * W / 2 * s, y + sl * L / 2 * s + sw * W / 2 * c))
    return pts


def clip_area(A, B):
    """Area of the intersection of two convex CCW polygons (Sutherland-Hodgman)."""
    out = list(A)
    n = len(B)
    for i in range(n):
        if not out:
            break
        p, q = B[i], B[(i + 1) % n]
        inp, out = out, []
        inside = lambda r: (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0]) >= 0
        for j in range(len(inp)):
            cur, prv = inp[j], inp[j - 1]
            if inside(cur):
                if not inside(prv):
                    out.append(_isect(prv, cur, p, q))
                out.append(cur)
            elif inside(prv):
                out.append(_isect(prv, cur, p, q))
    if len(out) < 3:
        return 0.0
    a = 0.0
    for j in range(len(out)):
        a += out[j - 1][0] * out[j][1] - out[j][0] * out[j - 1][1]
    return 0.5 * a


def _isect(a, b, p, q):
    d1 = (b[0] - a[0], b[1] - a[1])
    d2 = (q[0] - p[0], q[1] - p[1])
    den = d1[0] * d2[1] - d1[1] * d2[0]
    t = ((p[0] - a[0]) * d2[1] - (p[1] - a[1]) * d2[0]) / den
    return (a[0] + t * d1[0], a[1] + t * d1[1])


def seg_point_dist(p, a, b):
    ab = np.subtract(b, a)
    t = np.clip(np.dot(np.subtract(p, a), ab) / np.dot(ab, ab), 0, 1)
    return np.hypot(*(np.subtract(p, a) - t * ab))


def poly_dist(A, B):
    """Distance between disjoint convex polygons: min of vertex-edge distances."""
    d = np.inf
    for P, Q in ((A, B), (B, A)):
        for p in P:
            for i in range(len(Q)):
                d = min(d, seg_point_dist(p, Q[i], Q[(i + 1) % len(Q)]))
    return d


def rand_box(rng, spread=6.0):
    return (rng.uniform(-spread, spread), rng.uniform(-spread, spread), rng.uniform(-np.pi, np.pi),
            rng.uniform(4, 5.5), rng.uniform(1.8, 2.2))


def test_overlap_sign_matches_clipping_area():
    rng = np.random.default_rng(0)
    n_over = n_sep = 0
    for _ in range(3000):
        A, B = rand_box(rng), rand_box(rng)
        d = oracle.box_depth(A, B)
        if abs(d) < 1e-4:
            continue
        area = clip_area(corners(A), corners(B))
        assert (area > 1e-12) == (d > 0), (A, B, d, area)
        n_over += d > 0
        n_sep += d <= 0
    assert n_over > 200 and n_sep > 200


def test_axis_aligned_interval_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(500):
        L1, W1, L2, W2 = rng.uniform(1, 6, 4)
        dx, dy = rng.uniform(-8, 8, 2)
        ex = min((L1 + L2) / 2 - abs(dx), (W1 + W2) / 2 - abs(dy))
        d = oracle.box_depth((3.0, -2.0, 0.0, L1, W1), (3.0 + dx, -2.0 + dy, 0.0, L2, W2))
        assert abs(d - ex) < 1e-12
        # the same pair with B rotated by 90 degrees and L/W swapped
        d2 = oracle.box_depth((3.0, -2.0, 0.0, L1, W1), (3.0 + dx, -2.0 + dy, np.pi / 2, W2, L2))
        assert abs(d2 - ex) < 1e-12


def test_symmetry_rigid_motion_and_swap():
    rng = np.random.default_rng(2)
    for _ in range(500):
        A, B = rand_box(rng), rand_box(rng)
        d = oracle.box_depth(A, B)
        assert abs(d - oracle.box_depth(B, A)) < 1e-12
        r, tx, ty = rng.uniform(-np.pi, np.pi), rng.uniform(-300, 300), rng.uniform(-300, 300)
        c, s = np.cos(r), np.sin(r)
        mv = lambda q: (c * q[0] - s * q[1] + tx, s * q[0] + c * q[1] + ty, q[2] + r, q[3], q[4])
        assert abs(d - oracle.box_depth(mv(A), mv(B))) < 1e-9
        sw = lambda q: (q[0], q[1], q[2] + np.pi / 2, q[4], q[3])
        assert abs(d - oracle.box_depth(sw(A), B)) < 1e-12
        assert abs(d - oracle.box_depth((A[0], A[1], A[2] + np.pi, A[3], A[4]), B)) < 1e-12


def test_separated_depth_bounds_polygon_distance():
    rng = np.random.default_rng(3)
    cnt = 0
    for _ in range(1500):
        A, B = rand_box(rng, 9), rand_box(rng, 9)
        d = oracle.box_depth(A, B)
        if d >= -1e-9:
            continue
        cnt += 1
        dist = poly_dist(corners(A), corners(B))
        assert -d <= dist + 1e-12
        # the largest separating gap of two rectangles is attained on an edge
        # normal when the closest features are an edge and a vertex
    assert cnt > 500


def test_overlap_depth_is_translation_to_separate_axis_aligned():
    # For axis-aligned boxes the depth is the minimum translation distance:
    # moving B by d along the shallower axis makes the clipped area vanish.
    A = (0.0, 0.0, 0.0, 4.0, 2.0)
    B = (3.0, 0.5, 0.0, 4.0, 2.0)
    d = oracle.box_depth(A, B)
    assert abs(d - 1.0) < 1e-12
    assert clip_area(corners(A), corners((3.0 + d + 1e-9, 0.5, 0.0, 4.0, 2.0))) == 0.0
    assert clip_area(corners(A), corners((3.0 + d - 1e-3, 0.5, 0.0, 4.0, 2.0))) > 0.0


def test_metrics_collision_flags_and_band():
    # Scene metrics: ov_i = max_j d_ij over valid j; invalid agents report 0.
    agents = [dict(x=0, y=0, th=0, L=4, W=2), dict(x=3, y=0, th=0, L=4, W=2),
              dict(x=30, y=0, th=0, L=4, W=2), dict(x=1, y=0, th=0, L=4, W=2, valid=0),
              dict(x=34.00005, y=0, th=0, L=4, W=2)]
    b = tiny_batch(agents)
    o = oracle.Oracle(b)
    m = o.metrics(o.initial_state(), 10)
    assert abs(m["ov"][0] - 1.0) < 1e-12 and abs(m["ov"][1] - 1.0) < 1e-12
    assert m["flags"][0] & 1 and m["flags"][1] & 1
    assert m["ov"][3] == 0 and m["flags"][3] == 0
    assert not m["flags"][2] & 1 and m["flags"][2] & 4  # touching within the band
    assert m["reward"][0] == -sum(int(f & 1) + int((f >> 1) & 1) for f in m["flags"])
    # a lone valid agent has no pair: ov = -inf
    o1 = oracle.Oracle(tiny_batch([dict(x=0, y=0)]))
    assert o1.metrics(o1.initial_state(), 10)["ov"][0] == -np.inf


def test_log_divergence_uses_the_same_time_step():
    # Log row t is (t, -t): the divergence at step t is the distance to it.
    log = np.zeros((91, 2, 2))
    log[:, :, 0] = np.arange(91)[:, None]
    log[:, :, 1] = -np.arange(91)[:, None]
    b = tiny_batch([dict(x=3.0, y=4.0), dict(x=50.0, y=-7.0, valid=0)], log=log)
    o = oracle.Oracle(b)
    st = o.initial_state()
    for t in (0, 10, 37, 90):
        m = o.metrics(st, t)
        assert abs(m["logdiv"][0] - np.hypot(3.0 - t, 4.0 + t)) < 1e-12
        assert m["logdiv"][1] == 0.0
