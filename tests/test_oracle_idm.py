"""Pins of the oracle's IDM route-following agent (Sec. 3.5).

The paper names the Intelligent Driver Model (Treiber, Hennecke, Helbing 2000)
without equations.  Expected values here are the textbook model's defining
properties: free-road acceleration a(1 - (v/v0)^4) (zero at the desired
speed), the steady-state car-following gap s_e = (s0 + vT)/sqrt(1 - (v/v0)^4)
at which a follower at the leader's speed does not accelerate, a standing
vehicle accelerating only beyond the minimum gap s0, plus the geometry of the
route (pose on the polyline, heading of its segment) and of the lead search.
"""
import numpy as np

import oracle
from tests.scenes import straight_route, tiny_batch

AMAX, B, TH, S0, DT = 2.0, 3.0, 1.5, 2.0, 0.1


def _scene(follower, others=(), route=None):
    agents = [dict(follower, kind=2)] + [dict(o) for o in others]
    route = straight_route(follower["x"], follower["y"], follower.get("th", 0.0)) if route is None else route
    return tiny_batch(agents, routes={0: route})


def _state(v_list, pos, th):
    n = len(v_list)
    st = dict(x=np.array([p[0] for p in pos], float), y=np.array([p[1] for p in pos], float),
              th=np.array(th, float), vx=np.array(v_list, float) * np.cos(th),
              vy=np.array(v_list, float) * np.sin(th), s=np.zeros(n))
    return st


def _step(b, st):
    o = oracle.Oracle(b)
    return o.transition(st, np.zeros((3, b.N_tot)))


def test_free_road_at_desired_speed_and_from_rest():
    b = _scene(dict(x=0.0, y=0.0, th=0.0, v0=10.0))
    s1, band, lead = _step(b, _state([10.0], [(0, 0)], [0.0]))
    assert lead[0] == -1 and not band[0]
    assert abs(np.hypot(s1["vx"][0], s1["vy"][0]) - 10.0) < 1e-12
    assert abs(s1["s"][0] - 1.0) < 1e-12 and abs(s1["x"][0] - 1.0) < 1e-12 and abs(s1["y"][0]) < 1e-12
    s1, _, _ = _step(b, _state([0.0], [(0, 0)], [0.0]))
    assert abs(s1["vx"][0] - AMAX * DT) < 1e-12
    assert abs(s1["s"][0] - 0.5 * AMAX * DT * DT) < 1e-12


def test_equilibrium_gap_gives_zero_acceleration():
    for v, v0 in ((8.0, 10.0), (5.0, 12.0), (11.0, 14.0)):
        se = (S0 + v * TH) / np.sqrt(1 - (v / v0) ** 4)
        L = 4.5
        b = _scene(dict(x=0.0, y=0.0, v0=v0, L=L), [dict(x=0.0, y=0.0, L=L)])
        st = _state([v, v], [(0, 0), (se + L, 0)], [0.0, 0.0])
        s1, band, lead = _step(b, st)
        assert lead[0] == 1 and not band[0]
        assert abs(np.hypot(s1["vx"][0], s1["vy"][0]) - v) < 1e-12


def test_standing_vehicle_accelerates_only_beyond_min_gap():
    L = 4.0
    for g, a_exp in ((S0, 0.0), (4.0, AMAX * (1 - (S0 / 4.0) ** 2)), (8.0, AMAX * (1 - (S0 / 8.0) ** 2))):
        b = _scene(dict(x=0.0, y=0.0, v0=10.0, L=L), [dict(x=0.0, y=0.0, L=L)])
        s1, _, lead = _step(b, _state([0.0, 0.0], [(0, 0), (g + L, 0)], [0.0, 0.0]))
        assert lead[0] == 1
        assert abs(s1["vx"][0] - max(0.0, a_exp * DT)) < 1e-12
    # closer than s0: braking demand, speed stays at zero
    b = _scene(dict(x=0.0, y=0.0, v0=10.0, L=L), [dict(x=0.0, y=0.0, L=L)])
    s1, _, _ = _step(b, _state([0.0, 0.0], [(0, 0), (1.0 + L, 0)], [0.0, 0.0]))
    assert s1["vx"][0] == 0.0 and s1["s"][0] == 0.0


def test_hard_braking_clamps_speed_at_zero():
    L = 4.5
    b = _scene(dict(x=0.0, y=0.0, v0=15.0, L=L), [dict(x=0.0, y=0.0, L=L)])
    s1, _, lead = _step(b, _state([15.0, 0.0], [(0, 0), (3.0 + L, 0)], [0.0, 0.0]))
    assert lead[0] == 1 and s1["vx"][0] == 0.0
    assert abs(s1["s"][0] - 0.5 * 15.0 * DT) < 1e-12


def test_lead_search_geometry():
    L, W = 4.5, 2.0
    f = dict(x=0.0, y=0.0, v0=10.0, L=L, W=W)
    cases = [
        ([(-10.0, 0.0, 0.0)], -1),                      # behind
        ([(20.0, 5.0, 0.0)], -1),                       # beside the lane
        ([(40.0, 0.0, 0.0), (20.0, 0.0, 0.0)], 2),      # nearer of two ahead
        ([(70.0, 0.0, 0.0)], -1),                       # beyond the 64 m look-ahead
        ([(15.0, 0.0, np.pi / 2)], 1),                  # crossing in front
        ([(20.0, 1.9, 0.0)], 1),                        # widened by half the follower's width
    ]
    for others, exp in cases:
        ag = [dict(x=o[0], y=o[1], th=o[2], L=L, W=W) for o in others]
        b = _scene(f, ag)
        st = _state([5.0] + [0.0] * len(ag), [(0, 0)] + [(o[0], o[1]) for o in others],
                    [0.0] + [o[2] for o in others])
        _, _, lead = _step(b, st)
        assert lead[0] == exp, (others, lead)
    # the crossing vehicle's speed along the route does not count as lead speed
    ag = [dict(x=15.0, y=0.0, th=np.pi / 2, L=L, W=W)]
    b = _scene(f, ag)
    st = _state([5.0, 7.0], [(0, 0), (15.0, 0.0)], [0.0, np.pi / 2])
    st0 = _state([5.0, 0.0], [(0, 0), (15.0, 0.0)], [0.0, np.pi / 2])
    a1, _, _ = _step(b, st)
    a0, _, _ = _step(b, st0)
    assert abs(a1["vx"][0] - a0["vx"][0]) < 1e-9


def test_invalid_agents_are_not_leads():
    f = dict(x=0.0, y=0.0, v0=10.0)
    b = _scene(f, [dict(x=20.0, y=0.0, valid=0)])
    _, _, lead = _step(b, _state([5.0, 0.0], [(0, 0), (20.0, 0.0)], [0.0, 0.0]))
    assert lead[0] == -1


def test_pose_on_route_and_segment_heading():
    # arc route: the new pose lies on the polyline at parameter s', heading
    # that of the segment holding s'
    r, h = 30.0, 0.5
    dphi = 2 * np.arcsin(h / 2 / r)
    k = np.arange(320)
    route = np.stack([r * np.sin(k * dphi), r - r * np.cos(k * dphi)], 1)
    b = _scene(dict(x=0.0, y=0.0, v0=12.0), route=route)
    st = _state([9.0], [(0, 0)], [0.0])
    st["s"][:] = 3.3
    s1, band, _ = _step(b, st)
    sp = s1["s"][0]
    assert 3.3 < sp < 3.3 + 1.3
    j = int(np.floor(sp / h))
    tau = sp / h - j
    rt = route.astype(np.float32).astype(np.float64)
    p = rt[j] + tau * (rt[j + 1] - rt[j])
    assert np.hypot(s1["x"][0] - p[0], s1["y"][0] - p[1]) < 1e-12
    d = rt[j + 1] - rt[j]
    assert abs(s1["th"][0] - np.arctan2(d[1], d[0])) < 1e-12
    assert abs(np.hypot(s1["vx"][0], s1["vy"][0]) - (sp - 3.3) * 2 / DT + 9.0) < 1e-9


def test_route_end_extrapolates_last_segment():
    route = straight_route(0.0, 0.0, 0.0, n=5)
    b = _scene(dict(x=0.0, y=0.0, v0=10.0), route=route)
    st = _state([10.0], [(1.9, 0)], [0.0])
    st["s"][:] = 1.9
    s1, _, _ = _step(b, st)
    assert abs(s1["x"][0] - s1["s"][0]) < 1e-12 and s1["s"][0] > 2.0


def test_ambiguity_band_flags():
    L, W = 4.5, 2.0
    f = dict(x=0.0, y=0.0, v0=10.0, L=L, W=W)
    # lead whose widened box ends exactly on the first look-ahead sample that
    # it contains: the first-hit sample is undecided
    c = 0.5 * L + 2.0 * 8 + 0.5 * L + 0.5 * W
    b = _scene(f, [dict(x=c, y=0.0, L=L, W=W)])
    _, band, lead = _step(b, _state([5.0, 0.0], [(0, 0), (c, 0.0)], [0.0, 0.0]))
    assert lead[0] == 1 and band[0]
    # vehicle grazing the lane at exactly the widened half width
    b = _scene(f, [dict(x=20.0, y=0.0, L=L, W=W)])
    _, band, _ = _step(b, _state([5.0, 0.0], [(0, 0), (20.0, 2.0)], [0.0, 0.0]))
    assert band[0]
    # well inside: no band
    b = _scene(f, [dict(x=20.0, y=0.0, L=L, W=W)])
    _, band, _ = _step(b, _state([5.0, 0.0], [(0, 0), (20.3, 0.4)], [0.0, 0.0]))
    assert not band[0]


def test_free_road_acceleration_textbook_value():
    # Free-road term of the IDM (Treiber et al. 2000) with exponent 4:
    # a_free(v) = a (1 - (v/v0)^4); e.g. v = v0/2 gives 15/16 of a.
    for v, v0 in ((5.0, 10.0), (3.0, 12.0), (14.0, 14.0)):
        b = _scene(dict(x=0.0, y=0.0, v0=v0))
        s1, _, _ = _step(b, _state([v], [(0, 0)], [0.0]))
        assert abs(s1["vx"][0] - (v + AMAX * (1 - (v / v0) ** 4) * DT)) < 1e-12
