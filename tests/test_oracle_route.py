"""Pins of the oracle's route metrics (Sec. 3.4 route progress ratio and
off-route) on hand-built paths: a straight road with known arc lengths, a
polygonal circle whose arc length is a sum of equal chords, parallel
off-route paths at known offsets, the choice between two on-route paths,
and the undefined cases.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch


def _batch(ego, paths, on, log_start, log_end, others=()):
    """One scene whose first agent is the ego at `ego` (x, y), with the given
    paths (lists of points) and on-route flags, and a log from log_start to
    log_end (rows 0 and T_LOG-1; the rows between hold the start)."""
    agents = [dict(x=ego[0], y=ego[1], th=0.0, v=1.0)] + [dict(x=o[0], y=o[1]) for o in others]
    log = np.zeros((synth.T_LOG, len(agents), 2))
    log[:, 0] = log_start
    log[-1, 0] = log_end
    b = tiny_batch(agents, log=log)
    b.path_off = np.array([0, len(paths)], np.int32)
    b.path_pt_off = np.concatenate([[0], np.cumsum([len(p) for p in paths])]).astype(np.int32)
    b.path_x = np.concatenate([np.asarray(p, float)[:, 0] for p in paths])
    b.path_y = np.concatenate([np.asarray(p, float)[:, 1] for p in paths])
    b.path_on = np.array(on, np.uint8)
    return b


def _route(b):
    o = oracle.Oracle(b)
    prog, fl = o.route(o.initial_state())
    return prog[0], fl[0]


ROAD = [(float(x), 0.0) for x in range(0, 101)]


def test_straight_road_progress_and_distance_threshold():
    prog, fl = _route(_batch((35.0, 2.0), [ROAD], [1], (10.0, 0.0), (60.0, 0.0)))
    assert prog == pytest.approx(0.5) and fl == 0
    prog, fl = _route(_batch((80.0, -1.0), [ROAD], [1], (10.0, 0.0), (60.0, 0.0)))
    assert prog == pytest.approx(1.4)  # driving past the logged end: above 1
    prog, fl = _route(_batch((5.0, 0.0), [ROAD], [1], (10.0, 0.0), (60.0, 0.0)))
    assert prog == pytest.approx(-0.1)  # behind the logged start
    _, fl = _route(_batch((35.0, 5.5), [ROAD], [1], (10.0, 0.0), (60.0, 0.0)))
    assert fl & 1  # farther than 5 m from the on-route path
    _, fl = _route(_batch((35.0, 4.5), [ROAD], [1], (10.0, 0.0), (60.0, 0.0)))
    assert not fl & 1
    _, fl = _route(_batch((35.0, 5.0), [ROAD], [1], (10.0, 0.0), (60.0, 0.0)))
    assert fl & 2  # at the threshold: band


def test_closer_to_an_off_route_path():
    lane = [(float(x), 3.0) for x in range(0, 101)]
    _, fl = _route(_batch((35.0, 2.6), [ROAD, lane], [1, 0], (10.0, 0.0), (60.0, 0.0)))
    assert fl & 1  # 2.6 m from the route, 0.4 m from the off-route lane: 2.2 > 2
    _, fl = _route(_batch((35.0, 2.4), [ROAD, lane], [1, 0], (10.0, 0.0), (60.0, 0.0)))
    assert not fl & 1  # 2.4 - 0.6 = 1.8 < 2
    _, fl = _route(_batch((35.0, 2.5), [ROAD, lane], [1, 0], (10.0, 0.0), (60.0, 0.0)))
    assert fl & 2  # exactly 2 m nearer: band


def test_polygonal_circle_arc_length():
    R, n = 50.0, 180
    ang = np.radians(np.arange(n + 1))
    circle = np.stack([R * np.cos(ang), R * np.sin(ang)], 1)
    chord = 2 * R * np.sin(np.radians(0.5))
    # ego 1 m radially outside vertex 70, log from vertex 10 to vertex 130
    ego = (R + 1.0) * np.array([np.cos(ang[70]), np.sin(ang[70])])
    prog, fl = _route(_batch(ego, [circle], [1], circle[10], circle[130]))
    # the ego and logged positions are float32 (~3e-6 m rounding over ~50 m of arc)
    assert prog == pytest.approx((70 - 10) * chord / ((130 - 10) * chord), abs=1e-7)
    assert fl == 0


def test_nearest_on_route_path_and_ties():
    far = [(float(x), 3.0) for x in range(0, 101)]
    shifted = [(float(x) + 20.0, -1.0) for x in range(0, 101)]  # arc lengths offset by 20 m
    prog_a, _ = _route(_batch((35.0, 0.5), [ROAD, shifted], [1, 1], (10.0, 0.0), (60.0, 0.0)))
    # 0.5 m from ROAD, 1.5 m from the shifted road: ROAD is the progress path
    assert prog_a == pytest.approx(0.5)
    prog_b, _ = _route(_batch((35.0, -0.9), [ROAD, shifted], [1, 1], (10.0, 0.0), (60.0, 0.0)))
    # 0.1 m from the shifted road: its arc lengths (ego 15, log 0 (clamped) and 40)
    assert prog_b == pytest.approx((15.0 - 0.0) / (40.0 - 0.0))
    _, fl = _route(_batch((35.0, -0.5), [ROAD, shifted], [1, 1], (10.0, 0.0), (60.0, 0.0)))
    assert fl & 4  # equidistant on-route paths: progress ambiguous
    prog_c, _ = _route(_batch((35.0, 1.5), [far, ROAD], [0, 1], (10.0, 0.0), (60.0, 0.0)))
    assert prog_c == pytest.approx(0.5)  # the off-route lane is never the progress path


def test_undefined_cases():
    prog, fl = _route(_batch((35.0, 0.0), [ROAD], [0], (10.0, 0.0), (60.0, 0.0)))
    assert np.isnan(prog) and fl == 0  # no on-route path
    prog, _ = _route(_batch((35.0, 0.0), [ROAD], [1], (10.0, 0.0), (10.0, 0.0)))
    assert np.isnan(prog)  # the log makes no progress
