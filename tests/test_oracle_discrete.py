"""Pins of the oracle's discrete action spaces (Sec. 5.2: a discrete action
space's expert discretises the continuous inverse).

Grid values and indices are checked against hand-computed uniform grids,
nearest-value rounding against brute force over the grid, clamping, the
flat index layout, encode-decode round trips, and the discrete expert
replaying logs written with on-grid actions exactly like the continuous one.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08710_b300 import synth
from tests.scenes import tiny_batch
from tests.test_oracle_expert import _bicycle_log_batch

P = oracle.Params()


def _grid(mx, n):
    step = np.float32(2) * np.float32(mx) / np.float32(n - 1)
    return (np.arange(n, dtype=np.float32) - np.float32((n - 1) / 2)) * step


def test_grid_and_nearest_index_bicycle():
    b = tiny_batch([dict(x=0.0, y=0.0), dict(x=5.0, y=5.0)])
    o = oracle.Oracle(b)
    rng = np.random.default_rng(0)
    ga, gk = _grid(P.disc_a_max, P.disc_na), _grid(P.disc_k_max, P.disc_nk)
    assert ga[0] == -6 and ga[-1] == 6 and gk[P.disc_nk // 2] == 0 and (gk == -gk[::-1]).all()  # symmetric through 0
    T = 200
    act = np.zeros((T, 3, 2))
    act[:, 0] = rng.uniform(-7, 7, (T, 2))     # beyond the range: clamped to the ends
    act[:, 1] = rng.uniform(-0.35, 0.35, (T, 2))
    idx, band = o.discretize(act)
    ia = np.abs(act[:, 0, :, None] - ga).argmin(-1)  # brute force nearest
    ik = np.abs(act[:, 1, :, None] - gk).argmin(-1)
    ok = band == 0
    assert (idx[ok] == (ia * P.disc_nk + ik)[ok]).all()
    dec = o.decode_actions(idx)
    np.testing.assert_array_equal(dec[:, 0], ga[idx // P.disc_nk].astype(np.float64))
    np.testing.assert_array_equal(dec[:, 1], gk[idx % P.disc_nk].astype(np.float64))
    assert (dec[:, 2] == 0).all()
    # round trip: grid values map to themselves
    idx2, _ = o.discretize(dec)
    assert (idx2 == idx).all()


def test_delta_flat_index_and_invalid_agents():
    b = tiny_batch([dict(x=0.0, y=0.0, kind=1), dict(x=5.0, y=5.0, kind=1, valid=0)])
    o = oracle.Oracle(b)
    gd, gt = _grid(P.disc_d_max, P.disc_nd), _grid(P.disc_t_max, P.disc_nt)
    act = np.zeros((1, 3, 2))
    act[0, :, 0] = [gd[3], gd[20], gt[7]]
    idx, _ = o.discretize(act)
    assert idx[0, 0] == (3 * P.disc_nd + 20) * P.disc_nt + 7
    assert idx[0, 1] == -1  # invalid agent
    np.testing.assert_array_equal(o.decode_actions(idx)[0, :, 0], [gd[3], gd[20], gt[7]])


def test_band_at_rounding_boundaries():
    b = tiny_batch([dict(x=0.0, y=0.0)])
    o = oracle.Oracle(b)
    ga = _grid(P.disc_a_max, P.disc_na)
    mid = float((ga[4] + ga[5]) / 2)  # halfway between two grid values
    idx, band = o.discretize(np.array([[[mid], [0.0], [0.0]]]))
    assert band[0, 0] == 1
    idx, band = o.discretize(np.array([[[float(ga[4]) + 0.1], [0.0], [0.0]]]))
    assert band[0, 0] == 0 and idx[0, 0] // P.disc_nk == 4


def test_discrete_expert_on_logs_written_with_grid_actions():
    # logs written by the bicycle model with actions on the grid: the discrete
    # expert recovers those grid actions and replays the log to float32
    # rounding (like the continuous expert); off-grid logs make it drift
    b, acts = _bicycle_log_batch(21, N=8, T=20)
    o = oracle.Oracle(b)
    idx, band = o.discretize(acts)
    assert not band.any()
    grid = o.decode_actions(idx)
    # rewrite the logs from the grid actions
    b2, _ = _bicycle_log_batch(21, N=8, T=20)
    st = oracle.Oracle(b2).initial_state()
    rows = {k: [st[k]] for k in ("x", "y", "th", "vx", "vy")}
    oo = oracle.Oracle(b2)
    for k in range(20):
        st, _, _ = oo.transition(st, grid[k])
        for key in rows:
            rows[key].append(st[key])
    for key, arr in (("x", "log_x"), ("y", "log_y"), ("th", "log_th"), ("vx", "log_vx"), ("vy", "log_vy")):
        lg = getattr(b2, arr).astype(np.float64)
        lg[synth.T0:synth.T0 + 21] = np.array(rows[key])
        lg[synth.T0 + 21:] = rows[key][-1]
        setattr(b2, arr, lg.astype(np.float32))
    o2 = oracle.Oracle(b2)
    ctrl = np.full(b2.N_tot, oracle.CTRL_EXPERT_DISCRETE, np.uint8)
    _, m = o2.rollout(o2.initial_state(), None, synth.T0, 20, ctrl=ctrl)
    assert m["logdiv"].max() < 3e-5, m["logdiv"].max()
    _, m_off = oracle.Oracle(b).rollout(oracle.Oracle(b).initial_state(), None, synth.T0, 20, ctrl=ctrl)
    assert m_off["logdiv"].max() > 1e-3  # the original logs' actions are off the grid
