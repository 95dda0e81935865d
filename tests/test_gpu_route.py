"""Route metrics on the GPU against the FP64 oracle (needs a B300).

Progress ratio within 1e-4 (float32 arc lengths summed over up to a few
hundred segments), off-route flags bit-exact outside the oracle's bands, at
several states of free-running rollouts of two workloads.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth
from tests.gpu_harness import run_rollout, state64

pytestmark = pytest.mark.gpu
TOL_PROGRESS = 1e-4


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def _check_states(wsim, b, states):
    sim = wsim.Sim(wsim.DeviceBatch(b))
    o = oracle.Oracle(b)
    ag = np.arange(b.N_tot)
    checked = amb = offr = 0
    for rows in states:
        st = wsim.State(b.N_tot, data=torch.as_tensor(np.ascontiguousarray(rows)).cuda())
        gp, gf = sim.route_metrics(st)
        gp, gf = gp.cpu().numpy().astype(np.float64), gf.cpu().numpy()
        op, of = o.route(state64(rows, ag))
        band, ambig = (of & 2) != 0, (of & 4) != 0
        assert np.array_equal(gf[~band], (of & 1)[~band]), "off-route flag"
        assert np.array_equal(np.isnan(gp[~ambig]), np.isnan(op[~ambig])), "undefined progress"
        ok = ~ambig & ~np.isnan(op)
        assert np.abs(gp[ok] - op[ok]).max(initial=0) <= TOL_PROGRESS, np.abs(gp[ok] - op[ok]).max()
        checked += int(ok.sum())
        amb += int(ambig.sum())
        offr += int(gf.sum())
    torch.cuda.synchronize()
    assert sim.status() == 0
    sim.close()
    return checked, amb, offr


def test_route_metrics_along_rollouts(wsim):
    for cfg, S in ((0, None), (1, 64)):
        b = synth.make_batch(cfg, seed=2, S=S)
        g = run_rollout(b)
        init = np.zeros((10, b.N_tot), np.float32)
        init[0], init[1], init[4], init[6], init[7] = b.x, b.y, b.th, b.vx, b.vy
        states = [init] + [g["traj"][:, k, :] for k in (0, 9, 39, 79)]
        checked, amb, offr = _check_states(wsim, b, states)
        print("workload", cfg, "progress checked", checked, "ambiguous", amb, "off-route", offr)
        assert checked > 0


def test_expert_stays_on_route_random_actions_leave_it(wsim):
    # the delta expert follows its log, which the on-route path runs through:
    # progress reaches ~1 at the end and it never leaves the route; random
    # bicycle actions drive most egos off it
    b = synth.make_batch(1, seed=3, S=32)
    b.kind[b.agent_off[:-1]] = synth.KIND_DELTA
    ctrl = np.full(b.N_tot, 1, np.uint8)
    ctrl[b.agent_off[:-1]] = 2
    g = run_rollout(b, ctrl=ctrl)
    rows = g["final"]
    sim = wsim.Sim(wsim.DeviceBatch(b))
    gp, gf = sim.route_metrics(wsim.State(b.N_tot, data=torch.as_tensor(rows).cuda()))
    gp, gf = gp.cpu().numpy(), gf.cpu().numpy()
    sim.close()
    ok = ~np.isnan(gp)
    assert np.abs(gp[ok] - 1.0).max() < 1e-3 and not gf.any()
