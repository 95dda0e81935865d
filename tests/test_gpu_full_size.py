"""The three large workloads at full size, in the benchmark's launch
configuration, against the FP64 oracle (needs a B300).

Each batch is drawn in full, the rollout's launch shapes are autotuned on
it exactly as bench.py does (wsim_autotune over 8 steps), and one
scene-resident rollout of all 80 steps runs with every state stored.  The
oracle then checks a sample of scenes at every step, teacher-forced
(positions 1e-5 m, heading 1e-6 rad, velocity 1e-5 m/s, route parameter
1e-5 m, log divergence 1e-5 m, overlap depth and off-road distance 2e-5 m or
4 float32 ulps; flags and rewards bit-exact outside the bands):

- 1,024 scenes x 128 agents, 20k-point roadgraphs, IDM: 16 scenes;
- 4,096 uneven scenes (8-128 agents, 1k-30k points): 32 scenes, spread over
  the roadgraph sizes (so over every size bucket) with the largest roadgraph
  and the most agents;
- 16,384 scenes x 128 agents, 30k-point roadgraphs, delta/bicycle egos and
  IDM: 8 scenes from both halves and the extremes of road-edge count.

The per-quantity maxima are printed.
"""
import os

import numpy as np
import pytest
import torch

from paper_2310_08710_b300 import synth
from tests import gpu_harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def _draw(cfg):
    return synth.make_batch(cfg, seed=0, workers=min(32, os.cpu_count() or 1))


def _edge_points(b):
    """Road-edge points per scene (a proxy of the packed segment count)."""
    e = (b.rg_type == synth.RG_EDGE).astype(np.int64)
    return np.add.reduceat(e, b.rg_off[:-1])


def _run_sampled(w, b, scenes):
    """Autotuned scene-resident rollout of the whole batch; the states and
    metric rows of the sampled scenes as a batch of their own."""
    db = w.DeviceBatch(b)
    sim = w.Sim(db)
    st0 = w.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().contiguous()
    tune = sim.autotune(st0, act, synth.T0, 8)
    st = st0.clone()
    traj = w.State(b.N_tot, rows=b.T)
    m = w.Metrics(b.N_tot, b.S, rows=b.T)
    sim.rollout(st, act, m, synth.T0, b.T, mode=w.MODE_FUSED, traj=traj)
    torch.cuda.synchronize()
    status = sim.status()
    ag = np.concatenate([np.arange(b.agent_off[s], b.agent_off[s + 1]) for s in scenes]).astype(np.int64)
    idx = torch.as_tensor(ag, device="cuda")
    sidx = torch.as_tensor(np.asarray(scenes, np.int64), device="cuda")
    gpu = dict(traj=traj.data.view(10, b.T, b.N_tot)[:, :, idx].cpu().numpy(),
               ov=m.ov[:, idx].cpu().numpy(), off=m.off[:, idx].cpu().numpy(),
               logdiv=m.logdiv[:, idx].cpu().numpy(), flags=m.flags[:, idx].cpu().numpy(),
               reward=m.reward[:, sidx].cpu().numpy(), status=status)
    sim.close()
    del traj, m, db
    torch.cuda.empty_cache()
    return b.subset(scenes), gpu, tune


def _check(b, scenes, wsim_mod):
    sub, gpu, tune = _run_sampled(wsim_mod, b, scenes)
    assert gpu["status"] == 0
    c = H.teacher_forced(sub, gpu, list(range(sub.S)), range(b.T))
    print(f"{b.S} scenes, tuning {tune}\n  {len(scenes)} scenes x {b.T} steps checked: {c}")
    assert c["steps"] == b.T
    return c


def test_batch_1024x128_idm_16_scenes(wsim):
    b = _draw(1)
    scenes = np.linspace(0, b.S - 1, 16).astype(int).tolist()
    c = _check(b, scenes, wsim)
    assert c["band_idm"] <= 0.02 * c["agent_steps"]


def test_uneven_4096_full_size_32_scenes(wsim):
    b = _draw(2)
    R = np.diff(b.rg_off)
    Nn = np.diff(b.agent_off)
    order = np.argsort(_edge_points(b), kind="stable")
    spread = order[np.linspace(0, b.S - 1, 30).astype(int)].tolist()
    scenes = sorted(set(spread) | {int(np.argmax(R)), int(np.argmax(Nn))})
    assert len(scenes) >= 31
    _check(b, scenes, wsim)


def test_sweep_16384x128_full_size_8_scenes(wsim):
    b = _draw(4)
    e = _edge_points(b)
    S = b.S
    scenes = sorted({0, S // 2 - 1, S // 2, S - 1, int(np.argmax(e)), int(np.argmin(e)),
                     int(np.argmax(e[: S // 2])), int(np.argmax(e[S // 2:])) + S // 2})
    while len(scenes) < 8:
        scenes = sorted(set(scenes) | {int(np.random.default_rng(len(scenes)).integers(0, S))})
    assert b.kind[b.agent_off[0]] == synth.KIND_DELTA and b.kind[b.agent_off[S - 1]] == synth.KIND_BICYCLE
    c = _check(b, scenes, wsim)
    assert c["band_idm"] <= 0.02 * c["agent_steps"]
