"""Discrete action spaces on the GPU against the oracle (needs a B300).

Indices bit-exact outside the oracle's rounding band, decoded grid values
bit-exact, and teacher-forced parity of rollouts driven by the discrete
expert (ctrl 4).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth
from tests.gpu_harness import run_rollout, teacher_forced
from tests.test_gpu_expert import mixed_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wsim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    return w


def test_discretize_and_decode_match_the_oracle(wsim):
    b = mixed_batch(seed=4, S=4, N=40, R=2000)
    rng = np.random.default_rng(4)
    T = 30
    act = np.zeros((T, 3, b.N_tot), np.float32)
    act[:, 0] = rng.uniform(-8, 8, (T, b.N_tot))
    act[:, 1] = rng.uniform(-0.4, 0.4, (T, b.N_tot))
    act[:, 2] = rng.uniform(-0.4, 0.4, (T, b.N_tot))
    delta = b.kind == synth.KIND_DELTA
    act[:, 1, delta] = rng.uniform(-8, 8, (T, int(delta.sum())))
    sim = wsim.Sim(wsim.DeviceBatch(b))
    g_idx = sim.discretize(torch.as_tensor(act).cuda())
    g_dec = sim.decode_actions(g_idx)
    bad = sim.decode_actions(torch.full_like(g_idx, 10 ** 7))  # past every grid
    torch.cuda.synchronize()
    status = sim.status()
    sim.close()
    g_idx, g_dec = g_idx.cpu().numpy(), g_dec.cpu().numpy()
    o = oracle.Oracle(b)
    o_idx, band = o.discretize(act.astype(np.float64))
    ok = band == 0
    assert np.array_equal(g_idx[ok], o_idx[ok])
    assert (g_idx[:, b.kind == synth.KIND_IDM] == -1).all()
    assert np.array_equal(g_dec.astype(np.float64), o.decode_actions(g_idx))
    assert status == wsim.EINVAL  # the out-of-range indices
    assert (bad.cpu().numpy()[:, :, b.kind != synth.KIND_IDM] == 0).all()


def test_discrete_expert_teacher_forced(wsim):
    b = mixed_batch(seed=5, S=6, N=40, R=3000)
    ctrl = np.full(b.N_tot, 4, np.uint8)  # discrete expert for the policy agents, IDM for the rest
    g = run_rollout(b, ctrl=ctrl, no_actions=True)
    assert g["status"] == 0
    rep = {}
    teacher_forced(b, g, list(range(b.S)), range(b.T), report=rep, ctrl=ctrl)
    print("discrete expert", rep)
