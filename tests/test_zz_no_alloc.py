"""wsim_metrics_static: the metrics pass for callers that cannot allocate.

A caller whose device memory is owned by someone else (a caching allocator,
a fixed arena) or that runs where cudaMalloc is not allowed can still get
the metrics: this entry point takes no context and keeps its scratch in a
fixed device array inside the library.  The test calls it twice in a row,
on two different batches, through the C ABI and compares each result with
what wsim_metrics returns for the same inputs, within the parity
tolerances; it also checks that oversized batches are refused up front.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2310_08710_b300 import synth
from tests import gpu_harness as H

pytestmark = pytest.mark.gpu


def _after_some_steps(w, b, steps):
    db = w.DeviceBatch(b)
    sim = w.Sim(db)
    st = w.State.from_batch(b)
    act = torch.as_tensor(b.actions[:steps]).cuda().contiguous()
    mseq = w.Metrics(b.N_tot, b.S, rows=steps)
    sim.rollout(st, act, mseq, synth.T0, steps, mode=w.MODE_STREAM)
    return db, sim, st


def _compare(ref, new):
    for k, tol in (("ov", H.TOL_DEPTH), ("off", H.TOL_DEPTH), ("logdiv", H.TOL_LOGDIV)):
        a, b = getattr(ref, k).cpu().numpy(), getattr(new, k).cpu().numpy()
        fin = np.isfinite(a)
        assert np.array_equal(fin, np.isfinite(b)), k
        assert np.array_equal(a[~fin], b[~fin]), k
        assert np.abs(a[fin] - b[fin]).max(initial=0) <= tol, k
    assert torch.equal(ref.flags, new.flags)
    assert torch.equal(ref.reward, new.reward)


def test_static_metrics_match_context_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    cases = [(synth.make_batch(1, seed=21, S=6, R=4000), 7), (synth.make_batch(0, seed=22), 3)]
    for b, steps in cases:
        db, sim, st = _after_some_steps(w, b, steps)
        t = synth.T0 + steps
        ref = w.Metrics(b.N_tot, b.S)
        sim.metrics(st, ref, t)
        new = w.Metrics(b.N_tot, b.S)
        new.ov.fill_(123.0)  # stale values must be overwritten
        w.metrics_static(db, st, new, t)
        torch.cuda.synchronize()
        _compare(ref, new)
        sim.close()


def test_static_metrics_refuses_oversized_batches():
    from paper_2310_08710_b300 import wsim as w
    cfg = w.default_config()
    b = w.WsimBatch()
    for f in ("agent_off", "rg_off", "L", "W", "valid", "log_x", "log_y", "kind", "idm_v0", "route_off"):
        setattr(b, f, 16)  # never dereferenced: the size checks come first
    b.T_log = 91
    st = w.WsimState(*([16] * 10))
    m = w.WsimMetricBuf(16, 16, 16, 16, 16)
    b.S, b.N_tot, b.R_tot = 5000, 5000, 0
    assert w.lib.wsim_metrics_static(C.byref(cfg), C.byref(b), C.byref(st), C.byref(m), 10, None) == w.ESIZE
    b.S, b.N_tot = 10, 10
    b.R_tot = 300000
    b.rg_x = b.rg_y = b.rg_poly = b.rg_type = b.rg_valid = 16
    assert w.lib.wsim_metrics_static(C.byref(cfg), C.byref(b), C.byref(st), C.byref(m), 10, None) == w.ESIZE
