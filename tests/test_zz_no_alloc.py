"""wsim_metrics_static: the metrics pass for callers that cannot allocate.

A caller whose device memory is owned by someone else (a caching allocator,
a fixed arena) or that runs where cudaMalloc is not allowed can still get
the metrics: this entry point takes no context and keeps its scratch in a
fixed device array inside the library.  The test calls it twice in a row,
on two different batches, through the C ABI and compares each result with
what wsim_metrics returns for the same inputs, within the parity
tolerances, and once with the FP64 oracle.  It also checks that oversized
batches are refused up front, that a batch whose road edges only overflow
the fixed arrays once every run is padded is refused on the device, that
malformed CSR offsets are refused before any roadgraph range is read, and
that a valid call after each refusal succeeds.  This file is collected last
on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2310_08710_b300 import synth
from tests import gpu_harness as H
from tests.scenes import tiny_batch

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


def _metrics_or_code(w, db, st, b, t):
    """wsim_metrics_static through the C ABI: (return code, metrics)."""
    m = w.Metrics(b.N_tot, b.S)
    m.ov.fill_(123.0)
    cfg = w.default_config()
    rc = w.lib.wsim_metrics_static(C.byref(cfg), C.byref(db.c), C.byref(st.c()), C.byref(m.c()), t,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, m


def test_static_metrics_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    b = synth.make_batch(1, seed=23, S=4, R=5000)
    steps = 9
    db, sim, st = _after_some_steps(w, b, steps)
    t = synth.T0 + steps
    rc, m = _metrics_or_code(w, db, st, b, t)
    assert rc == w.OK
    rows = st.data.cpu().numpy()
    me = oracle.Oracle(b).metrics(H.state64(rows, np.arange(b.N_tot)), t)
    for k, tol in (("ov", H.TOL_DEPTH), ("off", H.TOL_DEPTH), ("logdiv", H.TOL_LOGDIV)):
        g = getattr(m, k).cpu().numpy()[0].astype(np.float64)
        e = me[k]
        fin = np.isfinite(e)
        assert np.array_equal(np.isfinite(g), fin), k
        assert np.array_equal(g[~fin], e[~fin]), k
        assert (np.abs(g[fin] - e[fin]) <= H._ulp_tol(tol, e[fin])).all(), k
    gf, ef = m.flags.cpu().numpy()[0], me["flags"]
    b_ov, b_off = (ef & 4) != 0, (ef & 8) != 0
    assert np.array_equal((gf & 1)[~b_ov], (ef & 1)[~b_ov])
    assert np.array_equal((gf & 2)[~b_off], (ef & 2)[~b_off])
    sim.close()


def test_static_metrics_refusals_then_valid_call():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08710_b300 import wsim as w
    # (1) 20,000 road edges of two points each: 40,000 points pass the host
    # bound (R_tot + 15 S <= 262,144), but every one-segment run is padded to
    # 16 positions, 320,000 in all: refused on the device.
    pts = [(np.array([[3.0 * (i % 200), 3.0 * (i // 200)], [3.0 * (i % 200) + 1.0, 3.0 * (i // 200)]]), 1)
           for i in range(20000)]
    big = tiny_batch([dict(x=10.0, y=10.0, v=2.0), dict(x=40.0, y=12.0, th=0.4, v=3.0)], roadgraph=pts)
    db = w.DeviceBatch(big)
    st = w.State.from_batch(big)
    rc, m = _metrics_or_code(w, db, st, big, synth.T0)
    assert rc == w.ESIZE
    assert (m.ov == 123.0).all()  # nothing written
    # (2) a valid batch, then the same batch with its device CSR offsets
    # broken in ways that stay inside the arrays
    b = synth.make_batch(0, seed=24, S=3, R=2000)
    db = w.DeviceBatch(b)
    st = w.State.from_batch(b)
    rc, ref = _metrics_or_code(w, db, st, b, synth.T0)
    assert rc == w.OK
    good_rg = db.rg_off.clone()
    good_ag = db.agent_off.clone()
    R = b.R_tot
    bad_rg = ([0, 1000, 2500, R - 1],              # ends before R_tot
              [0, 3000, 2000, R],                  # decreasing
              [5, 2000, 4000, R])                  # does not start at 0
    for off in bad_rg:
        db.rg_off.copy_(torch.tensor(off, dtype=torch.int32))
        rc, m = _metrics_or_code(w, db, st, b, synth.T0)
        assert rc == w.EINVAL, off
        assert (m.ov == 123.0).all()
        db.rg_off.copy_(good_rg)
        rc, m = _metrics_or_code(w, db, st, b, synth.T0)  # the status word was cleared
        assert rc == w.OK
        _compare(ref, m)
    n = b.N_tot
    db.agent_off.copy_(torch.tensor([0, 40, 20, n], dtype=torch.int32))  # decreasing
    rc, _ = _metrics_or_code(w, db, st, b, synth.T0)
    assert rc == w.EINVAL
    db.agent_off.copy_(good_ag)
    rc, m = _metrics_or_code(w, db, st, b, synth.T0)
    assert rc == w.OK
    _compare(ref, m)
