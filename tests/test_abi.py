"""The C ABI library loads and exports every entry point include/*.h declares.

No GPU needed: the library is opened with ctypes and symbols are resolved;
only entry points that reject their arguments before any CUDA call are
invoked.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(wsim_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2310_08710_b300 import build
    build.build()
    lib = C.CDLL(build.SO)
    declared = _declared()
    assert {"wsim_init", "wsim_step", "wsim_metrics", "wsim_rollout", "wsim_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_host_side_argument_checks_without_gpu():
    from paper_2310_08710_b300 import wsim
    lib = wsim.lib
    assert lib.wsim_init(None, None, None, None) == wsim.EINVAL
    h = C.c_void_p()
    cfg = wsim.default_config()
    assert abs(cfg.dt - 0.1) < 1e-7 and cfg.ckpt_every == 10
    assert cfg.kin_amax == 6.0 and abs(cfg.kin_kmax - 0.3) < 1e-7  # Sec. 3.4 limits
    b = wsim.WsimBatch()
    b.S = 0
    assert lib.wsim_init(C.byref(h), C.byref(cfg), C.byref(b), None) == wsim.ESIZE
    b.S, b.T_log = 1, 91
    assert lib.wsim_init(C.byref(h), C.byref(cfg), C.byref(b), None) == wsim.EINVAL  # null arrays
    assert lib.wsim_step(None, None, None, None, None, None, 0, None) == wsim.EINVAL
    assert lib.wsim_rollout(None, None, None, None, 10, 80, 0, None, None, None) == wsim.EINVAL
    assert lib.wsim_expert_actions(None, 10, 80, None, None) == wsim.EINVAL
    assert lib.wsim_observe(None, None, None, 128, 64, None, None, None, None, None) == wsim.EINVAL
    assert lib.wsim_route_metrics(None, None, None, None, None) == wsim.EINVAL
    assert lib.wsim_rollout_record(None, None, None, 10, 80, 10, None, None, None, None) == wsim.EINVAL
    assert lib.wsim_rollout_backward(None, None, None, None, None, None, None) == wsim.EINVAL
    assert lib.wsim_discretize(None, None, 1, None, None) == wsim.EINVAL
    assert lib.wsim_decode_actions(None, None, 1, None, None) == wsim.EINVAL
    assert (cfg.disc_na, cfg.disc_nk, cfg.disc_nd, cfg.disc_nt) == (13, 31, 25, 13)
    assert cfg.route_max_dist == 5.0 and cfg.route_max_rel == 2.0
    assert lib.wsim_strerror(wsim.ETIMEOUT).decode().startswith("a bounded")


def test_product_path_has_no_oracle_import():
    # The library package never reaches the oracle: no import, no load.
    pkg = os.path.join(ROOT, "paper_2310_08710_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "liboracle" not in src, f
