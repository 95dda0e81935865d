#!/usr/bin/env python
"""Throughput of the batched closed-loop rollout on B300.

One step = one 80-step rollout of the whole scene batch: per step of it,
action resolution, IDM sim agents, bicycle/delta dynamics, pairwise box
overlap, off-road signed distance, log divergence and reward (the Step of the
paper's runtime benchmark, Sec. 5.1, driven for a full episode as in its
Rollout column).  Metric: agent-steps/s (agent slots x simulated steps per
second), all scenes on one GPU, inputs resident in HBM.

The default workload is the largest single-GPU one: 16,384 scenes x 128
agents x 80 steps with 30,000-point roadgraphs, delta egos in the first half
of the batch and bicycle egos in the second, IDM sim agents.  The line also
carries, under "extra", the 1,024 x 128 IDM batch, and under "bptt" the
gradient steps/s of backpropagation through whole rollouts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wsim|reference]

Under torchrun every rank simulates its own batch (different seeds) and the
value is the total over ranks divided by the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-steps/s (step+overlap+offroad) on 1 B300; BPTT grad steps/s vs plain"
UNIT = "agent-steps/s"
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
FP32_PEAK_SOURCE = "derived: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz"
# FP32 operations (FMUL/FADD 1, FFMA 2) per unit of counted work, counted
# from the kernels' inner loops.  The method's own work:
FLOPS_PER_EVAL = 15       # corner x road-edge segment distance
FLOPS_PER_PAIR_COUNT = 22  # SAT depth of a pair: 44, and the counter counts each evaluated pair twice
FLOPS_PER_TEST = 16       # IDM look-ahead sample x box test
FLOPS_PER_IDM_STEP = 800  # IDM agent-step: 32 look-ahead samples on the route, acceleration, advance
FLOPS_PER_AGENT = 60      # dynamics + log divergence per agent-step
# ... and the culling tests that only decide what the method evaluates:
FLOPS_PER_TILE = 10       # culling-tile bound test
FLOPS_PER_BOUND = 11      # overlap pair bound test
FLOPS_PER_FILTER = 9      # IDM lead-candidate circle test
# Backpropagation through the rollout, per valid pair and step: the loss
# term (SAT depth and softplus, 58) and its adjoint (SAT depth with the active
# axis' partial derivatives, sigmoid, both agents' sums, 75); per agent-step:
# forward dynamics 60, log divergence term 5, adjoint of the dynamics 40,
# and the recomputed forward step of a checkpoint segment 60 (ck-1)/ck.
BPTT_PAIR_FWD, BPTT_PAIR_ADJ = 58, 75
BPTT_AGENT_FWD, BPTT_AGENT_LOSS, BPTT_AGENT_ADJ = 60, 5, 40


ROLLOUT_SOURCES = ("wsim_rollout.cu", "wsim_phases.cuh", "wsim_device.cuh", "wsim_internal.h")


def source_hash(names=ROLLOUT_SOURCES) -> str:
    """sha256 (first 16 hex digits) of the sources a kernel is built from (by
    default the scene-resident rollout kernel's) and the C ABI header."""
    import hashlib
    c = os.path.join(ROOT, "paper_2310_08710_b300", "csrc")
    files = [os.path.join(c, n) for n in names] + [os.path.join(ROOT, "include", "wsim.h")]
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the last ncu capture of this kernel on this
    workload, if it was taken on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel, {}).get(workload)
    except (OSError, ValueError, AttributeError):
        return None
    if not rec or rec.get("source_sha256_16") != source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wsim", choices=["wsim", "reference"])
    ap.add_argument("--workload", type=int, default=4,
                    help="synthetic workload id (paper_2310_08710_b300.synth.WORKLOADS); "
                         "4 = 16384 scenes x 128 agents, 30k-point roadgraphs, IDM")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 1024 x 128 batch reported under 'extra'")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="fused", choices=["fused", "graph"],
                    help="rollout path timed: scene-resident kernel or graph of per-step launches")
    ap.add_argument("--scenes", type=int, default=None, help="override the scene count (profiling only)")
    ap.add_argument("--shape", type=int, default=None,
                    help="pin one launch shape of the scene-resident rollout instead of autotuning (profiling)")
    ap.add_argument("--bptt-only", action="store_true", help="run only the BPTT leg (profiling)")
    ap.add_argument("--bptt-workload", type=int, default=3,
                    help="synthetic workload of --bptt-only (3 = 256 scenes x 64 agents; 4 = the 30k-point sweep)")
    ap.add_argument("--bptt-scenes", type=int, default=None, help="override the --bptt-only leg's scene count")
    ap.add_argument("--profile", action="store_true",
                    help="time the main path only (no mode comparison, end-to-end or CPU legs)")
    ap.add_argument("--expert-only", action="store_true", help="run only the expert leg on the workload (profiling)")
    ap.add_argument("--observe-only", action="store_true",
                    help="run only the observation and route-metric leg on the workload (profiling)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.rows = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=2)

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        pw = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def combine_ranks(pg, times_ms, units, device):
    """Whole-job view of per-rank measurements: the slowest rank's times and
    the total units of all ranks (weak scaling: every rank simulates its own
    scenes, nothing else is exchanged)."""
    if pg is None:
        return (*times_ms, units)
    import torch
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    pg.all_reduce(u)
    return (*t.tolist(), u.item())


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "wsim" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def gen_workers(scenes: int) -> int:
    """Processes that draw the synthetic scenes (large batches only)."""
    return min(32, os.cpu_count() or 1) if scenes >= 512 else 1


def make(synth, cfg, seed, S=None, scenes=None):
    n = len(scenes) if scenes is not None else (S or synth.WORKLOADS[cfg].S)
    return synth.make_batch(cfg, seed=seed, S=S, scenes=scenes, workers=gen_workers(n))


def workload_config(synth, cfg, S=None, b=None) -> dict:
    """The workload's description; totals from the batch, or from the
    workload definition when it has fixed agent and point counts."""
    wl = synth.WORKLOADS[cfg]
    S = S or wl.S
    if b is not None:
        n_tot, r_tot = int(b.N_tot), int(b.R_tot)
    elif isinstance(wl.N, int) and isinstance(wl.R, int):
        n_tot, r_tot = S * wl.N, S * wl.R
    else:
        n_tot = r_tot = None
    return {"workload": wl.name, "scenes": int(S), "agents": n_tot, "rollout_steps": int(wl.T),
            "roadgraph_points": r_tot, "dt_s": 0.1,
            "rollout_mode": "scene-resident rollout kernel (one launch per rollout)",
            "l2": "inputs larger than L2 (road-edge segments + routes + logs streamed every rollout)"}


def oracle_probe_seconds(synth, cfg, seed, S=None) -> float:
    """Single-thread seconds of the oracle's full rollout of one scene (from
    8 steps of scene 0)."""
    import oracle
    probe = synth.make_batch(cfg, seed=seed, S=S, scenes=[0])
    o = oracle.Oracle(probe)
    t = time.perf_counter()
    o.rollout(o.initial_state(), probe.actions, synth.T0, 8, nthreads=1)
    return (time.perf_counter() - t) * (probe.T / 8)


def cpu_baseline(synth, cfg, seed, S, seconds: float) -> dict:
    """The FP64 oracle's free-running rollout on host cores, bounded sample
    (the first scenes of the same workload, drawn on their own)."""
    import oracle
    cores = os.cpu_count() or 1
    per_scene = oracle_probe_seconds(synth, cfg, seed, S)
    total = S or synth.WORKLOADS[cfg].S
    n = int(max(1, min(total, round(seconds * cores / max(per_scene, 1e-3)))))
    sub = make(synth, cfg, seed, S=S, scenes=list(range(n)))
    o = oracle.Oracle(sub)
    st = o.initial_state()
    t = time.perf_counter()
    o.rollout(st, sub.actions, synth.T0, sub.T, nthreads=cores)
    dt = time.perf_counter() - t
    return {"value": sub.N_tot * sub.T / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of {total} scenes x {sub.T} steps (free-running FP64 rollout, OpenMP over scenes)",
            "seconds": dt}


def run_reference(args, ws, rank, pg):
    """The oracle on the host cores: each step a bounded sample of the
    workload (rank 0 only; the other ranks exit without work)."""
    from paper_2310_08710_b300 import synth
    if rank != 0:
        return
    import oracle
    cores = os.cpu_count() or 1
    # size each step so that the whole run stays within a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    per_scene = oracle_probe_seconds(synth, args.workload, args.seed, args.scenes)
    total = args.scenes or synth.WORKLOADS[args.workload].S
    n = int(max(1, min(total, budget * cores / max(per_scene, 1e-3) * 0.8)))
    sub = make(synth, args.workload, args.seed, S=args.scenes, scenes=list(range(n)))
    o = oracle.Oracle(sub)
    st = o.initial_state()
    for _ in range(args.warmup):
        o.rollout(st, sub.actions, synth.T0, sub.T, nthreads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.rollout(st, sub.actions, synth.T0, sub.T, nthreads=cores)
    dt = (time.perf_counter() - t) / max(1, args.steps)
    v = sub.N_tot * sub.T / dt
    sample = f"{n} of {total} scenes x {sub.T} steps per step (free-running FP64 rollout, OpenMP over scenes)"
    full = None if isinstance(synth.WORKLOADS[args.workload].N, int) else make(synth, args.workload, args.seed,
                                                                                S=args.scenes)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(synth, args.workload, args.scenes, full),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


def alu_roofline(kernel, flops, ms, **more):
    a = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": a, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": a / FP32_PEAK_TFLOPS, "peak_source": FP32_PEAK_SOURCE, "flops_per_launch": flops,
            "launch_ms": ms, **more}


def hbm_roofline(kernel, nbytes, ms, **more):
    peak, src = hbm_peak_gbs()
    a = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
            "peak_source": src, "bytes_per_launch": int(nbytes), "launch_ms": ms, **more}


def timed(torch, fn, reps, warm=3, stream=None):
    """Mean ms of fn() over reps runs after warm runs (CUDA events on the
    current stream)."""
    stream = stream or torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def rollout_roofline(synth, b, cnt, launch_ms, kernel, workload_key):
    """Counted FP32 work of the rollout kernel over its launch time: the
    method's own evaluations in the numerator, the culling tests beside it."""
    T, N = b.T, b.N_tot
    idm_steps = int(((b.kind == synth.KIND_IDM) & (b.valid != 0)).sum()) * T
    method = (FLOPS_PER_EVAL * cnt[0] + FLOPS_PER_PAIR_COUNT * cnt[2] + FLOPS_PER_TEST * cnt[3]
              + FLOPS_PER_IDM_STEP * idm_steps + FLOPS_PER_AGENT * N * T)
    overhead = FLOPS_PER_TILE * cnt[1] + FLOPS_PER_BOUND * cnt[4] + FLOPS_PER_FILTER * cnt[5]
    r = alu_roofline(kernel, float(method), launch_ms,
                     traffic=recorded_traffic(kernel, workload_key) if kernel == "k_rollout" else None)
    r["overhead_flops"] = float(overhead)
    r["overhead_frac"] = overhead / (launch_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS
    r["counts_per_rollout"] = {"corner_segment_evals": int(cnt[0]), "tile_tests": int(cnt[1]),
                               "sat_pairs_x2": int(cnt[2]), "idm_sample_tests": int(cnt[3]),
                               "pair_bound_tests": int(cnt[4]), "idm_circle_tests": int(cnt[5]),
                               "idm_agent_steps": idm_steps, "agent_steps": N * T}
    r["flops_per_unit"] = {"corner_segment_eval": FLOPS_PER_EVAL, "sat_pair_x2": FLOPS_PER_PAIR_COUNT,
                           "idm_sample_test": FLOPS_PER_TEST, "idm_agent_step": FLOPS_PER_IDM_STEP,
                           "agent_step": FLOPS_PER_AGENT, "overhead": {"tile_test": FLOPS_PER_TILE,
                                                                       "pair_bound_test": FLOPS_PER_BOUND,
                                                                       "idm_circle_test": FLOPS_PER_FILTER}}
    return r


class Rollout:
    """One batch on the device with the scene-resident rollout, tuned."""

    def __init__(self, wsim, synth, torch, b, mode, shape=None):
        self.wsim, self.synth, self.torch, self.b = wsim, synth, torch, b
        self.db = wsim.DeviceBatch(b)
        self.sim = wsim.Sim(self.db)
        self.st0 = wsim.State.from_batch(b)
        self.st = self.st0.clone()
        self.act = torch.as_tensor(b.actions).cuda().contiguous()
        self.m = wsim.Metrics(b.N_tot, b.S, rows=b.T)
        self.mode = wsim.MODE_FUSED if mode == "fused" else wsim.MODE_GRAPH
        if shape is not None:
            self.sim.set_tuning(single_shape=shape)
            self.tune = self.sim.get_tuning()
        else:
            self.tune = self.sim.autotune(self.st0, self.act, synth.T0, 8) if self.mode == wsim.MODE_FUSED else None

    def run(self, mode=None):
        self.st.data.copy_(self.st0.data)
        self.sim.rollout(self.st, self.act, self.m, self.synth.T0, self.b.T,
                         mode=self.mode if mode is None else mode)

    def launches(self):
        if self.mode != self.wsim.MODE_FUSED:
            return self.b.T
        t = self.tune
        return sum(1 for n in t["bucket_scenes"] if n) if t and t["split"] else 1

    def counts(self):
        self.sim.set_counting(True)
        self.run()
        cnt = [int(x) for x in self.sim.counters()]
        self.sim.set_counting(False)
        return cnt

    def e2e(self, reps):
        """The same rollout through the public API with every step's inputs
        copied from pinned host memory and its result (reward and flags
        rows) read back, all inside the timed region.  Streamed: two sets of
        device buffers; on a second stream the next step's inputs go up and
        the last step's results come down while the current rollout runs
        (a step waits for its inputs, a buffer is reused only after the
        copies that read it).  Returns (ms per step streamed, ms per step
        with copy, rollout and read-back in series, bytes up, bytes down)."""
        torch, b, wsim = self.torch, self.b, self.wsim
        h_act = torch.as_tensor(b.actions).pin_memory()
        h_st = self.st0.data.cpu().pin_memory()
        h_rew = torch.empty((b.T, b.S), dtype=torch.int32).pin_memory()
        h_flags = torch.empty((b.T, b.N_tot), dtype=torch.uint8).pin_memory()

        def step():
            self.act.copy_(h_act, non_blocking=True)
            self.st.data.copy_(h_st, non_blocking=True)
            self.sim.rollout(self.st, self.act, self.m, self.synth.T0, b.T, mode=self.mode)
            h_rew.copy_(self.m.reward, non_blocking=True)
            h_flags.copy_(self.m.flags, non_blocking=True)
        ms_serial = timed(torch, step, reps, warm=2)

        acts = [self.act, torch.empty_like(self.act)]
        sts = [self.st, self.st.clone()]
        ms_ = [self.m, wsim.Metrics(b.N_tot, b.S, rows=b.T)]
        comp, copy = torch.cuda.current_stream(), torch.cuda.Stream()
        ev = lambda: torch.cuda.Event()
        inputs_in, compute_done, results_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]

        def upload(k):  # inputs of step k into buffer k % 2, on the copy stream
            q = k % 2
            with torch.cuda.stream(copy):
                copy.wait_event(compute_done[q])  # the rollout that read this buffer is done
                acts[q].copy_(h_act, non_blocking=True)
                sts[q].data.copy_(h_st, non_blocking=True)
                inputs_in[q].record(copy)

        def run(n):
            upload(0)
            for k in range(n):
                q = k % 2
                if k + 1 < n:
                    upload(k + 1)
                comp.wait_event(inputs_in[q])
                comp.wait_event(results_out[q])  # the metric rows of step k-2 have been read
                self.sim.rollout(sts[q], acts[q], ms_[q], self.synth.T0, b.T, mode=self.mode)
                compute_done[q].record(comp)
                with torch.cuda.stream(copy):
                    copy.wait_event(compute_done[q])
                    h_rew.copy_(ms_[q].reward, non_blocking=True)
                    h_flags.copy_(ms_[q].flags, non_blocking=True)
                    results_out[q].record(copy)
            comp.wait_stream(copy)  # the last read-back inside the timed region

        for q in range(2):  # events start recorded
            compute_done[q].record(comp)
            results_out[q].record(comp)
        run(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        run(reps)
        e1.record(comp)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return ms, ms_serial, h_act.numel() * 4 + h_st.numel() * 4, h_rew.numel() * 4 + h_flags.numel()

    def close(self):
        assert self.sim.status() == 0
        self.sim.close()


def modes_leg(wsim, synth, torch, R, plain_scenes):
    """The same rollout through the per-step paths: a CUDA graph of T
    persistent step launches (whole batch), and one launch per scene and
    phase (the plain baseline; on the first `plain_scenes` scenes when the
    batch is larger, its rate per agent-step is what compares)."""
    b = R.b
    ms = timed(torch, lambda: R.run(wsim.MODE_GRAPH), 3, warm=1)
    out = {"graph_of_steps": {"value": b.N_tot * b.T / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms,
                              "rollouts_timed": 3, "scenes": b.S}}
    if plain_scenes is not None and plain_scenes < b.S:
        P = Rollout(wsim, synth, torch, b.subset(list(range(plain_scenes))), "fused", shape=3)
    else:
        P = R
    mp = timed(torch, lambda: P.run(wsim.MODE_PLAIN), 1, warm=1)
    out["plain_per_scene"] = {"value": P.b.N_tot * P.b.T / (mp / 1e3), "unit": UNIT, "ms_per_rollout": mp,
                              "rollouts_timed": 1, "scenes": P.b.S}
    if P is not R:
        P.close()
    return out


def bptt_pairs(b) -> int:
    """Valid agent pairs summed over scenes (each scene's pairs are evaluated
    at every step by the loss and its adjoint)."""
    v = np.add.reduceat(b.valid.astype(np.int64), b.agent_off[:-1]) if b.N_tot else np.zeros(b.S, np.int64)
    v = np.where(np.diff(b.agent_off) > 0, v, 0)
    return int((v * (v - 1) // 2).sum())


def bptt_leg(wsim, synth, torch, b, plain, reps=5):
    """Gradient steps/s of the differentiable rollout: one gradient step =
    forward rollout with the loss plus the reverse sweep giving dL/d(every
    action), checkpointed every 10 steps and storing every step."""
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().contiguous()
    out = {"workload": f"{b.S} scenes x up to {int(np.diff(b.agent_off).max())} agents x {b.T} steps, "
                       "loss = log divergence^2 + softplus overlap"}
    pairs, T = bptt_pairs(b), b.T
    agents = int(b.valid.sum())
    # Pairs the kernel evaluates: those not ruled out by the exact cut (a
    # pair whose depth bound lies below -120 tau adds exactly 0); counted
    # once, forward and adjoint evaluate the same pairs (2 per pair each).
    sim.set_counting(True)
    sim.loss_grad(st, act, synth.T0, T, 10)
    evaluated = [int(x) for x in sim.counters()][2] // 4
    sim.set_counting(False)
    out["pairs_x_steps"] = {"valid": pairs * T, "evaluated": evaluated}
    legs = [("ckpt10", 10, False, reps), ("store_all", 1, False, reps)]
    if plain:
        legs.append(("plain_per_scene_ckpt10", 10, True, 1))
    for name, ck, pl, n in legs:
        ms = timed(torch, lambda: sim.loss_grad(st, act, synth.T0, T, ck, plain=pl), n, warm=1)
        out[name] = {"grad_steps_per_s": 1e3 / ms, "ms": ms, "agent_steps_per_s": b.N_tot * T / (ms / 1e3)}
        if not pl:
            flops = (evaluated * (BPTT_PAIR_FWD + BPTT_PAIR_ADJ)
                     + agents * T * (BPTT_AGENT_FWD + BPTT_AGENT_LOSS + BPTT_AGENT_ADJ
                                     + BPTT_AGENT_FWD * (ck - 1) / ck))
            out[name]["roofline"] = alu_roofline("k_bptt", float(flops), ms, traffic=None,
                                                 counted={"evaluated_pairs_x_steps": evaluated,
                                                          "valid_agent_steps": agents * T})
    stc, mf = st.clone(), wsim.Metrics(b.N_tot, b.S, rows=T)

    def fwd():
        stc.data.copy_(st.data)
        sim.rollout(stc, act, mf, synth.T0, T, mode=wsim.MODE_FUSED)
    out["forward_rollout_ms"] = timed(torch, fwd, reps, warm=1)
    # The general differentiable rollout: recorded forward (metric rows, their
    # deciding indices, checkpoints every 10 steps, the loss) and the backward
    # of a weighted sum of every metric row and the loss, to the actions and
    # the initial state (wsim_rollout_record + wsim_rollout_backward).
    g = torch.Generator(device="cuda").manual_seed(7)
    wts = [torch.randn((T, b.N_tot), device="cuda", generator=g) for _ in range(3)]
    lw = torch.ones(b.S, dtype=torch.float64, device="cuda")
    ms_rec = timed(torch, lambda: sim.rollout_record(st, act, mf, synth.T0, T, 10), reps, warm=1)
    ms_bwd = timed(torch, lambda: sim.rollout_backward(act, *wts, loss_w=lw), reps, warm=1)
    out["metric_grad_ckpt10"] = {"grad_steps_per_s": 1e3 / (ms_rec + ms_bwd), "ms": ms_rec + ms_bwd,
                                 "record_ms": ms_rec, "backward_ms": ms_bwd,
                                 "objective": "loss + random weights on every log divergence, overlap and "
                                              "off-road row; gradients to actions and initial state"}
    assert sim.status() == 0
    sim.close()
    return out


def expert_leg(wsim, synth, torch, R, reps):
    """The paper's expert actor (Sec. 5.2) on the bench's scenes with every
    valid agent a bicycle policy agent: (1) the open-loop expert actions of
    all 80 steps (one HBM-bound launch), (2) the closed-loop expert rollout
    (RolloutExpert of the Sec. 5.1 runtime table: every agent's action fitted
    to the log each step, all metrics incl. kinematic infeasibility), (3)
    log playback of every agent with all metrics."""
    b = R.b
    eb = copy.copy(b)
    eb.kind = np.full_like(b.kind, synth.KIND_BICYCLE)
    edb = copy.copy(R.db)  # shares every device array but the kinds
    edb.kind = torch.as_tensor(eb.kind).cuda()
    edb.c = type(R.db.c).from_buffer_copy(R.db.c)
    edb.c.kind = edb.kind.data_ptr()
    sim = wsim.Sim(edb)
    N, S, T = eb.N_tot, eb.S, eb.T
    st = R.st0.clone()
    act = torch.empty((T, 3, N), dtype=torch.float32, device="cuda")
    sim.autotune(R.st0, R.act, synth.T0, 8)
    out = {"workload": f"{S} scenes x up to {int(np.diff(eb.agent_off).max())} agents x {T} steps, "
                       "every valid agent a bicycle expert"}
    ms = timed(torch, lambda: sim.expert_actions(synth.T0, T, act), reps)
    valid = eb.valid.astype(bool)
    # algorithmic bytes: every action row written (12 B per agent-step); for a
    # valid policy agent its log rows t0 .. t0+T read once (heading, velocity:
    # 12 B per row); kind and valid (2 B per agent)
    nbytes = N * T * 12 + int(valid.sum()) * (T + 1) * 12 + N * 2
    out["expert_actions"] = {"ms": ms, "agent_steps_per_s": N * T / (ms / 1e3),
                             "roofline": hbm_roofline("k_expert_actions", nbytes, ms, traffic=None)}
    for name, ctrl_v in (("rollout_expert", wsim.CTRL_EXPERT), ("rollout_expert_discrete", wsim.CTRL_EXPERT_DISCRETE),
                         ("log_playback", wsim.CTRL_LOG)):
        ctrl = torch.full((N,), ctrl_v, dtype=torch.uint8, device="cuda")

        def run():
            st.data.copy_(R.st0.data)
            sim.rollout(st, None, R.m, synth.T0, T, mode=wsim.MODE_FUSED, ctrl=ctrl)
        ms = timed(torch, run, reps)
        out[name] = {"value": N * T / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms}
        if name.startswith("rollout_expert"):
            lg = R.m.logdiv.cpu().numpy()[:, valid]
            out[name]["ade_m"] = float(lg.mean())
            out[name]["kin_infeasible_frac"] = float(((R.m.flags.cpu().numpy()[:, valid] & 4) != 0).mean())
    assert sim.status() == 0
    sim.close()
    return out


def observe_leg(wsim, synth, torch, R, reps):
    """Observation (Sec. 3.2) of the bench's initial state: (1) the ego of
    every scene with the 256 nearest roadgraph points, (2) every valid agent
    with the 64 nearest; both with all other agents of the scene in the
    observer's frame.  And the route metrics (Sec. 3.4) of every scene."""
    b, sim, st = R.b, R.sim, R.st0
    N = b.N_tot
    M = int(np.diff(b.agent_off).max())
    out = {"workload": f"{b.S} scenes x up to {M} agents, {int(np.diff(b.rg_off).max())}-point roadgraphs"}
    ego = torch.zeros(N, dtype=torch.uint8, device="cuda")
    ego[torch.as_tensor(b.agent_off[:-1].astype(np.int64), device="cuda")] = 1
    for name, obs, K in (("ego_k256", ego, 256), ("all_agents_k64", None, 64)):
        res = sim.observe(st, M, K, observers=obs)
        ms = timed(torch, lambda: sim.observe(st, M, K, observers=obs, out=res), reps, warm=2)
        n_obs = int(obs.sum().item()) if obs is not None else int(b.valid.sum())
        # algorithmic bytes per observer: its rows written (M agents x (5
        # floats + 1 flag), K points x (2 floats + 1 index)) and the scene's
        # agent state read once (x, y, lo words, heading, velocity, valid: 33 B)
        nbytes = n_obs * (M * 21 + K * 12 + M * 33)
        out[name] = {"ms": ms, "observers": n_obs, "observations_per_s": n_obs / (ms / 1e3), "K": K, "M": M,
                     "roofline": hbm_roofline("k_observe", nbytes, ms, traffic=None)}
        del res
    ms = timed(torch, lambda: sim.route_metrics(st), reps, warm=2)
    # per scene: its route path points read once (8 B each), the ego's state
    # and two logged positions (~40 B), 5 B written
    npts = int(b.path_pt_off[-1]) if b.path_pt_off is not None else 0
    out["route_metrics"] = {"ms": ms, "scenes": b.S,
                            "roofline": hbm_roofline("k_route", npts * 8 + b.S * 45, ms, traffic=None)}
    assert sim.status() == 0
    return out


def main():
    args = parse()
    ws, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank, pg)
        return
    import torch
    from paper_2310_08710_b300 import synth, wsim
    torch.cuda.set_device(local)
    seed = args.seed + 1000 * rank
    if args.bptt_only:
        b = make(synth, args.bptt_workload, seed + 1, S=args.bptt_scenes)
        out = bptt_leg(wsim, synth, torch, b, plain=False, reps=args.steps)
        if rank == 0:
            print(json.dumps({"profile": True, "bptt": out}), flush=True)
        return
    b = make(synth, args.workload, seed, S=args.scenes)
    T, N, S = b.T, b.N_tot, b.S
    R = Rollout(wsim, synth, torch, b, args.mode, args.shape)
    if args.expert_only:
        out = expert_leg(wsim, synth, torch, R, args.steps)
        if rank == 0:
            print(json.dumps({"profile": True, "expert": out}), flush=True)
        return
    if args.observe_only:
        out = observe_leg(wsim, synth, torch, R, args.steps)
        if rank == 0:
            print(json.dumps({"profile": True, "observe": out}), flush=True)
        return
    cnt = R.counts()  # work counters of one (untimed) rollout: the roofline numerator
    for _ in range(max(3, args.warmup)):
        R.run()
    torch.cuda.synchronize()
    assert R.sim.status() == 0

    clk = ClockSampler(local)
    time.sleep(0.5)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        R.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if pg:
        pg.barrier()
    clocks = clk.stop()
    assert R.sim.status() == 0
    wkey = f"workload {args.workload}" + (f", {args.scenes} scenes" if args.scenes else "")
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "mode": args.mode, "ms_per_step": ms, "scenes": S, "tune": R.tune,
                              "value": N * T / (ms / 1e3), "counts": cnt}), flush=True)
        return

    ms_e2e, ms_e2e_serial, h2d, d2h = R.e2e(args.steps)
    modes = modes_leg(wsim, synth, torch, R, plain_scenes=256)
    # the batched result: the scene-resident rollout against the per-step
    # paths on the same B300, as ratios of agent-steps/s
    modes["resident_over_graph_of_steps"] = (N * T / (ms / 1e3)) / modes["graph_of_steps"]["value"]
    modes["resident_over_plain_per_scene"] = (N * T / (ms / 1e3)) / modes["plain_per_scene"]["value"]
    observe = observe_leg(wsim, synth, torch, R, args.steps)
    expert = expert_leg(wsim, synth, torch, R, args.steps)
    bptt = {"config3": bptt_leg(wsim, synth, torch, make(synth, 3, seed + 1), plain=True)}
    if args.workload == 4 and S >= 2048:
        bptt["config4_2048"] = bptt_leg(wsim, synth, torch, b.subset(list(range(2048))), plain=False, reps=3)
    launches = R.launches()
    roof = rollout_roofline(synth, b, cnt, ms if args.mode == "fused" else ms / T,
                            "k_rollout" if args.mode == "fused" else "k_step", wkey)
    if launches > 1:
        roof["note"] = f"{launches} concurrent launches (one per size bucket) per rollout; time of the rollout"
    tune = R.tune
    R.close()
    del R

    extra = {}
    if not args.no_extra and args.workload != 1:
        b1 = make(synth, 1, seed)
        R1 = Rollout(wsim, synth, torch, b1, "fused")
        c1 = R1.counts()
        m1 = timed(torch, R1.run, args.steps)
        md1 = modes_leg(wsim, synth, torch, R1, plain_scenes=None)
        extra["config1"] = {"config": workload_config(synth, 1, b=b1), "value": b1.N_tot * b1.T / (m1 / 1e3),
                            "unit": UNIT, "ms_per_rollout": m1, "rollout_tuning": R1.tune,
                            "roofline": rollout_roofline(synth, b1, c1, m1, "k_rollout", "workload 1"),
                            "modes": md1,
                            "resident_over_graph_of_steps": (b1.N_tot * b1.T / (m1 / 1e3))
                            / md1["graph_of_steps"]["value"],
                            "resident_over_plain_per_scene": (b1.N_tot * b1.T / (m1 / 1e3))
                            / md1["plain_per_scene"]["value"]}
        R1.close()

    ms, ms_e2e, ms_e2e_serial, units = combine_ranks(pg, [ms, ms_e2e, ms_e2e_serial], N * T, "cuda")
    _, valid_units = combine_ranks(pg, [ms], int(b.valid.sum()) * T, "cuda")
    if rank != 0:
        return
    value = units / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "value_valid_agents_only": valid_units / (ms / 1e3),
        "data": "synthetic", "config": {**workload_config(synth, args.workload, S, b), "rollout_tuning": tune},
        "roofline": roof,
        "e2e": {"value": units / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "streamed": "next step's inputs up and last step's reward and flags down on a second stream "
                            "during the rollout (two buffer sets)",
                "serial_value": units / (ms_e2e_serial / 1e3)},
        "gpu_launches": args.steps * launches,
        "modes": modes,
        "bptt": bptt,
        "expert": expert,
        "observe": observe,
        "extra": extra,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(synth, args.workload, seed, args.scenes, args.cpu_sample_seconds)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
