#!/usr/bin/env python
"""Throughput of the batched closed-loop rollout on B300.

One step = one 80-step rollout of the whole scene batch: per step of it,
action resolution, IDM sim agents, bicycle/delta dynamics, pairwise box
overlap, off-road signed distance, log divergence and reward (the Step of the
paper's runtime benchmark, Sec. 5.1, driven for a full episode as in its
Rollout column).  Metric: agent-steps/s (agent slots x simulated steps per
second), all scenes on one GPU, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wsim|reference]

Under torchrun every rank simulates its own batch (different seeds) and the
value is the total over ranks divided by the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
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
# FP32 operations per unit of counted work (counted from the kernels' inner loops).
FLOPS_PER_EVAL = 15      # corner x road-edge segment distance
FLOPS_PER_TILE = 10      # culling-tile bound test
FLOPS_PER_PAIR = 44      # ordered SAT pair
FLOPS_PER_TEST = 16      # IDM look-ahead sample x box test
FLOPS_PER_AGENT = 60     # dynamics + log divergence per agent-step
FLOPS_PER_BOUND = 11     # overlap pair bound test (culling)
FLOPS_PER_FILTER = 9     # IDM lead-candidate circle test
FLOPS_PER_IDM_STEP = 800 # IDM agent-step: 32 look-ahead samples on the route, acceleration, advance


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


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the last ncu capture, if it is of this build."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
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
    ap.add_argument("--workload", type=int, default=1,
                    help="synthetic workload id (paper_2310_08710_b300.synth.WORKLOADS); 1 = 1024 scenes x 128 agents, IDM")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="fused", choices=["fused", "graph"],
                    help="rollout path timed: scene-resident kernel or graph of per-step launches")
    ap.add_argument("--scenes", type=int, default=None, help="override the scene count (profiling only)")
    ap.add_argument("--shape", type=int, default=None,
                    help="pin one launch shape of the scene-resident rollout instead of autotuning (profiling)")
    ap.add_argument("--bptt-only", action="store_true", help="run only the BPTT leg (profiling)")
    ap.add_argument("--bptt-workload", type=int, default=3,
                    help="synthetic workload of the BPTT leg (3 = 256 scenes x 64 agents; 4 = the 30k-point sweep)")
    ap.add_argument("--bptt-scenes", type=int, default=None, help="override the BPTT leg's scene count")
    ap.add_argument("--profile", action="store_true",
                    help="time the main path only (no mode comparison, end-to-end or CPU legs)")
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


def workload_desc(cfg):
    from paper_2310_08710_b300 import synth
    wl = synth.WORKLOADS[cfg]
    return wl


def cpu_baseline(b, seconds: float, reps: int = 1) -> dict:
    """The FP64 oracle's free-running rollout on host cores, bounded sample."""
    import oracle
    cores = os.cpu_count() or 1
    # about 6e3 agent-steps/s per core on 128-agent IDM scenes
    per_scene = 0.0
    probe = b.subset([0])
    o = oracle.Oracle(probe)
    t = time.perf_counter()
    o.rollout(o.initial_state(), probe.actions, 10, 8, nthreads=1)
    per_scene = (time.perf_counter() - t) * (b.T / 8)
    n = int(max(1, min(b.S, round(seconds * cores / max(per_scene, 1e-3)))))
    sub = b.subset(list(range(n)))
    o = oracle.Oracle(sub)
    st = o.initial_state()
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        o.rollout(st, sub.actions, 10, b.T, nthreads=cores)
        times.append(time.perf_counter() - t)
    dt = statistics.median(times)
    return {"value": sub.N_tot * b.T / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of {b.S} scenes x {b.T} steps (free-running FP64 rollout, OpenMP over scenes)",
            "seconds": dt}


def run_reference(args, ws, rank, pg):
    from paper_2310_08710_b300 import synth
    if rank != 0:
        return
    b = synth.make_batch(args.workload, seed=args.seed, S=args.scenes,
                         workers=gen_workers(args.scenes or synth.WORKLOADS[args.workload].S))
    import oracle
    cores = os.cpu_count() or 1
    # size each step so that the whole run stays within a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    probe = b.subset([0])
    o = oracle.Oracle(probe)
    t = time.perf_counter()
    o.rollout(o.initial_state(), probe.actions, 10, 8, nthreads=1)
    per_scene = (time.perf_counter() - t) * (b.T / 8)
    n = int(max(1, min(b.S, budget * cores / max(per_scene, 1e-3) * 0.8)))
    sub = b.subset(list(range(n)))
    o = oracle.Oracle(sub)
    st = o.initial_state()
    for _ in range(args.warmup):
        o.rollout(st, sub.actions, 10, b.T, nthreads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.rollout(st, sub.actions, 10, b.T, nthreads=cores)
    dt = (time.perf_counter() - t) / args.steps
    v = sub.N_tot * b.T / dt
    sample = f"{n} of {b.S} scenes x {b.T} steps per step (free-running FP64 rollout, OpenMP over scenes)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, b),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bptt_leg(wsim, synth, torch, args, rank):
    """Gradient steps/s of the differentiable rollout (256 scenes x 64 agents x
    80 steps, bicycle agents, synthetic workload 3): one gradient step = forward rollout with the
    loss plus the reverse sweep giving dL/d(every action)."""
    b = synth.make_batch(args.bptt_workload, seed=args.seed + 1000 * rank, S=args.bptt_scenes,
                         workers=gen_workers(args.bptt_scenes or synth.WORKLOADS[args.bptt_workload].S))
    sim = wsim.Sim(wsim.DeviceBatch(b))
    st = wsim.State.from_batch(b)
    act = torch.as_tensor(b.actions).cuda().contiguous()
    out = {"workload": f"{b.S} scenes x up to {int(np.diff(b.agent_off).max())} agents x {b.T} steps "
                       f"({synth.WORKLOADS[args.bptt_workload].name}), "
                       "loss = log divergence^2 + softplus overlap"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, ck, plain, reps in (("ckpt10", 10, False, 5), ("store_all", 1, False, 5), ("plain_per_scene_ckpt10", 10, True, 1)):
        sim.loss_grad(st, act, synth.T0, b.T, ck, plain=plain)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            sim.loss_grad(st, act, synth.T0, b.T, ck, plain=plain)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"grad_steps_per_s": 1e3 / ms, "ms": ms, "agent_steps_per_s": b.N_tot * b.T / (ms / 1e3)}
    stc, mf = st.clone(), wsim.Metrics(b.N_tot, b.S, rows=b.T)
    sim.rollout(stc, act, mf, synth.T0, b.T, mode=wsim.MODE_FUSED)
    e0.record()
    for _ in range(5):
        stc.data.copy_(st.data)
        sim.rollout(stc, act, mf, synth.T0, b.T, mode=wsim.MODE_FUSED)
    e1.record()
    torch.cuda.synchronize()
    out["forward_rollout_ms"] = e0.elapsed_time(e1) / 5
    assert sim.status() == 0
    sim.close()
    return out


def gen_workers(scenes: int) -> int:
    """Processes that draw the synthetic scenes (large batches only)."""
    return min(32, os.cpu_count() or 1) if scenes >= 512 else 1


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


def expert_leg(wsim, synth, torch, args, rank, b, reps):
    """The paper's expert actor (Sec. 5.2) on the bench's scenes with every
    valid agent a bicycle policy agent: (1) the open-loop expert actions of
    all 80 steps (one HBM-bound launch), (2) the closed-loop expert rollout
    (RolloutExpert of the Sec. 5.1 runtime table: every agent's action fitted
    to the log each step, all metrics incl. kinematic infeasibility), (3)
    log playback of every agent with all metrics."""
    import copy
    eb = copy.copy(b)
    eb.kind = np.full_like(b.kind, synth.KIND_BICYCLE)
    sim = wsim.Sim(wsim.DeviceBatch(eb))
    N, S, T = eb.N_tot, eb.S, eb.T
    st0 = wsim.State.from_batch(eb)
    st = st0.clone()
    m = wsim.Metrics(N, S, rows=T)
    act = torch.empty((T, 3, N), dtype=torch.float32, device="cuda")
    sim.autotune(st0, torch.as_tensor(eb.actions).cuda().contiguous(), synth.T0, 8)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    out = {"workload": f"{S} scenes x up to {int(np.diff(eb.agent_off).max())} agents x {T} steps, "
                       "every valid agent a bicycle expert"}

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: sim.expert_actions(synth.T0, T, act))
    valid = eb.valid.astype(bool)
    # algorithmic bytes: every action row written (12 B per agent-step); for a
    # valid policy agent its log rows t0 .. t0+T read once (heading, velocity:
    # 12 B per row); kind and valid (2 B per agent)
    nbytes = N * T * 12 + int(valid.sum()) * (T + 1) * 12 + N * 2
    peak, src = hbm_peak_gbs()
    gbs = nbytes / (ms / 1e3) / 1e9
    out["expert_actions"] = {"ms": ms, "agent_steps_per_s": N * T / (ms / 1e3),
                             "roofline": {"bound": "hbm", "kernel": "k_expert_actions", "achieved": gbs,
                                          "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                          "bytes_per_launch": nbytes, "peak_source": src, "traffic": None}}
    for name, ctrl_v in (("rollout_expert", wsim.CTRL_EXPERT), ("rollout_expert_discrete", wsim.CTRL_EXPERT_DISCRETE),
                         ("log_playback", wsim.CTRL_LOG)):
        ctrl = torch.full((N,), ctrl_v, dtype=torch.uint8, device="cuda")

        def run():
            st.data.copy_(st0.data)
            sim.rollout(st, None, m, synth.T0, T, mode=wsim.MODE_FUSED, ctrl=ctrl)
        ms = timed(run)
        out[name] = {"value": N * T / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms}
        if name.startswith("rollout_expert"):
            lg = m.logdiv.cpu().numpy()[:, valid]
            out[name]["ade_m"] = float(lg.mean())
            out[name]["kin_infeasible_frac"] = float(((m.flags.cpu().numpy()[:, valid] & 4) != 0).mean())
    assert sim.status() == 0
    sim.close()
    return out


def observe_leg(wsim, synth, torch, b, sim, st, reps):
    """Observation (Sec. 3.2) of the bench's state: (1) the ego of every scene
    with the 256 nearest roadgraph points, (2) every valid agent with the 64
    nearest; both with all other agents of the scene in the observer's frame."""
    N = b.N_tot
    M = int(np.diff(b.agent_off).max())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{b.S} scenes x up to {M} agents, {int(np.diff(b.rg_off).max())}-point roadgraphs"}
    ego = torch.zeros(N, dtype=torch.uint8, device="cuda")
    ego[torch.as_tensor(b.agent_off[:-1].astype(np.int64), device="cuda")] = 1
    for name, obs, K in (("ego_k256", ego, 256), ("all_agents_k64", None, 64)):
        res = sim.observe(st, M, K, observers=obs)
        for _ in range(2):
            sim.observe(st, M, K, observers=obs, out=res)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            sim.observe(st, M, K, observers=obs, out=res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        n_obs = int(obs.sum().item()) if obs is not None else int(b.valid.sum())
        out[name] = {"ms": ms, "observers": n_obs, "observations_per_s": n_obs / (ms / 1e3), "K": K, "M": M}
        del res
    prog, offr = sim.route_metrics(st)
    for _ in range(2):
        sim.route_metrics(st)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        sim.route_metrics(st)
    e1.record()
    torch.cuda.synchronize()
    out["route_metrics"] = {"ms": e0.elapsed_time(e1) / reps, "scenes": b.S}
    assert sim.status() == 0
    return out


def config_dict(args, b):
    wl = workload_desc(args.workload)
    return {"workload": wl.name, "scenes": int(b.S),
            "agents": int(b.N_tot), "rollout_steps": int(b.T), "roadgraph_points": int(b.R_tot),
            "dt_s": 0.1, "rollout_mode": ("scene-resident rollout kernel (one launch per rollout)"
                                          if args.mode == "fused" else "persistent step kernel x80, CUDA graph"),
            "l2": "inputs larger than L2 (road-edge segments + routes + logs streamed every rollout)"}


def main():
    args = parse()
    ws, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank, pg)
        return
    import torch
    from paper_2310_08710_b300 import synth, wsim
    torch.cuda.set_device(local)
    if args.bptt_only:
        out = bptt_leg(wsim, synth, torch, args, rank)
        if rank == 0:
            print(json.dumps({"profile": True, "bptt": out}), flush=True)
        return
    b = synth.make_batch(args.workload, seed=args.seed + 1000 * rank, S=args.scenes,
                         workers=gen_workers(args.scenes or synth.WORKLOADS[args.workload].S))
    T, N, S = b.T, b.N_tot, b.S
    main_mode = wsim.MODE_FUSED if args.mode == "fused" else wsim.MODE_GRAPH
    db = wsim.DeviceBatch(b)
    sim = wsim.Sim(db)
    st0 = wsim.State.from_batch(b)
    st = st0.clone()
    act = torch.as_tensor(b.actions).cuda().contiguous()
    m = wsim.Metrics(N, S, rows=T)
    stream = torch.cuda.current_stream()

    def rollout():
        st.data.copy_(st0.data)
        sim.rollout(st, act, m, synth.T0, T, mode=main_mode)

    # Launch shapes per scene-size bucket, tuned on this workload (untimed).
    if args.shape is not None:
        sim.set_tuning(single_shape=args.shape)
        tune = sim.get_tuning()
    else:
        tune = sim.autotune(st0, act, synth.T0, 8) if main_mode == wsim.MODE_FUSED else None

    # Work counters of one rollout (untimed) for the roofline numerator.
    sim.set_counting(True)
    rollout()
    cnt = [int(x) for x in sim.counters()]
    sim.set_counting(False)
    for _ in range(max(3, args.warmup)):
        rollout()
    torch.cuda.synchronize()
    assert sim.status() == 0

    clk = ClockSampler(local)
    time.sleep(0.5)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rollout()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if pg:
        pg.barrier()
    clocks = clk.stop()
    assert sim.status() == 0

    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "mode": args.mode, "ms_per_step": ms, "scenes": S, "tune": tune,
                              "value": N * T / (ms / 1e3), "counts": cnt}), flush=True)
        return
    # End to end through the public API: pinned host inputs in, metrics out.
    h_act = torch.as_tensor(b.actions).pin_memory()
    h_st = st0.data.cpu().pin_memory()
    h_rew = torch.empty((T, S), dtype=torch.int32).pin_memory()
    h_flags = torch.empty((T, N), dtype=torch.uint8).pin_memory()
    for _ in range(2):
        act.copy_(h_act, non_blocking=True)
        st.data.copy_(h_st, non_blocking=True)
        sim.rollout(st, act, m, synth.T0, T, mode=main_mode)
        h_rew.copy_(m.reward, non_blocking=True)
        h_flags.copy_(m.flags, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        act.copy_(h_act, non_blocking=True)
        st.data.copy_(h_st, non_blocking=True)
        sim.rollout(st, act, m, synth.T0, T, mode=main_mode)
        h_rew.copy_(m.reward, non_blocking=True)
        h_flags.copy_(m.flags, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    h2d = h_act.numel() * 4 + h_st.numel() * 4
    d2h = h_rew.numel() * 4 + h_flags.numel()

    # The same rollout through the per-step paths, one timed rollout each:
    # a CUDA graph of T persistent step launches, and one launch per scene
    # and phase (the plain baseline).
    modes = {}
    for name, mode, reps in (("graph_of_steps", wsim.MODE_GRAPH, 3), ("plain_per_scene", wsim.MODE_PLAIN, 1)):
        st.data.copy_(st0.data)
        sim.rollout(st, act, m, synth.T0, T, mode=mode)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            st.data.copy_(st0.data)
            sim.rollout(st, act, m, synth.T0, T, mode=mode)
        e1.record(stream)
        torch.cuda.synchronize()
        mm = e0.elapsed_time(e1) / reps
        modes[name] = {"value": N * T / (mm / 1e3), "unit": UNIT, "ms_per_rollout": mm, "rollouts_timed": reps}
    assert sim.status() == 0

    observe = observe_leg(wsim, synth, torch, b, sim, st0, args.steps)
    bptt = bptt_leg(wsim, synth, torch, args, rank)
    expert = expert_leg(wsim, synth, torch, args, rank, b, args.steps)

    ms, ms_e2e, units = combine_ranks(pg, [ms, ms_e2e], N * T, "cuda")
    _, valid_units = combine_ranks(pg, [ms], int(b.valid.sum()) * T, "cuda")
    if rank != 0:
        return
    value = units / (ms / 1e3)
    fused = args.mode == "fused"
    # fused: one scene-resident launch per rollout; graph: T step launches
    # (each preceded by a 4-byte memset node, counted in the launch time)
    launch_ms = ms if fused else ms / T
    launches = T if not fused else (sum(1 for n in tune["bucket_scenes"] if n) if tune and tune["split"] else 1)
    idm_steps = int(((b.kind == synth.KIND_IDM) & (b.valid != 0)).sum()) * T
    flops = (FLOPS_PER_EVAL * cnt[0] + FLOPS_PER_TILE * cnt[1] + FLOPS_PER_PAIR * cnt[2] + FLOPS_PER_TEST * cnt[3]
             + FLOPS_PER_BOUND * cnt[4] + FLOPS_PER_FILTER * cnt[5] + FLOPS_PER_IDM_STEP * idm_steps
             + FLOPS_PER_AGENT * N * T) / launches
    achieved = flops / (launch_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "value_valid_agents_only": valid_units / (ms / 1e3),
        "data": "synthetic", "config": {**config_dict(args, b), "rollout_tuning": tune},
        "roofline": {"bound": "alu", "kernel": "k_rollout" if fused else "k_step", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": recorded_traffic("k_rollout") if fused else None,
                     "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz",
                     "flops_per_launch": flops, "launch_ms": launch_ms,
                     "counts_per_rollout": {"corner_segment_evals": int(cnt[0]), "tile_tests": int(cnt[1]),
                                            "sat_pairs": int(cnt[2]), "idm_sample_tests": int(cnt[3]),
                                            "pair_bound_tests": int(cnt[4]), "idm_circle_tests": int(cnt[5]),
                                            "idm_agent_steps": idm_steps}},
        "e2e": {"value": units / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": args.steps * launches,
        "modes": modes,
        "bptt": bptt,
        "expert": expert,
        "observe": observe,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(b, args.cpu_sample_seconds)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
