"""Throughput of the dual adaptive explicit monodomain solver on the 3D slab.

Workload (one bench "step"): the anisotropic TP06 slab, 101 x 101 x 26 nodes
(265 226), h = 0.02 cm, fibres rotating -60..+60 deg through the wall, corner
stimulus, 500 ms simulated with the 0.1 ms splitting step (5 000 Strang
steps) from the published initial state.  Metric: node-steps/s =
nodes x Strang steps / wall-second (whole job), and simulated ms per wall-s;
FP32 (compensated V) is the headline, FP64 is measured beside it together
with the FP32-vs-FP64 difference in mV and ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (plain FP64 numpy, one host core) on
a bounded sample of the same workload: the full slab over the first 2 ms of
the simulation (20 Strang steps) per bench step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s and sim-ms per wall-s, 3D slab; FP32 vs FP64 GPU at stated mV error"
UNIT = "node-steps/s"
SLAB = dict(nx=101, ny=101, nz=26, h=0.02)
T_END = 500.0
ORACLE_SAMPLE_STEPS = 20


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


def _clock_sampler(path):
    cmd = ["nvidia-smi",
           "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def _clock_summary(path, dev_index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9 or p[0] != str(dev_index):
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
    except FileNotFoundError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_reference(args):
    """CPU oracle on a bounded sample of the slab workload."""
    rank, world = _dist()
    if rank != 0:
        return
    import inputs
    from oracle import scheme

    wl = inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    times = []
    n_nodes = wl.n_nodes
    for it in range(args.warmup + args.steps):
        sim = scheme.simulation_from_workload(wl)
        t0 = time.perf_counter()
        sim.run(ORACLE_SAMPLE_STEPS)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    sec = sum(times) / len(times)
    value = n_nodes * ORACLE_SAMPLE_STEPS / sec
    sample = f"full slab ({n_nodes} nodes), first {ORACLE_SAMPLE_STEPS} Strang steps (2 ms incl. the stimulus) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "tp06_slab_101x101x26_h0.02", "sample_steps": ORACLE_SAMPLE_STEPS},
        "sim_ms_per_wall_s": ORACLE_SAMPLE_STEPS * 0.1 / sec,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _cpu_baseline_sample():
    import inputs
    from oracle import scheme

    wl = inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    sim = scheme.simulation_from_workload(wl)
    t0 = time.perf_counter()
    sim.run(ORACLE_SAMPLE_STEPS)
    sec = time.perf_counter() - t0
    return {"value": wl.n_nodes * ORACLE_SAMPLE_STEPS / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"full slab, first {ORACLE_SAMPLE_STEPS} Strang steps (2 ms), numpy FP64, {sec:.1f} s"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import inputs
    from paper_2011_04747_gb300 import binding, build as _build

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if not os.path.exists(binding.LIB_PATH):
        if rank == 0:
            _build.build()
        if world > 1:
            dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    wl = inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    n_nodes = wl.n_nodes
    n_steps = int(round(T_END / wl.dt))

    def make(prec):
        s = binding.solver_from_workload(wl, precision=prec, graph_steps=args.graph_steps,
                                         bucket_k=bool(args.bucket))
        s.daeti_set_stream(stream)
        return s

    flush = torch.empty(int(256 * 2 ** 20 // 4), dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def timed_runs(solver, k, w):
        ck = solver.daeti_save_state()                  # initial state
        times = []
        for it in range(w + k):
            solver.daeti_load_state(ck)
            flush.fill_(float(it))
            torch.cuda.synchronize(dev)
            if world > 1:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.daeti_advance(T_END)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if it >= w:
                times.append(e0.elapsed_time(e1) / 1e3)
        solver.daeti_synchronize()
        return times

    # ---- FP32 (headline) ------------------------------------------------------------
    s32 = make("fp32_kahan")
    stab = s32.daeti_get_stability()
    clk_path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    sampler, fh = _clock_sampler(clk_path)
    t32 = timed_runs(s32, args.steps, args.warmup)
    if sampler:
        sampler.terminate()
        sampler.wait()
        fh.close()
    clocks = _clock_summary(clk_path, local)
    v32 = s32.daeti_read_v()
    a32 = s32.daeti_read_activation()
    sub32 = s32.daeti_get_substeps()
    sec32 = sum(t32) / len(t32)
    if world > 1:
        tt = torch.tensor([sec32], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        sec32 = float(tt.item())
    value = world * n_nodes * n_steps / sec32

    # ---- per-kernel timing pass (CUDA events around every launch, no graph) ------------
    ck = None
    s32.daeti_set_profiling(True)
    s32.daeti_init_state()
    s32.daeti_advance(T_END)
    s32.daeti_synchronize()
    kt = {}
    for which, name in ((0, "reaction"), (1, "diffusion"), (2, "bucket")):
        ms, nl = s32.daeti_get_kernel_time(which)
        b, f = s32.daeti_kernel_work(which)
        kt[name] = {"total_ms": ms, "launches": nl, "avg_us": 1e3 * ms / max(nl, 1), "bytes_per_launch": b}
    s32.daeti_set_profiling(False)

    # ---- e2e through the C ABI with host buffers -----------------------------------
    state0 = None
    e2e_times = []
    for it in range(2 + max(1, args.steps // 2)):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s32.daeti_init_state(state0)                    # host -> device
        s32.daeti_advance(T_END)
        vh = s32.daeti_read_v()                         # device -> host (waits)
        ah = s32.daeti_read_activation()
        t1 = time.perf_counter()
        if it >= 2:
            e2e_times.append(t1 - t0)
    n_states = s32.n_states
    h2d = n_nodes * (n_states + 2) * 4
    d2h = 2 * n_nodes * 8
    e2e_val = world * n_nodes * n_steps / (sum(e2e_times) / len(e2e_times))
    s32.close()

    # ---- FP64 beside it -------------------------------------------------------------
    sec64, dv, dact = None, None, None
    if not args.no_fp64:
        s64 = make("fp64")
        t64 = timed_runs(s64, max(1, args.steps // 2), 1)
        v64 = s64.daeti_read_v()
        a64 = s64.daeti_read_activation()
        s64.close()
        sec64 = sum(t64) / len(t64)
        both = (a32 >= 0) & (a64 >= 0)
        dv = float(np.max(np.abs(v32 - v64)))
        dact = float(np.max(np.abs(a32[both] - a64[both]))) if both.any() else None

    # ---- roofline of the dominant kernel -----------------------------------------------
    peaks = _peaks()
    dom = max(("reaction", "diffusion", "bucket"), key=lambda k: kt[k]["total_ms"])
    sub_per_launch = sub32 / max(len(t32) + args.warmup, 1) / n_steps if sub32 else None
    if dom == "diffusion":
        roof = {"bound": "hbm", "achieved": kt[dom]["bytes_per_launch"] / (kt[dom]["avg_us"] * 1e-6) / 1e9,
                "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s"}
    else:
        roof = {"bound": "hbm", "achieved": kt[dom]["bytes_per_launch"] / (kt[dom]["avg_us"] * 1e-6) / 1e9,
                "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["kernel"] = dom

    launches_per_step = 2 * stab["l"] + 2
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec32 * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "tp06_slab_101x101x26_h0.02_500ms", "nodes": n_nodes, "strang_steps": n_steps,
                   "dt_ms": wl.dt, "l": stab["l"], "k_max": stab["k_max"], "dt_s_ms": stab["dt_s"],
                   "precision": "fp32_kahan", "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{world}"},
        "sim_ms_per_wall_s": T_END / sec32,
        "fp64": None if sec64 is None else {"value": world * n_nodes * n_steps / sec64,
                                             "ms_per_step": sec64 * 1e3, "sim_ms_per_wall_s": T_END / sec64},
        "fp32_vs_fp64": {"max_abs_dv_mv_at_500ms": dv, "max_abs_dact_ms": dact},
        "reaction_substeps_per_node_step": sub_per_launch / n_nodes if sub_per_launch else None,
        "kernels": kt,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": (launches_per_step * n_steps + n_steps // max(args.graph_steps, 1)) * args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def profile_run(args):
    """A short plain run of the bench workload for external profilers."""
    import inputs
    from paper_2011_04747_gb300 import binding, build as _build

    if not os.path.exists(binding.LIB_PATH):
        _build.build()
    wl = inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    s = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=args.graph_steps,
                                     bucket_k=bool(args.bucket))
    s.daeti_advance(args.profile_run)
    s.daeti_synchronize()
    s.close()
    print(f"profile run: {args.profile_run} ms simulated")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--graph-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--bucket", type=int, default=1, help="group nodes by k before step A (1) or not (0)")
    ap.add_argument("--profile-run", type=float, default=0.0,
                    help="only simulate this many ms once on the slab (FP32), for profilers; no timing")
    args = ap.parse_args()
    if args.profile_run > 0:
        profile_run(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
