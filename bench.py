"""Throughput of the dual adaptive explicit monodomain solver.

Headline workload (one bench "step"): the anisotropic TP06 slab, 101 x 101 x
26 nodes (265 226), h = 0.02 cm, fibres rotating -60..+60 deg through the
wall, corner stimulus, 500 ms simulated with the 0.1 ms splitting step (5 000
Strang steps) from the published initial state.  Metric: node-steps/s =
nodes x Strang steps / wall-second (whole job) and simulated ms per wall-s;
FP32 with compensated V is the headline, FP64 is measured beside it with the
FP32-vs-FP64 difference in mV and ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload slab|slab_l|square|sheet|tets|batch|adjoint]

``--impl reference`` times the CPU oracle (plain FP64 numpy, one host core) on
a bounded sample of the same workload.  Other workloads print their own line
(they are not the headline).  Under torchrun every rank runs its own replica
(weak scaling, no data-path collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s and sim-ms per wall-s, 3D slab; FP32 vs FP64 GPU at stated mV error"
UNIT = "node-steps/s"
SLAB = dict(nx=101, ny=101, nz=26, h=0.02)
T_END = 500.0
ORACLE_SAMPLE_STEPS = 20
# the CPU-baseline window: Strang steps 100..119 (10-12 ms), while the
# wavefront crosses the slab (the first 2 ms are the stimulus at rest)
ORACLE_WINDOW_START = 100
REDUCED_SLAB = dict(nx=25, ny=23, nz=7)    # FP32 vs the oracle over the whole 500 ms
SM_COUNT = 152
FP32_LANES_PER_SM = 128
XU_LANES_PER_SM = 16
TP06_XU_PER_SUBSTEP = 82.0     # SFU (MUFU) instructions per TP06 sub-step, ncu opcode count (profiles/)
# DRAM bytes (read + write) per reaction launch, mean of three resting-phase
# launches captured with warm caches (profiles/reaction_tp06_fp32_slab.md; the
# state stays in L2)
REACTION_DRAM_BYTES_PER_LAUNCH = 12373.0


def _dist():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


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
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ reference arm
def _oracle_at_window(wl):
    """The oracle advanced (untimed) to the start of the CPU-baseline window."""
    from oracle import scheme

    sim = scheme.simulation_from_workload(wl)
    sim.run(ORACLE_WINDOW_START)
    return sim


def _oracle_snapshot(sim):
    return (sim.S.copy(), sim.n, sim.v_sync.copy(), sim.k.copy(), sim.act.copy(), sim.rrate.copy())


def _oracle_restore(sim, snap):
    S, n, vs, k, act, rr = snap
    sim.S[:] = S
    sim.n = n
    sim.v_sync[:] = vs
    sim.k[:] = k
    sim.act[:] = act
    sim.rrate[:] = rr


def _oracle_window_seconds(sim, snap, steps):
    _oracle_restore(sim, snap)
    t0 = time.perf_counter()
    sim.run(steps)
    return time.perf_counter() - t0


def _window_worker(slab, t_end, steps, barrier, out):
    """One host core of the all-core baseline: its own oracle on the same window."""
    import inputs

    sim = _oracle_at_window(inputs.tp06_slab_3d(**slab, t_end=t_end))
    snap = _oracle_snapshot(sim)
    barrier.wait()
    out.put(_oracle_window_seconds(sim, snap, steps))


def _all_core_window(steps):
    """Every host core runs the oracle on the window at once (spawned
    processes, one numpy thread each); aggregate node-steps/s."""
    import multiprocessing as mp

    import inputs

    cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_window_worker, args=(SLAB, T_END, steps, barrier, out)) for _ in range(cores)]
    for p in procs:
        p.start()
    secs = [out.get() for _ in procs]
    for p in procs:
        p.join()
    n = inputs.tp06_slab_3d(**SLAB, t_end=T_END).n_nodes
    return {"value": sum(n * steps / t for t in secs), "cores": cores, "max_s": max(secs)}


def run_reference(args):
    """CPU oracle on a bounded sample of the slab workload (rank 0 only):
    each timed step runs the oracle over Strang steps 100..119 (10-12 ms,
    the wavefront crossing the slab) from a state the oracle reached itself."""
    rank, world = _dist()
    if rank != 0:
        return
    import inputs

    wl = inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    sim = _oracle_at_window(wl)
    snap = _oracle_snapshot(sim)
    times = []
    for it in range(args.warmup + args.steps):
        sec = _oracle_window_seconds(sim, snap, ORACLE_SAMPLE_STEPS)
        if it >= args.warmup:
            times.append(sec)
    sec = sum(times) / len(times)
    value = wl.n_nodes * ORACLE_SAMPLE_STEPS / sec
    sample = (f"full slab ({wl.n_nodes} nodes), Strang steps {ORACLE_WINDOW_START}..{ORACLE_WINDOW_START + ORACLE_SAMPLE_STEPS - 1} "
              f"(wavefront) per step, numpy FP64 on one host core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "tp06_slab_101x101x26_h0.02", "sample_steps": ORACLE_SAMPLE_STEPS,
                   "window_start_step": ORACLE_WINDOW_START},
        "sim_ms_per_wall_s": ORACLE_SAMPLE_STEPS * 0.1 / sec,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _cpu_baseline_slab(wl, all_cores=True):
    """The oracle on the wavefront window of the slab: one core, and every core at once."""
    sim = _oracle_at_window(wl)
    snap = _oracle_snapshot(sim)
    sec = _oracle_window_seconds(sim, snap, ORACLE_SAMPLE_STEPS)
    out = {"value": wl.n_nodes * ORACLE_SAMPLE_STEPS / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{wl.name}: Strang steps {ORACLE_WINDOW_START}..{ORACLE_WINDOW_START + ORACLE_SAMPLE_STEPS - 1} "
                     f"(10-12 ms, wavefront) from the oracle's own state, numpy FP64, one host core, {sec:.1f} s"}
    if all_cores:
        try:
            out["all_cores"] = _all_core_window(ORACLE_SAMPLE_STEPS)
            out["all_cores"]["unit"] = UNIT
            out["all_cores"]["sample"] = "the same window run by one oracle process per host core at once"
        except Exception as e:          # reported, not fatal: the GPU numbers stand without it
            out["all_cores"] = {"error": repr(e)}
    return out


def _cpu_baseline_sample(wl, steps=ORACLE_SAMPLE_STEPS):
    from oracle import scheme

    sim = scheme.simulation_from_workload(wl)
    t0 = time.perf_counter()
    sim.run(steps)
    sec = time.perf_counter() - t0
    return {"value": wl.n_nodes * steps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{wl.name}: first {steps} Strang steps, numpy FP64, one host core, {sec:.1f} s"}


# ------------------------------------------------------------------ our arm
def max_over_ranks(dist, x, device, world):
    """The slowest rank's time: whole-job throughput divides by it."""
    if world == 1:
        return x
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Env:
    def __init__(self, args):
        import torch
        import torch.distributed as dist

        from paper_2011_04747_gb300 import binding, build as _build

        self.torch, self.dist, self.binding = torch, dist, binding
        self.rank, self.world = _dist()
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if self.world > 1:
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        torch.cuda.set_device(self.local)
        if not os.path.exists(binding.LIB_PATH):
            if self.rank == 0:
                _build.build()
            if self.world > 1:
                dist.barrier()
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.current_stream(self.dev)
        self.flush = torch.empty(int(256 * 2 ** 20 // 4), dtype=torch.float32, device=self.dev)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max_over_ranks(self, x):
        return max_over_ranks(self.dist, x, self.dev, self.world)

    def timed(self, fn, k, w, reset=None):
        """Average seconds of fn() over k timed repetitions after w warm-ups,
        CUDA events on the launching stream, L2 flushed before each one."""
        torch = self.torch
        times = []
        for it in range(w + k):
            if reset:
                reset()
            self.flush.fill_(float(it))
            torch.cuda.synchronize(self.dev)
            self.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            torch.cuda.synchronize(self.dev)
            if it >= w:
                times.append(e0.elapsed_time(e1) / 1e3)
        return self.max_over_ranks(sum(times) / len(times))


def _launch_samples(s, ck, n_steps, dt, every_ms=10.0, count=20):
    """Reaction and synchronising-diffusion launch durations (us) at states of
    one run, by daeti_time_launches, with the run's sub-steps per launch."""
    s.daeti_load_state(ck)
    out = []
    t = every_ms / 2
    while t < n_steps * dt:
        s.daeti_advance(t)
        snap = s.daeti_save_state()
        sub0 = s.daeti_get_substeps()
        r_ms = s.daeti_time_launches(0, count)
        sub = (s.daeti_get_substeps() - sub0) / (2 * count)      # warm-up replay + timed replay
        s.daeti_load_state(snap)
        s.daeti_advance(t + dt)                                   # back in the run's bucketing mode
        d_ms = s.daeti_time_launches(2, count)
        s.daeti_load_state(snap)
        out.append({"t_ms": t, "reaction_us": r_ms * 1e3, "sync_diffusion_us": d_ms * 1e3,
                    "substeps_per_launch": sub})
        t += every_ms
    return out


def _aligned_max_dv(snaps_a, snaps_b, act_a, act_b, every_ms, after_ms=5.0):
    """max over nodes and snapshots t >= act_a + after_ms of |V_a(t) - V_b(t + act_b - act_a)|
    (V_b linearly interpolated between snapshots; reading R-dV: traces aligned
    by their activation times; the upstroke itself is left out, where 1 ms
    snapshots cannot resolve a ~300 mV/ms slope)."""
    import numpy as np

    m, n = snaps_a.shape
    t = (np.arange(m) + 1) * every_ms
    both = (act_a >= 0) & (act_b >= 0)
    shift = np.where(both, act_b - act_a, 0.0)
    worst = 0.0
    cols = np.arange(n)
    for j in range(m):
        ok = both & (t[j] >= act_a + after_ms)
        f = (t[j] + shift) / every_ms - 1.0
        i0 = np.floor(f).astype(np.int64)
        ok &= (i0 >= 0) & (i0 < m - 1)
        if not ok.any():
            continue
        i0c = np.clip(i0, 0, m - 2)
        w = f - i0c
        vb = (1.0 - w) * snaps_b[i0c, cols] + w * snaps_b[i0c + 1, cols]
        d = np.abs(snaps_a[j].astype(np.float64) - vb)[ok]
        worst = max(worst, float(d.max()))
    return worst


def _fp32_vs_fp64(s32, ck, s64, n_steps, dt, every=10):
    """Lockstep FP32 and FP64 runs of the same workload from the same initial
    state, V of every node every `every` steps (1 ms) over the whole run."""
    import numpy as np

    s32.daeti_load_state(ck)
    s64.daeti_init_state(None)
    m = n_steps // every
    n = s32.n_nodes
    a32, a64 = np.empty((m, n), np.float32), np.empty((m, n), np.float32)
    for j in range(m):
        t = (j + 1) * every * dt
        s32.daeti_advance(t)
        s64.daeti_advance(t)
        a32[j] = s32.daeti_read_v()
        a64[j] = s64.daeti_read_v()
    act32, act64 = s32.daeti_read_activation(), s64.daeti_read_activation()
    dv_t = np.abs(a32.astype(np.float64) - a64.astype(np.float64)).max(axis=1)
    both = (act32 >= 0) & (act64 >= 0)
    out = {"snapshots": m, "snapshot_every_ms": every * dt,
           "max_abs_dv_mv": float(dv_t.max()), "at_ms": float((int(np.argmax(dv_t)) + 1) * every * dt),
           "max_abs_dv_mv_at_end": float(dv_t[-1]),
           "max_abs_dv_mv_aligned_from_5ms_after_activation":
               _aligned_max_dv(a32, a64, act32, act64, every * dt),
           "max_abs_dact_ms": float(np.abs(act32[both] - act64[both]).max()) if both.any() else None,
           "same_activated_set": bool(np.array_equal(act32 >= 0, act64 >= 0))}
    del a32, a64
    return out


def _fp32_vs_oracle_reduced(binding):
    """FP32 GPU vs the FP64 oracle on a reduced slab (same physics, 25 x 23 x 7
    nodes) over the whole 500 ms, V of every node every 1 ms."""
    import numpy as np

    import inputs
    from oracle import scheme

    wl = inputs.tp06_slab_3d(**REDUCED_SLAB, t_end=T_END)
    n_steps, every = int(round(T_END / wl.dt)), 10
    g = binding.solver_from_workload(wl, precision="fp32_kahan")
    sim = scheme.simulation_from_workload(wl)
    t0 = time.perf_counter()
    m = n_steps // every
    gs, os_ = np.empty((m, wl.n_nodes)), np.empty((m, wl.n_nodes))
    for j in range(m):
        g.daeti_advance((j + 1) * every * wl.dt)
        gs[j] = g.daeti_read_v()
        sim.run(every)
        os_[j] = sim.S[0]
    ga = g.daeti_read_activation()
    g.close()
    dv_t = np.abs(gs - os_).max(axis=1)
    both = (ga >= 0) & (sim.act >= 0)
    return {"workload": f"tp06_slab_{wl.n[0]}x{wl.n[1]}x{wl.n[2]}_h0.02_500ms", "nodes": wl.n_nodes,
            "max_abs_dv_mv": float(dv_t.max()), "at_ms": float((int(np.argmax(dv_t)) + 1) * every * wl.dt),
            "max_abs_dv_mv_aligned_from_5ms_after_activation": _aligned_max_dv(gs, os_, ga, sim.act, every * wl.dt),
            "max_abs_dact_ms": float(np.abs(ga[both] - sim.act[both]).max()) if both.any() else None,
            "same_activated_set": bool(np.array_equal(ga >= 0, sim.act >= 0)),
            "oracle_s": time.perf_counter() - t0}


def _adjoint_precision(binding, stream):
    """Adjoint workload (256 x 256 MS, 2000 steps, 64 sensors every 1 ms,
    32 slots): FP32 gradient against the FP64 gradient of the same schedule."""
    import numpy as np

    import inputs

    wl, d_node, sensors, _ = inputs.ms_adjoint_2d()
    nx = wl.n[0]
    ey, ex = np.meshgrid(np.arange(nx - 1), np.arange(nx - 1), indexing="ij")
    conn = (ex + nx * ey).ravel()[:, None] + np.array([0, 1, nx, nx + 1])[None, :]

    def solver(de, prec):
        w = inputs.Workload(**{**wl.__dict__, "d_long": de, "d_trans": de, "fibre": None})
        s = binding.solver_from_workload(w, precision=prec)
        s.daeti_set_stream(stream)
        return s

    n_steps, every = 2000, 10
    g2 = inputs.lognormal_field_2d(nx, wl.h, seed_index=23) / 0.001
    tgt = solver((d_node * g2 ** 0.5)[conn].mean(axis=1), "fp64")
    data = []
    for j in range(n_steps // every):
        tgt.daeti_advance((j + 1) * every * wl.dt)
        data.append(tgt.daeti_read_v()[sensors])
    tgt.close()
    data = np.array(data)
    de = d_node[conn].mean(axis=1)
    res = {}
    for prec in ("fp64", "fp32_kahan"):
        s = solver(de, prec)
        res[prec] = s.daeti_adjoint(sensors, data, n_steps, every, 32, n_elem=len(de))
        s.close()
    (l64, g64, t64), (l32, g32, t32) = res["fp64"], res["fp32_kahan"]
    rng = np.random.default_rng(2011047 + 4)
    dirs = [rng.standard_normal(len(de)) * de for _ in range(20)]
    dd = [abs(g32 @ u - g64 @ u) / abs(g64 @ u) for u in dirs]
    return {"workload": "ms_adjoint_256x256_2000steps_32slots", "loss_rel_err": abs(l32 - l64) / abs(l64),
            "grad_d_rel_err_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
            "grad_d_rel_err_max": float(np.abs(g32 - g64).max() / np.abs(g64).max()),
            "directional_rel_err_max_20_dirs": float(max(dd)),
            "grad_tau_close_rel_err": abs(t32 - t64) / abs(t64)}


def diffusion_launch_work(l, fused, bytes_substep, bytes_sync):
    """Separate diffusion launches per Strang step and their algorithmic bytes
    per step.  Step I has l sub-steps (the last one inside the reaction launch
    when fused), step III has l, and the last of them also synchronises:
    bytes_substep (daeti_kernel_work(1)) per launch plus bytes_sync
    (daeti_kernel_work(2)) once per step."""
    launches = 2 * l - (1 if fused else 0)
    return launches, launches * bytes_substep + bytes_sync


def _reaction_roofline(solver, clocks, sub_per_step):
    """ALU roofline of the reaction kernel from the per-launch event-timed pass."""
    ms, nl = solver.daeti_get_kernel_time(0)
    bytes_launch, ops_per_sub = solver.daeti_kernel_work(0)
    avg_s = ms / max(nl, 1) / 1e3
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * mhz * 1e6 / 1e12
    achieved = ops_per_sub * sub_per_step / avg_s / 1e12
    xu_peak = SM_COUNT * XU_LANES_PER_SM * mhz * 1e6
    fused = solver.daeti_get_tuning()["fuse_diffusion"]
    label = "reaction (TP06, FP32" + (", with the fused diffusion sub-step)" if fused else ")")
    return {"bound": "alu", "kernel": label, "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": REACTION_DRAM_BYTES_PER_LAUNCH,
            "avg_launch_us": avg_s * 1e6, "ops_per_node_substep": ops_per_sub,
            "substeps_per_launch": sub_per_step,
            "peak_basis": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz (sampled), 1 op/lane/cycle",
            "xu_frac": TP06_XU_PER_SUBSTEP * sub_per_step / avg_s / xu_peak,
            "xu_peak_basis": f"{XU_LANES_PER_SM} SFU lanes per SM (ncu rates its XU pipe at 32 lanes: half this fraction)",
            "bytes_per_launch": bytes_launch,
            "bytes_frac_of_measured_hbm": bytes_launch / avg_s / 1e9 / _peaks().get("hbm_gbs", 6786.9)}


def bench_slab(args, env):
    import numpy as np

    import inputs
    from paper_2011_04747_gb300 import autotune

    binding = env.binding
    wl = inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    n_nodes, n_steps = wl.n_nodes, int(round(T_END / wl.dt))

    def make(prec):
        s = binding.solver_from_workload(wl, precision=prec, graph_steps=args.graph_steps, bucket_k=bool(args.bucket))
        s.daeti_set_stream(env.stream)
        return s

    s32 = make("fp32_kahan")
    tune = None
    if not args.no_autotune:
        # 100 ms: the stimulus, the upstroke and the start of the plateau (a
        # 20 ms window, stimulus and upstroke only, favoured shapes that lose
        # over the whole run)
        rep = autotune.autotune(s32, sim_ms=100.0, extra_key="|slab|100ms")
        tune = {k: rep[k] for k in ("cached", "candidates", "rejected", "search_s", "ms_per_sim_ms") if k in rep}
        s32.daeti_set_stream(env.stream)
    stab = s32.daeti_get_stability()
    ck = s32.daeti_save_state()
    # raw nvidia-smi samples: a temporary file unless DAETI_CLOCKS_DIR names a folder to keep them in
    clk_dir = os.environ.get("DAETI_CLOCKS_DIR") or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, f"daeti_clocks_rank{env.rank}.csv")
    os.makedirs(clk_dir, exist_ok=True)
    sampler, fh = _clock_sampler(clk_path)
    sec32 = env.timed(lambda: s32.daeti_advance(T_END), args.steps, args.warmup,
                      reset=lambda: s32.daeti_load_state(ck))
    if sampler:
        sampler.terminate()
        sampler.wait()
        fh.close()
    clocks = _clock_summary(clk_path, env.local)
    sub_total = s32.daeti_get_substeps()          # counted since the last load_state: one 500 ms run
    sub_per_step = sub_total / n_steps if sub_total else 0.0
    value = env.world * n_nodes * n_steps / sec32

    # per-kernel timing passes over the same 500 ms: mode 2 = event-record
    # nodes around every launch inside the captured graphs (the roofline's
    # kernel time), mode 1 = events around plain launches (adds the host
    # launch cost to each interval; kept for comparison)
    kt, kt_plain = {}, {}
    for mode, dst in ((2, kt), (1, kt_plain)):
        s32.daeti_load_state(ck)
        s32.daeti_set_profiling(mode)
        s32.daeti_advance(T_END)
        s32.daeti_synchronize()
        for which, name in ((0, "reaction"), (1, "diffusion")):
            ms, nl = s32.daeti_get_kernel_time(which)
            b, f = s32.daeti_kernel_work(which)
            if which == 1:
                # average over the step's launches, the synchronising one included
                per_step, b_step = diffusion_launch_work(stab["l"], s32.daeti_get_tuning()["fuse_diffusion"], b,
                                                         s32.daeti_kernel_work(2)[0])
                b = b_step / per_step
            dst[name] = {"total_ms": ms, "launches": nl, "avg_us": 1e3 * ms / max(nl, 1), "bytes_per_launch": b}
        if mode == 2:
            roof = _reaction_roofline(s32, clocks, sub_per_step)
        else:
            roof["plain_launch_frac"] = _reaction_roofline(s32, clocks, sub_per_step)["frac"]
        d = dst["diffusion"]
        d["bytes_GBs"] = d["bytes_per_launch"] / (d["avg_us"] * 1e-6) / 1e9
        s32.daeti_set_profiling(0)
    roof["event_nodes_frac"] = roof["frac"]

    # Launch durations in graph context: every 10 ms of the run (at 5, 15,
    # ..., 495 ms), 20 back-to-back launches of the reaction kernel and of the
    # synchronising diffusion sub-step, each replayed as one graph between two
    # CUDA events at the run's own state (saved before, restored after; one
    # step is re-run after a restore so that the bucketing mode is the run's)
    samples = _launch_samples(s32, ck, n_steps, wl.dt)
    roof_ops = s32.daeti_kernel_work(0)[1]      # counted operations per node sub-step
    r_ops = sum(roof_ops * sm["substeps_per_launch"] for sm in samples)
    r_s = sum(sm["reaction_us"] for sm in samples) * 1e-6
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * mhz * 1e6 / 1e12
    roof.update({"achieved": r_ops / r_s / 1e12, "frac": r_ops / r_s / 1e12 / peak,
                 "avg_launch_us": r_s * 1e6 / len(samples),
                 "substeps_per_launch": sum(sm["substeps_per_launch"] for sm in samples) / len(samples),
                 "xu_frac": TP06_XU_PER_SUBSTEP * r_ops / roof_ops / r_s / (SM_COUNT * XU_LANES_PER_SM * mhz * 1e6),
                 "timing": ("graph replays of 20 back-to-back reaction launches at the run's state every 10 ms "
                            "(50 samples), CUDA events around each replay on the launching stream; "
                            "event_nodes_frac: event-record nodes around every launch of the 500 ms run; "
                            "plain_launch_frac: events around plain launches"),
                 "samples": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in sm.items()}
                             for sm in samples[::5]]})
    bytes_launch = roof["bytes_per_launch"]
    roof["bytes_frac_of_measured_hbm"] = bytes_launch / (r_s / len(samples)) / 1e9 / _peaks().get("hbm_gbs", 6780.0)
    d_s = sum(sm["sync_diffusion_us"] for sm in samples) * 1e-6 / len(samples)
    kt["diffusion"]["graph_replay_avg_us"] = d_s * 1e6
    kt["reaction"]["graph_replay_avg_us"] = r_s * 1e6 / len(samples)

    # e2e through the C ABI with host buffers: the initial state (published
    # values at every node, n_states x n doubles) from pinned host memory
    s32.daeti_init_state(None)
    init_host = env.torch.empty((s32.n_states, n_nodes), dtype=env.torch.float64, pin_memory=True)
    init_host.numpy()[:] = s32.daeti_read_state()
    e2e = []
    for it in range(2 + max(1, args.steps // 2)):
        env.torch.cuda.synchronize(env.dev)
        t0 = time.perf_counter()
        s32.daeti_init_state(init_host.numpy())     # host -> device
        s32.daeti_advance(T_END)
        s32.daeti_read_v()                      # device -> host (waits)
        s32.daeti_read_activation()
        if it >= 2:
            e2e.append(time.perf_counter() - t0)
    e2e_val = env.world * n_nodes * n_steps / env.max_over_ranks(sum(e2e) / len(e2e))
    ns = s32.n_states
    tuning_used = s32.daeti_get_tuning()

    sec64 = err64 = None
    if not args.no_fp64:
        s64 = make("fp64")
        sec64 = env.timed(lambda: s64.daeti_advance(T_END), max(1, args.steps // 2), 1,
                          reset=lambda: s64.daeti_init_state(None))
        # V of every node every 1 ms of the whole run in both precisions
        err64 = _fp32_vs_fp64(s32, ck, s64, n_steps, wl.dt)
        s64.close()
    err_oracle = adj_err = None
    if env.rank == 0 and not args.no_cpu_baseline:
        err_oracle = _fp32_vs_oracle_reduced(binding)
    if not args.no_fp64:
        adj_err = _adjoint_precision(binding, env.stream)

    s32.close()
    # launches per step as counted by the per-kernel pass (the same sequence the graphs replay)
    launches_per_step = (kt["reaction"]["launches"] + kt["diffusion"]["launches"]) / n_steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": env.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec32 * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "tp06_slab_101x101x26_h0.02_500ms", "nodes": n_nodes, "strang_steps": n_steps,
                   "dt_ms": wl.dt, "l": stab["l"], "k_max": stab["k_max"], "dt_s_ms": stab["dt_s"],
                   "precision": "fp32_kahan", "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{env.world}", "tuning": tuning_used, "autotune": tune},
        "sim_ms_per_wall_s": env.world * T_END / sec32,
        "fp64": None if sec64 is None else {"value": env.world * n_nodes * n_steps / sec64,
                                             "ms_per_step": sec64 * 1e3, "sim_ms_per_wall_s": T_END / sec64},
        "fp32_vs_fp64": err64,
        "fp32_vs_oracle": err_oracle,
        "adjoint_fp32_vs_fp64": adj_err,
        "reaction_substeps_per_node_step": sub_per_step / n_nodes if sub_per_step else None,
        "kernels": kt, "kernels_plain_launches": kt_plain, "roofline": roof, "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": n_nodes * ns * 8,
                "d2h_bytes_per_step": 2 * n_nodes * 8},
        "gpu_launches": int(round(launches_per_step * n_steps + n_steps // max(tuning_used["graph_steps"], 1) + 2))
        * args.steps,
    }
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline_slab(wl)
    return line


def bench_simple(args, env, wl, name, precision="fp32_kahan", t_end=None, steps_sample=10):
    """node-steps/s of one single-tissue workload (not the headline)."""
    from paper_2011_04747_gb300 import autotune

    binding = env.binding
    t_end = t_end or wl.t_end
    s = binding.solver_from_workload(wl, precision=precision, graph_steps=args.graph_steps)
    s.daeti_set_stream(env.stream)
    tune = None
    if not args.no_autotune:
        rep = autotune.autotune(s, sim_ms=min(t_end, 20.0), extra_key="|" + name)
        tune = {k: rep[k] for k in ("cached", "candidates", "rejected", "search_s") if k in rep}
        s.daeti_set_stream(env.stream)
    st = s.daeti_get_stability()
    ck = s.daeti_save_state()
    sec = env.timed(lambda: s.daeti_advance(t_end), args.steps, args.warmup, reset=lambda: s.daeti_load_state(ck))
    n_steps = int(round(t_end / st["dt"]))
    s.daeti_load_state(ck)
    # kernel times inside graphs (event-record nodes around each launch)
    s.daeti_set_profiling(2)
    prof_steps = int(round(min(t_end, 100 * st["dt"]) / st["dt"]))
    s.daeti_advance(prof_steps * st["dt"])
    s.daeti_synchronize()
    ms, nl = s.daeti_get_kernel_time(1)
    b_plain, _ = s.daeti_kernel_work(1)
    b_sync, _ = s.daeti_kernel_work(2)
    tuning_used = s.daeti_get_tuning()
    fused = tuning_used["fuse_diffusion"]
    s.daeti_set_profiling(0)
    s.close()
    # separate diffusion launches per step: step I's l sub-steps (the last one
    # inside the reaction launch when fused) and step III's l, the last of
    # which synchronises; GB/s counts each launch's algorithmic bytes
    per_step, b_step = diffusion_launch_work(st["l"], fused, b_plain, b_sync)
    total_b = prof_steps * b_step
    diff = {"avg_us": 1e3 * ms / max(nl, 1), "launches": nl, "synchronising_per_step": 1,
            "plain_per_step": per_step - 1, "bytes_plain": b_plain, "bytes_synchronising": b_plain + b_sync,
            "GBs": total_b / (ms / 1e3) / 1e9 if ms else None}
    if diff["GBs"]:
        diff["frac_of_measured_hbm"] = diff["GBs"] / _peaks().get("hbm_gbs", 6786.9)
    line = {"metric": UNIT + " (" + name + ")", "value": env.world * wl.n_nodes * n_steps / sec, "unit": UNIT,
            "n_gpus": env.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": precision,
            "data": "synthetic", "config": {"workload": name, "nodes": wl.n_nodes, "strang_steps": n_steps,
                                            "l": st["l"], "dt_s_ms": st["dt_s"], "tuning": tuning_used,
                                            "autotune": tune},
            "sim_ms_per_wall_s": t_end / sec, "diffusion_launch": diff}
    if env.rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline_sample(wl, steps_sample)
    return line


def bench_tets(args, env):
    """The pathophysiological workload as stated: 2.06 M-node jittered tet slab
    (30 % fibrosis, central scar), S1-S2 cross-field protocol, 1000 ms in
    FP32 with compensated V.  Beside the timed runs: the number of nodes above
    -40 mV every 50 ms (is activity still present at 1000 ms?) and the FP32
    run against the FP64 path in lockstep, V of every node every 1 ms."""
    import numpy as np

    import inputs

    wl = inputs.tet_slab_3d(t_end=1000.0)
    line = bench_simple(args, env, wl, "tp06_tet_slab_201x201x51_1000ms", t_end=1000.0, steps_sample=2)
    binding = env.binding
    s32 = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=args.graph_steps)
    s64 = binding.solver_from_workload(wl, precision="fp64", graph_steps=args.graph_steps)
    for s in (s32, s64):
        s.daeti_set_stream(env.stream)
    active, worst, worst_t, first_2mv, worst_50 = [], 0.0, 0.0, None, 0.0
    for j in range(1, 1001):
        s32.daeti_advance(float(j))
        s64.daeti_advance(float(j))
        v32, v64 = s32.daeti_read_v(), s64.daeti_read_v()
        dv = np.abs(v32 - v64)
        d = float(np.max(dv))
        worst_50 = max(worst_50, d)
        if d > worst:
            worst, worst_t = d, float(j)
        if first_2mv is None and d > 2.0:
            first_2mv = float(j)
        if j % 50 == 0:
            active.append({"t_ms": j, "nodes_above_-40mV": int((v32 > -40.0).sum()),
                           "max_abs_dv_mv_last_50ms": round(worst_50, 4),
                           "nodes_dv_above_2mV": int((dv > 2.0).sum())})
            worst_50 = 0.0
    a32, a64 = s32.daeti_read_activation(), s64.daeti_read_activation()
    s32.close()
    s64.close()
    both = (a32 >= 0) & (a64 >= 0)
    line["s2_time_ms"] = float(wl.stimuli[1].t_start)
    line["activity"] = active
    line["activity_at_1000ms"] = active[-1]["nodes_above_-40mV"]
    line["fp32_vs_fp64"] = {"max_abs_dv_mv_every_1ms": worst, "at_ms": worst_t,
                            "first_ms_above_2mV": first_2mv,
                            "max_abs_dact_ms": float(np.abs(a32[both] - a64[both]).max()) if both.any() else None,
                            "same_activated_set": bool(np.array_equal(a32 >= 0, a64 >= 0))}
    return line


def bench_batch(args, env):
    """512 uneven tissues in one batched launch sequence vs the same tissues run one by one."""
    import inputs

    binding = env.binding
    wls = inputs.batch_tissues()
    t_end = 300.0
    n_nodes = sum(w.n_nodes for w in wls)
    n_steps = int(round((t_end - 1.0) / 0.1))    # timed: 1 ms .. 300 ms
    secs = {}
    for bucket in (1, 0):
        # bucket_k = 1: the TP06 tissues' nodes grouped by k (warp-uniform sub-step counts)
        batch = binding.Batch(precision="fp32_kahan", graph_steps=args.graph_steps, stream=env.stream,
                              bucket_k=bool(bucket))
        for w in wls:
            d = binding.describe_workload(w)
            batch.daeti_batch_add(d)
            d.close()
        batch.daeti_batch_prepare()
        batch.daeti_batch_advance(1.0)        # graphs captured, caches warm; 1 ms of the run
        secs[bucket] = env.timed(lambda: batch.daeti_batch_advance(t_end), 1, 0)
        batch.close()
    sec_b = min(secs.values())      # the faster of the two (an autotuner's pick)
    best_bucket = 1 if secs[1] <= secs[0] else 0
    solvers = [binding.solver_from_workload(w, precision="fp32_kahan", graph_steps=args.graph_steps) for w in wls]
    for s in solvers:
        s.daeti_set_stream(env.stream)
        s.daeti_advance(1.0)                  # as the batch: graphs captured, first 1 ms untimed

    def seq():
        for s in solvers:
            s.daeti_advance(t_end)

    sec_s = env.timed(seq, 1, 0)
    for s in solvers:
        s.close()
    return {"metric": "aggregate node-steps/s, 512 batched tissues (MS/TP06 mixed, 32^2..256^2, 300 ms)",
            "value": env.world * n_nodes * n_steps / sec_b, "unit": UNIT, "n_gpus": env.world,
            "steps": 1, "warmup": 0, "ms_per_step": sec_b * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_512_tissues_300ms", "nodes": n_nodes, "strang_steps": n_steps,
                       "timed": "1 ms .. 300 ms of each run (the first 1 ms captures the graphs)"},
            "sequential": {"value": n_nodes * n_steps / sec_s, "ms": sec_s * 1e3},
            "k_lists_tp06": bool(best_bucket),
            "with_k_lists": {"value": env.world * n_nodes * n_steps / secs[1], "ms": secs[1] * 1e3},
            "without_k_lists": {"value": env.world * n_nodes * n_steps / secs[0], "ms": secs[0] * 1e3},
            "batched_over_sequential": sec_s / sec_b}


def bench_adjoint(args, env):
    """Gradient evaluations per second and adjoint/forward time ratio, 256^2 MS, 2000 steps, 32 slots."""
    import numpy as np

    import inputs

    binding = env.binding
    wl, d_node, sensors, _ = inputs.ms_adjoint_2d()
    nx = wl.n[0]
    ey, ex = np.meshgrid(np.arange(nx - 1), np.arange(nx - 1), indexing="ij")
    base = (ex + nx * ey).ravel()
    conn = base[:, None] + np.array([0, 1, nx, nx + 1])[None, :]
    de = d_node[conn].mean(axis=1)
    wl.d_long, wl.d_trans, wl.fibre = de, de, None
    s = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=args.graph_steps)
    s.daeti_set_stream(env.stream)
    data = np.zeros((200, len(sensors)))
    t_fwd = env.timed(lambda: s.daeti_adjoint(sensors, data, 2000, 10, 32, flags=4), args.steps, 1)
    t_adj = env.timed(lambda: s.daeti_adjoint(sensors, data, 2000, 10, 32, n_elem=len(de)), args.steps, 1)
    t_plain = env.timed(lambda: s.daeti_advance(s.time + 200.0), args.steps, 1)
    s.close()
    return {"metric": "gradient evaluations/s (256x256 MS, 2000 steps, 32 slots, FP32)",
            "value": 1.0 / t_adj, "unit": "gradients/s", "n_gpus": env.world, "steps": args.steps, "warmup": 1,
            "ms_per_step": t_adj * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": {"workload": "ms_adjoint_256x256_2000steps"},
            "adjoint_over_forward": t_adj / t_fwd, "adjoint_over_plain_advance": t_adj / t_plain,
            "forward_ms": t_fwd * 1e3, "plain_advance_ms": t_plain * 1e3}


def bench_accuracy(args, env):
    """Section 3.1's comparison on the 2D sheet 501 x 501 (TP06 standing in for
    O'Hara-Rudy), FP32 + Kahan: OST (dt 0.01 ms), OSTAR (dt_s-limited step) and
    DAETI (dt 0.1 ms), 500 ms each; errors against OST as in Section 3.3."""
    import inputs

    wl = inputs.aniso_sheet_2d()
    k, w = max(1, args.steps // 2), max(1, args.warmup // 2)

    def timer(s):
        return env.timed(lambda: s.daeti_advance(wl.t_end), k, w, reset=lambda: s.daeti_init_state(None))

    common = dict(precision="fp32_kahan", graph_steps=args.graph_steps)
    runs = [("ost", dict(scheme="ost", dt=0.01, **common)), ("ostar", dict(scheme="ostar", **common)),
            ("daeti", dict(scheme="daeti", **common))]
    from paper_2011_04747_gb300.compare import scheme_comparison

    per = scheme_comparison(env.binding, wl, runs, stream=env.stream, timer=timer)
    per["daeti"]["speedup_vs_ostar"] = per["ostar"]["wall_s"] / per["daeti"]["wall_s"]
    return {
        "metric": "DAETI speed-up over OST, 2D sheet 501x501 TP06 500 ms (Section 3.1 comparison)",
        "value": per["daeti"]["speedup_vs_ost"], "unit": "x", "n_gpus": env.world, "steps": k, "warmup": w,
        "ms_per_step": per["daeti"]["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32_kahan", "data": "synthetic",
        "config": {"workload": "tp06_sheet_501x501_h0.01_500ms_ost_ostar_daeti", "nodes": wl.n_nodes,
                   "probes": "centre + 11x11 grid, V every 0.1 ms", "cv_line": "centre row, x in [1, 4] cm"},
        "schemes": per,
    }


def run_ours(args):
    import inputs

    env = Env(args)
    wk = args.workload
    if wk == "slab":
        line = bench_slab(args, env)
    elif wk == "slab_l":
        line = bench_simple(args, env, inputs.tp06_slab_3d(401, 401, 26, t_end=50.0), "tp06_slab_401x401x26_50ms",
                            t_end=50.0, steps_sample=2)
    elif wk == "square":
        line = bench_simple(args, env, inputs.ms_square_2d(), "ms_square_41x41_100ms", precision="fp64",
                            steps_sample=1000)
    elif wk == "sheet":
        line = bench_simple(args, env, inputs.aniso_sheet_2d(t_end=50.0), "tp06_sheet_501x501_h0.01_50ms",
                            t_end=50.0, steps_sample=5)
    elif wk == "tets":
        line = bench_tets(args, env)
    elif wk == "batch":
        line = bench_batch(args, env)
    elif wk == "accuracy":
        line = bench_accuracy(args, env)
    else:
        line = bench_adjoint(args, env)
    if env.rank == 0:
        print(json.dumps(line), flush=True)
    if env.world > 1:
        env.dist.barrier()
        env.dist.destroy_process_group()


def profile_run(args):
    """A short plain run of the slab workload (101 x 101 x 26, or 401 x 401 x 26
    with --workload slab_l) for external profilers."""
    import inputs
    from paper_2011_04747_gb300 import binding, build as _build

    if not os.path.exists(binding.LIB_PATH):
        _build.build()
    wl = inputs.tp06_slab_3d(401, 401, 26, t_end=T_END) if args.workload == "slab_l" else \
        inputs.tp06_slab_3d(**SLAB, t_end=T_END)
    s = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=args.graph_steps,
                                     bucket_k=bool(args.bucket))
    if args.diff_block >= 0:
        s.daeti_set_tuning(diff_block=args.diff_block)
    if args.fuse_diffusion >= 0:
        s.daeti_set_tuning(fuse_diffusion=args.fuse_diffusion)
    if args.profile_from > 0:
        s.daeti_advance(args.profile_from)
    s.daeti_advance(args.profile_from + args.profile_run)
    s.daeti_synchronize()
    s.close()
    print(f"profile run: {args.profile_run} ms simulated after {args.profile_from} ms")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="slab",
                    choices=["slab", "slab_l", "square", "sheet", "tets", "batch", "adjoint", "accuracy"])
    ap.add_argument("--graph-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--bucket", type=int, default=1, help="group nodes by k before step A (1) or not (0)")
    ap.add_argument("--profile-run", type=float, default=0.0,
                    help="only simulate this many ms once on the slab (FP32), for profilers; no timing")
    ap.add_argument("--diff-block", type=int, default=-1,
                    help="with --profile-run: diffusion launch shape (0 = 2D tiles / 3D runs of nodes along y, "
                         "256 = one thread per node; default: the library's)")
    ap.add_argument("--fuse-diffusion", type=int, default=-1,
                    help="with --profile-run: 1 = last step-I diffusion sub-step inside the reaction launch, "
                         "0 = its own launch (default: the library's)")
    ap.add_argument("--profile-from", type=float, default=0.0,
                    help="with --profile-run: first advance to this time (ms), e.g. into the plateau "
                         "(60) or the resting phase (150)")
    args = ap.parse_args()
    if args.profile_run > 0:
        profile_run(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
