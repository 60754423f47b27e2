"""Autotuner for libdaeti launch shapes.

For a prepared ``Solver`` it times a short stretch of the simulation under
each candidate tuning (reaction block size and register cap, the diffusion
sub-step fused into the reaction launch or not, k bucketing, diffusion block
size, steps per CUDA graph, programmatic dependent launch), keeps only candidates whose final state is
bit-identical to the reference run (the shapes must not change results), and
applies the fastest.  Choices are cached as JSON keyed by the problem's
signature (mesh, model, precision, l, k_max, GPU name) so a later run of the
same configuration skips the search.
"""
from __future__ import annotations

import itertools
import json
import os
import time
from typing import Dict, Iterable, List, Optional

import numpy as np

DEFAULT_SPACE = {
    "react_block": (64, 128),
    "react_min_blocks": (6, 8, 10),
    "fuse_diffusion": (1, 0),
    "bucket_k": (1, 0),
    "diff_block": (0, 256),
    "graph_steps": (20, 100),
    "pdl": (1, 0),
}


def default_cache_path() -> str:
    return os.environ.get("DAETI_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "daeti_tuning.json"))


def signature(solver, extra: str = "") -> str:
    import torch

    st = solver.daeti_get_stability()
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    return (f"n={solver.n_nodes}|states={solver.n_states}|prec={solver.precision}|l={st['l']}|"
            f"kmax={st['k_max']}|dt={st['dt']:.6g}|gpu={gpu}{extra}")


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, entry: dict) -> None:
    data = load_cache(path)
    data[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(space: Optional[Dict[str, Iterable]] = None) -> List[dict]:
    space = dict(DEFAULT_SPACE if space is None else space)
    keys = sorted(space)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(space[k] for k in keys))]


def _time_advance(solver, t_start: float, sim_ms: float, reps: int) -> float:
    import torch

    stream = torch.cuda.current_stream()
    solver.daeti_set_stream(stream)
    best = float("inf")
    ck = solver.daeti_save_state()
    for _ in range(reps):
        solver.daeti_load_state(ck)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.daeti_advance(t_start + sim_ms)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def autotune(solver, sim_ms: float = 20.0, reps: int = 2, space=None, cache_path: Optional[str] = None,
             use_cache: bool = True, extra_key: str = "") -> dict:
    """Pick and apply the fastest result-preserving tuning; returns a report."""
    path = cache_path or default_cache_path()
    key = signature(solver, extra_key)
    if use_cache:
        hit = load_cache(path).get(key)
        if hit:
            solver.daeti_set_tuning(**hit["tuning"])
            return {"key": key, "cached": True, **hit}
    t0 = solver.time
    start = solver.daeti_save_state()
    base_tuning = solver.daeti_get_tuning()
    # reference result with the current tuning
    solver.daeti_advance(t0 + sim_ms)
    ref = solver.daeti_read_state()
    results = []
    t_search = time.perf_counter()
    for cand in candidates(space):
        solver.daeti_load_state(start)
        solver.daeti_set_tuning(**{**base_tuning, **cand})
        ms = _time_advance(solver, t0, sim_ms, reps)
        ok = np.array_equal(solver.daeti_read_state(), ref)
        results.append({"tuning": cand, "ms": ms, "identical": ok})
    good = [r for r in results if r["identical"]]
    best = min(good, key=lambda r: r["ms"]) if good else {"tuning": base_tuning, "ms": float("nan")}
    solver.daeti_load_state(start)
    solver.daeti_set_tuning(**{**base_tuning, **best["tuning"]})
    entry = {"tuning": solver.daeti_get_tuning(), "ms_per_sim_ms": best["ms"] / sim_ms,
             "candidates": len(results), "rejected": len(results) - len(good),
             "search_s": time.perf_counter() - t_search}
    store_cache(path, key, entry)
    return {"key": key, "cached": False, **entry, "all": results}
