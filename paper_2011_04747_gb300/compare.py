"""Comparison of integration schemes on one workload (Section 3).

Runs OST, OSTAR and DAETI (or any list of solver options) through the C ABI
and measures what Sections 3.1 and 3.3 compare: conduction velocity, APD90,
activation times, aligned action potentials and wall time, with Eq. 4 errors
against the first run.
"""
from __future__ import annotations

import numpy as np

from . import metrics


def scheme_comparison(binding, wl, runs, stream=None, timer=None, probes_per_side=11):
    """Section 3's comparison of OST, OSTAR and DAETI on a square sheet:
    each run (name, solver options) simulates wl.t_end ms; V is sampled every
    0.1 ms at a probes_per_side^2 grid of nodes (the centre among them).
    Returns per-scheme results: wall time (timer(solver) if given), CV along
    the centre row (middle 60 %), activation time and APD90 at the centre,
    and against the first run (OST): Eq. 4 nRMSE of activation times (all
    nodes) and of APD90 (probes), the largest APD90 difference over the
    probes, aligned max |dV| at the centre over the
    whole AP and from 5 ms after activation on, and the speed-up."""
    n, h, t_end = wl.n[0], wl.h, wl.t_end
    mid = n // 2
    sel = np.unique(np.round(np.linspace(0.05, 0.95, probes_per_side) * (n - 1)).astype(np.int64))
    probes = (sel[:, None] * n + sel[None, :]).ravel()
    probes = np.concatenate([[mid * n + mid], probes])
    row = mid * n + np.arange(n, dtype=np.int64)
    xs = np.arange(n) * h
    cv_sel = (xs >= 0.2 * xs[-1]) & (xs <= 0.8 * xs[-1])
    t_s = np.arange(1, int(round(t_end / 0.1)) + 1) * 0.1
    raw = {}
    for name, opts in runs:
        s = binding.solver_from_workload(wl, **opts)
        if stream is not None:
            s.daeti_set_stream(stream)
        st = s.daeti_get_stability()
        sec = timer(s) if timer else None
        s.daeti_init_state(None)
        tr = np.empty((t_s.size, probes.size))
        for j, t in enumerate(t_s):
            s.daeti_advance(float(np.round(t, 6)))
            tr[j] = s.daeti_read_v_nodes(probes)
        act = s.daeti_read_activation()
        s.close()
        apd = np.array([metrics.apd90(t_s, tr[:, q]) for q in range(probes.size)])
        raw[name] = (sec, st, act, tr, apd)
    per = {}
    ref_name = runs[0][0]
    r_sec, _, r_act, r_tr, r_apd = raw[ref_name]
    for name, (sec, st, act, tr, apd) in raw.items():
        d = {"wall_s": sec, "dt_ms": st["dt"], "l": st["l"], "k_max": st["k_max"],
             "cv_cm_per_ms": metrics.conduction_velocity(xs[cv_sel], act[row][cv_sel]),
             "lat_centre_ms": float(act[probes[0]]), "apd90_centre_ms": float(apd[0]),
             "all_activated": bool((act >= 0).all())}
        if name != ref_name:
            both = (act >= 0) & (r_act >= 0)
            ok = np.isfinite(apd) & np.isfinite(r_apd)
            d["e_lat"] = metrics.nrmse(act[both], r_act[both])
            d["e_apd_probes"] = metrics.nrmse(apd[ok], r_apd[ok])
            d["max_abs_dapd90_ms"] = float(np.abs(apd[ok] - r_apd[ok]).max())
            d["aligned_max_dv_mv"] = metrics.aligned_max_dv(t_s, tr[:, 0], r_tr[:, 0], act[probes[0]],
                                                            r_act[probes[0]])
            d["aligned_max_dv_mv_from_5ms"] = metrics.aligned_max_dv(t_s, tr[:, 0], r_tr[:, 0], act[probes[0]],
                                                                     r_act[probes[0]], after=5.0)
            if sec and r_sec:
                d["speedup_vs_" + ref_name] = r_sec / sec
        per[name] = d
    return per
