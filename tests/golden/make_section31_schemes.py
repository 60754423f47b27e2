"""Writes section31_schemes_oracle.json: the oracle's Section 3.1 scheme
comparison (OST, OSTAR, DAETI) on a 0.6 x 0.6 cm sheet with the spacing and
conductivities of Section 3.1 (h = 100 um, d0 = 0.0017 cm^2/ms, rho = 0.25,
fibres along X; TP06 epicardial in place of O'Hara-Rudy; 1 ms stimulus on
the X = 0 column), 400 ms, V sampled every 0.1 ms at a 6 x 6 probe grid and
the centre.  Measures (oracle/metrics.py): conduction velocity along the
centre row (middle 60 %), activation times (LAT) at the probes and along the
centre row, APD90 at the probes, and against OST the Eq. 4 errors of LAT
(all nodes) and APD90 (probes).

Only the oracle runs here:  python tests/golden/make_section31_schemes.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs as I  # noqa: E402
from oracle import metrics, scheme  # noqa: E402

N, LENGTH, T_END = 61, 0.6, 400.0
SCHEMES = (("ost", 0.01), ("ostar", None), ("daeti", None))


def probes_of(n):
    sel = np.unique(np.round(np.linspace(0.05, 0.95, 6) * (n - 1)).astype(np.int64))
    mid = n // 2
    return np.concatenate([[mid * n + mid], (sel[:, None] * n + sel[None, :]).ravel()])


def run():
    wl = I.aniso_sheet_2d(n=N, length=LENGTH, t_end=T_END)
    probes = probes_of(N)
    mid = N // 2
    row = mid * N + np.arange(N)
    xs = np.arange(N) * wl.h
    cv_sel = (xs >= 0.2 * xs[-1]) & (xs <= 0.8 * xs[-1])
    t_s = np.arange(1, int(round(T_END / 0.1)) + 1) * 0.1
    out = {"workload": f"tp06 sheet {N}x{N}, h = {wl.h} cm, {T_END} ms", "probes": probes.tolist(),
           "sample_ms": 0.1, "schemes": {}}
    acts, apds = {}, {}
    for name, dt in SCHEMES:
        sim = scheme.simulation_from_workload(wl, scheme=name, dt=dt)
        per_sample = int(round(0.1 / sim.dt))
        assert abs(per_sample * sim.dt - 0.1) < 1e-12
        tr = np.empty((t_s.size, probes.size))
        for j in range(t_s.size):
            sim.run(per_sample)
            tr[j] = sim.S[0][probes]
        act = sim.act.copy()
        apd = np.array([metrics.apd90(t_s, tr[:, q]) for q in range(probes.size)])
        acts[name], apds[name] = act, apd
        out["schemes"][name] = {
            "dt_ms": sim.dt, "l": sim.l, "k_max": sim.k_max,
            "all_activated": bool((act >= 0).all()),
            "cv_cm_per_ms": metrics.conduction_velocity(xs[cv_sel], act[row][cv_sel]),
            "lat_probes_ms": act[probes].tolist(), "lat_row_ms": act[row].tolist(),
            "lat_range_ms": float(act.max() - act.min()),
            "apd90_probes_ms": apd.tolist(),
        }
        print(name, "done", flush=True)
    for name in ("ostar", "daeti"):
        d = out["schemes"][name]
        d["e_lat_vs_ost"] = metrics.nrmse(acts[name], acts["ost"])
        d["e_apd_vs_ost"] = metrics.nrmse(apds[name], apds["ost"])
        d["max_abs_dapd90_vs_ost_ms"] = float(np.abs(apds[name] - apds["ost"]).max())
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "section31_schemes_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    run()
