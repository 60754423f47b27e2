"""Section 3.1's scheme comparison on the GPU against the oracle's own run
of it (tests/golden/section31_schemes_oracle.json, written by
make_section31_schemes.py from oracle/ only): OST (dt 0.01 ms), OSTAR (the
dt_s-limited step) and DAETI (dt 0.1 ms, l = 3, k_max = 10) on a 0.6 x 0.6
cm sheet with the Section 3.1 spacing and conductivities, 400 ms, FP64.

For each scheme the GPU reproduces the oracle's measures, so the scheme
differences it reports (CV, APD90, e_LAT and e_APD against OST, Eq. 4) are
the method's and not a GPU artefact:

* schedule: dt, l and k_max identical;
* activation times at the probes and along the centre row within the FP64
  bar (0.1 ms); eps = the largest such difference;
* CV along the centre row within 4 eps / (activation-time span of the fit)
  relative (a least-squares slope moves by at most that when its times move
  by eps);
* APD90 at the probes (the oracle's definition applied to the GPU's traces)
  within 0.1 ms (one sample);
* e_LAT and e_APD against OST within the change that such LAT and APD90
  differences can make in Eq. 4 (2 x 2 eps / LAT range, 2 x 0.1 ms / APD90
  range, plus the oracle's own value times 1e-6).
"""
import json
import os

import numpy as np
import pytest

import inputs as I
from oracle import metrics as om
from parity_util import ensure_lib, gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "section31_schemes_oracle.json")


def _run(binding, wl, name, probes):
    opts = dict(scheme=name, precision="fp64")
    if name == "ost":
        opts["dt"] = 0.01
    s = binding.solver_from_workload(wl, **opts)
    st = s.daeti_get_stability()
    t_s = np.arange(1, int(round(wl.t_end / 0.1)) + 1) * 0.1
    tr = np.empty((t_s.size, probes.size))
    for j, t in enumerate(t_s):
        s.daeti_advance(float(np.round(t, 6)))
        tr[j] = s.daeti_read_v_nodes(probes)
    act = s.daeti_read_activation()
    s.close()
    return st, t_s, tr, act


def test_scheme_comparison_matches_the_oracle():
    binding = ensure_lib()
    g = json.load(open(GOLDEN))
    wl = I.aniso_sheet_2d(n=61, length=0.6, t_end=400.0)
    n = wl.n[0]
    probes = np.array(g["probes"], dtype=np.int64)
    row = (n // 2) * n + np.arange(n)
    xs = np.arange(n) * wl.h
    cv_sel = (xs >= 0.2 * xs[-1]) & (xs <= 0.8 * xs[-1])
    acts, apds, eps = {}, {}, {}
    for name, o in g["schemes"].items():
        st, t_s, tr, act = _run(binding, wl, name, probes)
        assert abs(st["dt"] - o["dt_ms"]) <= 1e-15 and st["l"] == o["l"] and st["k_max"] == o["k_max"], name
        assert bool((act >= 0).all()) == o["all_activated"]
        d_lat = max(np.abs(act[probes] - o["lat_probes_ms"]).max(), np.abs(act[row] - o["lat_row_ms"]).max())
        assert d_lat <= 0.1, (name, d_lat)
        eps[name] = float(d_lat)
        span = float(np.ptp(np.array(o["lat_row_ms"])[cv_sel]))
        cv = om.conduction_velocity(xs[cv_sel], act[row][cv_sel])
        assert abs(cv / o["cv_cm_per_ms"] - 1.0) <= 4.0 * d_lat / span + 1e-12, (name, cv, o["cv_cm_per_ms"])
        apd = np.array([om.apd90(t_s, tr[:, q]) for q in range(probes.size)])
        assert np.abs(apd - o["apd90_probes_ms"]).max() <= 0.1, name
        acts[name], apds[name] = act, apd
    for name in ("ostar", "daeti"):
        o = g["schemes"][name]
        e_lat = om.nrmse(acts[name], acts["ost"])
        tol = 2.0 * 2.0 * max(eps[name], eps["ost"]) / g["schemes"]["ost"]["lat_range_ms"] + 1e-6 * o["e_lat_vs_ost"]
        assert abs(e_lat - o["e_lat_vs_ost"]) <= tol, (name, e_lat, o["e_lat_vs_ost"])
        e_apd = om.nrmse(apds[name], apds["ost"])
        apd_range = float(np.ptp(np.array(g["schemes"]["ost"]["apd90_probes_ms"])))
        assert abs(e_apd - o["e_apd_vs_ost"]) <= 2.0 * 0.1 / apd_range + 1e-6 * o["e_apd_vs_ost"], name
