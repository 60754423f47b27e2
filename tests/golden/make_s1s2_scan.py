"""Oracle scan for the S2 time of the S1-S2 cross-field protocol on the
fibrotic tet slab (reading R-S1S2: the S2 time on a 10 ms grid for which
activity persists at t = 1000 ms).

The oracle runs a reduced slab with the full in-plane mesh (201 x 201 x 3
nodes, h = 0.02 cm: 4 x 4 x 0.04 cm, the same jitter, 30 % fibrosis and
central scar, the same stimulus regions) for 1000 ms per S2 time and counts
the nodes above -40 mV every 10 ms.  Each run takes about 50 minutes of one
core; the runs are independent:

    python tests/golden/make_s1s2_scan.py run 200 210 ... 350   # one process per value
    python tests/golden/make_s1s2_scan.py collect               # writes s1s2_scan_oracle.json

Only the oracle runs here.
"""
import glob
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
PARTS = os.environ.get("S1S2_SCAN_DIR", os.path.join(ROOT, "_work"))


def run(s2):
    import inputs as I
    from oracle import scheme

    wl = I.tet_slab_3d(201, 201, 3, h=0.02, s2_time=float(s2), t_end=1000.0)
    sim = scheme.simulation_from_workload(wl)
    act = []
    t0 = time.time()
    for j in range(100):                    # every 10 ms
        sim.run(100)
        act.append(int((sim.S[0] > -40.0).sum()))
        if j % 10 == 9:
            with open(os.path.join(PARTS, f"s2scan_{s2}.json"), "w") as f:
                json.dump({"s2": s2, "active_every_10ms": act, "nodes": wl.n_nodes, "wall_s": time.time() - t0}, f)
    return s2, act


def collect():
    runs = {}
    for f in glob.glob(os.path.join(PARTS, "s2scan_*.json")):
        d = json.load(open(f))
        if len(d["active_every_10ms"]) == 100 and d["s2"] % 10 == 0:
            runs[d["s2"]] = d["active_every_10ms"]
    persists = sorted(s for s, a in runs.items() if a[-1] > 0)
    out = {"workload": "tet slab 201 x 201 x 3, h = 0.02 cm, 30 % fibrosis, scar r = 0.5 cm, TP06 endo, 1000 ms",
           "count": "nodes above -40 mV every 10 ms (10 .. 1000 ms)",
           "runs": {str(s): runs[s] for s in sorted(runs)},
           "s2_with_activity_at_1000ms": persists}
    path = os.path.join(HERE, "s1s2_scan_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, "persisting:", persists)


if __name__ == "__main__":
    if sys.argv[1] == "run":
        with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as p:
            for s2, act in p.imap_unordered(run, [int(v) for v in sys.argv[2:]]):
                print(s2, act[-10:], flush=True)
    else:
        collect()
