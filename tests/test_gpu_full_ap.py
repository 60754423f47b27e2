"""GPU vs oracle over whole action potentials: upstroke, plateau,
repolarisation and return to rest, element by element.

The headline slab spends most of its 500 ms in the plateau and repolarisation
phases; these cases cover them in tissue in both precisions (FP64 max|dV| <=
0.5 mV and activation <= 0.1 ms; FP32 with compensated V <= 2 mV and
<= 0.5 ms), with V snapshots every 1 ms:

* a TP06 slab of 25 x 23 x 7 nodes (ragged in x and y, 27-point stencil),
  500 ms: the corner stimulus, the wave crossing the slab, every node's
  repolarisation (TP06 APD90 ~ 290 ms) and the resting phase after it;
* a jittered tetrahedral mesh with fibrosis, a scar and an S2 stimulus
  (SELL-32 rows), 400 ms;
* the transmural slab (endocardial, mid-myocardial and epicardial layers,
  per-node cell types), 400 ms.

Each oracle run is shared by the two precisions.
"""
import functools

import numpy as np
import pytest

import inputs as I
from parity_util import act_error, gpu_available, run_gpu, run_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = {"fp64": (0.5, 0.1), "fp32_kahan": (2.0, 0.5)}
EVERY = 10            # snapshot every 10 steps = 1 ms

WORKLOADS = {
    "slab25x23x7_500ms": (lambda: I.tp06_slab_3d(25, 23, 7, t_end=500.0), 5000),
    "tets_400ms": (lambda: I.tet_slab_3d(13, 11, 6, h=0.02, fibrosis=0.3, scar_radius=0.05, s2_time=15.0,
                                         t_end=400.0), 4000),
    "transmural_400ms": (lambda: I.tp06_slab_3d(13, 11, 9, transmural=True, t_end=400.0), 4000),
}


@functools.lru_cache(maxsize=None)
def _oracle(name):
    make, steps = WORKLOADS[name]
    wl = make()
    o, oa, sim = run_oracle(wl, steps, EVERY)
    return o, oa, sim.l, sim.k_max


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_whole_action_potential(name, precision):
    make, steps = WORKLOADS[name]
    wl = make()
    o, oa, l, kmax = _oracle(name)
    g, ga, stab, _ = run_gpu(wl, steps, EVERY, precision=precision)
    assert stab["l"] == l and stab["k_max"] == kmax
    # the run covers a whole AP: nodes activated, and back near rest at the end
    assert (oa >= 0).mean() > 0.9
    assert o[-1].max() < -70.0, "the tissue has not repolarised by the end of the run"
    # ... through the plateau: most nodes above -20 mV at t = 150 ms
    assert (o[149] > -20.0).mean() > 0.8
    tv, ta = TOL[precision]
    dv_t = np.max(np.abs(g - o), axis=1)              # max over nodes, per snapshot
    da, same, nboth = act_error(ga, oa)
    assert same, "activated node sets differ"
    assert float(dv_t.max()) <= tv, f"max|dV| = {dv_t.max():.4g} mV at t = {(np.argmax(dv_t) + 1) * EVERY * wl.dt} ms"
    assert da <= ta, f"max|d act| = {da:.4g} ms"
