"""Stability data of daeti_prepare against the oracle (Eq. 3 and the
explicit-diffusion bound dt_ad * lambda_max < 2 of Section 2).

* lambda_max of M_L^-1 K from the GPU's FP64 Lanczos iteration equals the
  oracle's (dense eigenvalues up to 400 nodes, ARPACK above; itself pinned to
  dense eigenvalues in test_oracle_scheme) within 1e-9 relative, on a 2D
  isotropic square, the anisotropic sheet with l = 3, a layered 3D slab, a
  grid with D varying within layers (per-node rows) and a tetrahedral mesh.
* Gershgorin's dt_s bounds it: dt_s * lambda_max <= 0.9.
* A conductivity update that breaks the prepared schedule returns
  DAETI_EUNSTABLE and leaves the context as it was (stability data, operator
  and results unchanged).
"""
import numpy as np
import pytest

import inputs as I
from oracle import fem, scheme
from parity_util import ensure_lib, gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _heterogeneous(wl, seed=11):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.4, 1.6, wl.n_elems)
    wl.d_long = wl.d_long * f
    wl.d_trans = wl.d_trans * f
    return wl


CASES = {
    "square41": lambda: I.ms_square_2d(),
    "sheet37_l3": lambda: I.aniso_sheet_2d(n=37, length=0.36, model="tp06", amp=60.0),
    "slab21x17x6": lambda: I.tp06_slab_3d(21, 17, 6),
    "slab_per_node_rows": lambda: _heterogeneous(I.tp06_slab_3d(13, 11, 6)),
    "tets": lambda: I.tet_slab_3d(13, 11, 6, h=0.02, fibrosis=0.3, scar_radius=0.05, s2_time=15.0),
    "tets_larger": lambda: I.tet_slab_3d(31, 27, 9, h=0.02, fibrosis=0.3, scar_radius=0.15, s2_time=15.0),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_lambda_max_matches_oracle(case, precision):
    binding = ensure_lib()
    wl = CASES[case]()
    K, m = fem.assemble_workload(wl)
    lam_ref = scheme.lambda_max(K, m)
    dts_ref = scheme.gershgorin_dt(K, m)
    s = binding.solver_from_workload(wl, precision=precision)
    st = s.daeti_get_stability()
    s.close()
    assert abs(st["lambda_max"] - lam_ref) <= 1e-9 * lam_ref, (st["lambda_max"], lam_ref)
    assert abs(st["dt_s"] - dts_ref) <= 1e-12 * dts_ref
    assert st["dt_s"] * st["lambda_max"] <= 0.9 * (1 + 1e-12)
    # the prepared schedule is stable: dt_ad = dt / (2 l)
    assert st["dt"] / (2 * st["l"]) * st["lambda_max"] < 2.0
    if wl.tets is None and case != "slab_per_node_rows":
        dts, lam = binding.daeti_grid_stability_noalloc(wl.dim, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
        assert abs(lam - lam_ref) <= 1e-9 * lam_ref
        assert abs(dts - dts_ref) <= 1e-12 * dts_ref


def test_unstable_update_is_rejected_and_leaves_the_context_unchanged():
    binding = ensure_lib()
    wl = I.tp06_slab_3d(13, 11, 6, t_end=5.0)
    s = binding.solver_from_workload(wl, precision="fp64")
    before = s.daeti_get_stability()
    assert before["l"] == 1
    # l = 1 keeps dt_ad = 0.05 ms: D x 4 takes lambda_max past 2 / dt_ad = 40 /ms
    K, m = fem.assemble_workload(I.Workload(**{**wl.__dict__, "d_long": wl.d_long * 4, "d_trans": wl.d_trans * 4}))
    assert 0.05 * scheme.lambda_max(K, m) >= 2.0
    with pytest.raises(binding.DaetiError) as e:
        s.daeti_update_conductivity(wl.d_long * 4, wl.d_trans * 4, wl.fibre)
    assert e.value.code == binding.EUNSTABLE
    assert s.daeti_get_stability() == before
    s.daeti_advance(wl.t_end)
    v_after = s.daeti_read_state()
    s.close()
    fresh = binding.solver_from_workload(wl, precision="fp64")
    fresh.daeti_advance(wl.t_end)
    v_fresh = fresh.daeti_read_state()
    fresh.close()
    assert np.array_equal(v_after, v_fresh)
    # a stable update (D x 1.5) is accepted and changes lambda_max by the factor
    s = binding.solver_from_workload(wl, precision="fp64")
    s.daeti_update_conductivity(wl.d_long * 1.5, wl.d_trans * 1.5, wl.fibre)
    after = s.daeti_get_stability()
    s.close()
    assert abs(after["lambda_max"] - 1.5 * before["lambda_max"]) <= 1e-9 * after["lambda_max"]
    assert after["l"] == before["l"]
