"""The allocation-free stable-step entry point against the context path.

daeti_grid_stability_noalloc serves callers that cannot call cudaMalloc (a
host that owns all device memory, a plugin that must not allocate after
start-up).  It must report the same Gershgorin dt_s and lambda_max as
daeti_prepare + daeti_get_stability, call after call, while reusing one fixed
device array.  This file is named so that pytest collects it last.

Tolerances: dt_s within 1e-12 relative (as in the parity tests); lambda_max
within 1e-10 relative (both run the same Lanczos routine to convergence; its
dot products are summed with atomics, so the last bits may differ).
"""
import numpy as np
import pytest

import inputs as I
from parity_util import ensure_lib, gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _context_path(binding, wl):
    s = binding.solver_from_workload(wl, precision="fp64")
    st = s.daeti_get_stability()
    s.close()
    return st["dt_s"], st["lambda_max"]


@pytest.mark.parametrize("which", ["slab", "square", "sheet"])
def test_noalloc_matches_context_path_on_two_calls(which):
    binding = ensure_lib()
    wl = {"slab": I.tp06_slab_3d(), "square": I.ms_square_2d(),
          "sheet": I.aniso_sheet_2d(n=61, length=0.6)}[which]
    ref_dts, ref_lam = _context_path(binding, wl)
    for _ in range(2):
        dts, lam = binding.daeti_grid_stability_noalloc(wl.dim, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
        assert abs(dts - ref_dts) <= 1e-12 * ref_dts
        assert abs(lam - ref_lam) <= 1e-10 * ref_lam


def test_noalloc_rejects_oversized_grid():
    binding = ensure_lib()
    n = (1001, 1001, 1)
    ne = 1000 * 1000
    with pytest.raises(binding.DaetiError) as e:
        binding.daeti_grid_stability_noalloc(2, n, 0.01, np.full(ne, 0.001), np.full(ne, 0.001), None)
    assert e.value.code == binding.EINVAL and "exceeds" in str(e.value)


def test_noalloc_rejects_conductivity_varying_within_a_layer():
    binding = ensure_lib()
    wl = I.tp06_slab_3d(9, 7, 5)
    d = wl.d_long.copy()
    d[3] *= 1.5
    with pytest.raises(binding.DaetiError) as e:
        binding.daeti_grid_stability_noalloc(wl.dim, wl.n, wl.h, d, wl.d_trans, wl.fibre)
    assert e.value.code == binding.EUNSUPPORTED


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream and reads results on the host, so on a
    stream under capture it must return EINVAL before any work (and leave the
    capture intact); afterwards it works as before."""
    import torch

    binding = ensure_lib()
    wl = I.ms_square_2d(n=11)
    ref_dts, _ = _context_path(binding, wl)
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device="cuda")
    with torch.cuda.graph(graph, stream=stream):
        x += 1.0
        with pytest.raises(binding.DaetiError) as e:
            binding.daeti_grid_stability_noalloc(wl.dim, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre, stream=stream)
    assert e.value.code == binding.EINVAL and "capturing" in str(e.value)
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0            # recorded by the capture, run by the one replay
    dts, _ = binding.daeti_grid_stability_noalloc(wl.dim, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
    assert abs(dts - ref_dts) <= 1e-12 * ref_dts
