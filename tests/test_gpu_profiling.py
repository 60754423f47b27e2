"""Per-kernel timing modes leave results unchanged and count every launch.

Mode 1 times plain launches; mode 2 replays graphs whose launches are
bracketed by event-record nodes.  Both must give the state of an untimed run
bit for bit, and count one reaction and l diffusion launches per step (fused
step-I sub-step) with positive times.
"""
import numpy as np
import pytest

import inputs as I
from parity_util import ensure_lib, gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("mode", [1, 2])
def test_profiling_modes_count_launches_and_keep_results(mode):
    binding = ensure_lib()
    wl = I.tp06_slab_3d(21, 17, 6, t_end=10.0)
    ref = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=20)
    ref.daeti_advance(10.0)
    want = ref.daeti_read_state()
    ref.close()
    s = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=20)
    st = s.daeti_get_stability()
    s.daeti_set_profiling(mode)
    s.daeti_advance(10.0)
    got = s.daeti_read_state()
    tr, nr = s.daeti_get_kernel_time(0)
    td, nd = s.daeti_get_kernel_time(1)
    s.daeti_set_profiling(0)
    s.close()
    assert np.array_equal(got, want)
    assert nr == 100 and nd == 100 * st["l"]
    assert tr > 0 and td > 0
