"""The bench slab, tet-slab and batch workloads at their full sizes, in the
bench's launch configurations (FP32 with compensated V, CUDA graphs).

The oracle cannot run 2 M nodes or 13 M nodes in seconds, so these check
what holds at any size against paths that the oracle pins at small sizes:
sampled batch tissues bit for bit against the same tissues advanced alone
(the single-tissue path is oracle-checked), the smallest Mitchell-Schaeffer
and TP06 tissues of the batch against the oracle itself, and the full tet
slab in FP32 against the FP64 path (oracle-checked on small tet meshes)
within the FP32 tolerances, and the headline slab over its whole 500 ms run
in FP32 against the FP64 path (oracle-checked on reduced slabs over whole
action potentials)."""
import numpy as np
import pytest

import inputs as I
from parity_util import act_error, ensure_lib, gpu_available, run_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def test_full_tet_slab_fp32_against_fp64():
    binding = ensure_lib()
    wl = I.tet_slab_3d(t_end=50.0)                   # 201 x 201 x 51, 2.06 M nodes
    out = {}
    for prec in ("fp32_kahan", "fp64"):
        s = binding.solver_from_workload(wl, precision=prec, graph_steps=20)
        assert s.daeti_get_stability()["l"] == 5
        s.daeti_advance(5.0)
        out[prec] = (s.daeti_read_v(), s.daeti_read_activation())
        s.close()
    (v32, a32), (v64, a64) = out["fp32_kahan"], out["fp64"]
    assert np.all(np.isfinite(v32))
    assert float(np.max(np.abs(v32 - v64))) <= 2.0
    da, same, n_act = act_error(a32, a64)
    assert da <= 0.5
    assert n_act > 0                                 # the S1 front has started
    # Activated sets: equal, except nodes on the front whose V at the last
    # synchronisation lies within the FP32 V tolerance of the threshold (there
    # a 2 mV difference decides whether -40 mV has been crossed yet).
    differ = (a32 >= 0) != (a64 >= 0)
    vth = wl.v_threshold if wl.v_threshold is not None else -40.0
    near = np.abs(v64 - vth) <= 2.0
    assert not np.any(differ & ~near), (int(differ.sum()), int((differ & ~near).sum()))
    assert int(differ.sum()) <= max(1, n_act // 1000)


def test_full_batch_sampled_tissues():
    binding = ensure_lib()
    wls = I.batch_tissues()                          # 512 tissues, 32..256 nodes a side
    batch = binding.Batch(precision="fp32_kahan", graph_steps=20)
    for w in wls:
        d = binding.describe_workload(w, precision="fp32_kahan")
        batch.daeti_batch_add(d)
        d.close()
    batch.daeti_batch_prepare()
    assert batch.daeti_batch_info()["n_tissues"] == 512
    batch.daeti_batch_advance(5.0)
    sizes = np.array([w.n_nodes for w in wls])
    rng = np.random.default_rng(20110474)
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))} | set(rng.choice(len(wls), 6, replace=False).tolist()))
    for t in picks:
        s = binding.solver_from_workload(wls[t], precision="fp32_kahan")
        s.daeti_advance(5.0)
        assert np.array_equal(batch.daeti_batch_read_v(t), s.daeti_read_v()), t
        assert np.array_equal(batch.daeti_batch_read_activation(t), s.daeti_read_activation()), t
        s.close()
    for model in ("ms", "tp06"):
        t = min((i for i, w in enumerate(wls) if w.model == model), key=lambda i: sizes[i])
        o, oa, _ = run_oracle(wls[t], 50, 50)
        mv = 100.0 if model == "ms" else 1.0
        assert float(np.max(np.abs(batch.daeti_batch_read_v(t) - o[-1]))) * mv <= 2.0, model
        da, same, _ = act_error(batch.daeti_batch_read_activation(t), oa)
        assert same and da <= 0.5, model
    batch.close()


@pytest.mark.parametrize("dims", [(101, 101, 26), (401, 401, 26)])
def test_yrun_diffusion_bit_identical_at_bench_sizes(dims):
    """The 3D diffusion kernel with runs of 2 and 4 nodes along y per thread
    (diff_block = 0, packed FP32) against the one-thread-per-node kernel on
    the bench slab and the 4.18 M-node slab, over the stimulus and upstroke
    (lists, uniform-k votes and plain sub-steps), FP32 with compensated V:
    identical states."""
    binding = ensure_lib()
    wl = I.tp06_slab_3d(*dims, t_end=6.0)
    out = []
    for diff_block, rows in ((256, 0), (0, 2), (0, 4)):
        s = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=20)
        s.daeti_set_tuning(diff_block=diff_block, diff_rows=rows)
        s.daeti_advance(3.0)
        s.daeti_advance(6.0)
        out.append((s.daeti_read_v(), s.daeti_read_activation(), s.daeti_get_substeps()))
        s.close()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
        assert np.array_equal(out[0][1], o[1])
        assert out[0][2] == o[2]


def test_full_bench_slab_fp32_against_fp64_whole_run():
    """The headline workload as the bench runs it (101 x 101 x 26 TP06 slab,
    500 ms, FP32 with compensated V, graphs of 100 steps with programmatic
    dependent launch, k lists) against the FP64 path over the whole run,
    V of every node every 10 ms: within 2 mV, activation within 0.5 ms, the
    same activated set, every node activated and back at rest at the end."""
    binding = ensure_lib()
    wl = I.tp06_slab_3d(t_end=500.0)
    s32 = binding.solver_from_workload(wl, precision="fp32_kahan", graph_steps=100)
    s32.daeti_set_tuning(react_block=128, react_min_blocks=8, diff_block=256, fuse_diffusion=1, bucket_k=1, pdl=1)
    s64 = binding.solver_from_workload(wl, precision="fp64", graph_steps=100)
    worst = 0.0
    for t in range(10, 501, 10):
        s32.daeti_advance(float(t))
        s64.daeti_advance(float(t))
        worst = max(worst, float(np.max(np.abs(s32.daeti_read_v() - s64.daeti_read_v()))))
    a32, a64 = s32.daeti_read_activation(), s64.daeti_read_activation()
    v64 = s64.daeti_read_v()
    s32.close()
    s64.close()
    assert worst <= 2.0, worst
    da, same, n_act = act_error(a32, a64)
    assert same and da <= 0.5, (same, da)
    assert n_act == wl.n_nodes
    assert float(v64.max()) < -70.0
