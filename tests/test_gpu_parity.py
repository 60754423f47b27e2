"""GPU (CUDA through the C ABI) vs CPU oracle, element by element.

Tolerances: FP64 max|dV| <= 0.5 mV and activation-time error <= 0.1 ms;
FP32 with compensated V: <= 2 mV and <= 0.5 ms.  Mitchell-Schaeffer voltages
are dimensionless and compared in mV through V_mV = 100 v - 80.
"""
import numpy as np
import pytest

import inputs as I
from oracle import scheme
from parity_util import act_error, gpu_available, run_gpu, run_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = {"fp64": (0.5, 0.1), "fp32_kahan": (2.0, 0.5)}


def _mv(wl):
    return 100.0 if wl.model in ("ms", "cubic") else 1.0


def _compare(wl, n_steps, every, precision, scheme_name="daeti", tol=None, **gpu_opts):
    g, ga, stab, _ = run_gpu(wl, n_steps, every, precision=precision, scheme=scheme_name, **gpu_opts)
    o, oa, sim = run_oracle(wl, n_steps, every, scheme_name=scheme_name)
    assert stab["l"] == sim.l and stab["k_max"] == sim.k_max
    assert abs(stab["dt_s"] - sim.dt_s) <= 1e-12 * sim.dt_s
    assert abs(stab["dt"] - sim.dt) <= 1e-15
    dv = float(np.max(np.abs(g - o))) * _mv(wl)
    da, same, nboth = act_error(ga, oa)
    tv, ta = tol or TOL[precision]
    assert same, "activated node sets differ"
    assert dv <= tv, f"max|dV| = {dv:.4g} mV"
    assert da <= ta, f"max|d act| = {da:.4g} ms"
    return dv, da, nboth


def test_ms_square_full_config_fp64():
    wl = I.ms_square_2d()                       # 41 x 41, 100 ms, dt = 0.1
    dv, da, n = _compare(wl, 1000, 10, "fp64")
    assert n == wl.n_nodes                       # the wave crosses the whole square


def test_ms_square_full_config_fp32():
    wl = I.ms_square_2d()
    _compare(wl, 1000, 10, "fp32_kahan")


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_tp06_slab_small(precision):
    wl = I.tp06_slab_3d(21, 17, 6)              # ragged in x and y, 3D 27-point stencil
    _compare(wl, 400, 20, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_sheet_with_diffusion_substeps(precision):
    # h = 100 um, d0 = 0.0017, rho = 0.25: dt_s = 0.0132 ms, l = 3 (odd)
    wl = I.aniso_sheet_2d(n=37, length=0.36, model="tp06", amp=60.0)
    g, ga, stab, _ = run_gpu(wl, 1, 1, precision=precision)
    assert stab["l"] == 3
    _compare(wl, 300, 10, precision)


def test_sheet_ceil_rounding_l4():
    wl = I.aniso_sheet_2d(n=21, length=0.2, model="ms")
    g, ga, stab, _ = run_gpu(wl, 200, 10, precision="fp64", l_rounding="ceil")
    o, oa, sim = run_oracle(wl, 200, 10, l_round="ceil")
    assert stab["l"] == sim.l == 4
    assert float(np.max(np.abs(g - o))) * 100 <= 0.5


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_tet_mesh_sell_path(precision):
    wl = I.tet_slab_3d(13, 11, 6, h=0.02, fibrosis=0.3, scar_radius=0.05, s2_time=15.0)
    _compare(wl, 300, 20, precision)


def _heterogeneous(wl, seed=7):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.3, 1.7, wl.n_elems)
    wl.d_long = wl.d_long * f
    wl.d_trans = wl.d_trans * f
    return wl


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_heterogeneous_grid_per_node_rows(precision):
    """Structured grids whose D varies within a layer: one stencil row per node
    (2D isotropic Mitchell-Schaeffer; 3D TP06 slab with rotating fibres)."""
    _compare(_heterogeneous(I.ms_square_2d(n=23)), 400, 20, precision)
    _compare(_heterogeneous(I.tp06_slab_3d(13, 11, 6)), 300, 20, precision)
    if precision == "fp32_kahan":   # 67 600 nodes: the operator rows are built in two blocks
        _compare(_heterogeneous(I.ms_square_2d(n=260, length=259 * 0.025)), 100, 50, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_transmural_slab_per_node_cell_types(precision):
    """TP06 endocardial, mid-myocardial and epicardial layers through the wall
    (one cell type per node) against the oracle over the upstroke and plateau."""
    wl = I.tp06_slab_3d(13, 11, 9, transmural=True)
    _compare(wl, 1500, 100, precision)


def test_per_node_cell_types_of_one_type_equal_the_model_parameter():
    from parity_util import ensure_lib

    binding = ensure_lib()
    for ct in (0, 1, 2):
        wl = I.tp06_slab_3d(9, 7, 5, celltype=ct)
        w2 = I.Workload(**{**wl.__dict__})
        w2.cell_type = np.full(wl.n_nodes, ct, dtype=np.uint8)
        a = binding.solver_from_workload(wl, precision="fp32_kahan")
        b = binding.solver_from_workload(w2, precision="fp32_kahan")
        a.daeti_advance(20.0)
        b.daeti_advance(20.0)
        assert np.array_equal(a.daeti_read_state(), b.daeti_read_state()), ct
        a.close()
        b.close()
    s = binding.Solver()
    s.daeti_set_mesh_grid(2, (5, 5), 0.025)
    for bad in (np.zeros(24, np.uint8), np.full(25, 3, np.uint8)):
        with pytest.raises(binding.DaetiError) as e:
            s.daeti_set_cell_types(bad)
        assert e.value.code == binding.EINVAL
    s.daeti_set_conductivity(np.full(16, 0.001), None, None)
    s.daeti_set_cell_model("ms")
    s.daeti_set_cell_types(np.zeros(25, np.uint8))
    with pytest.raises(binding.DaetiError) as e:
        s.daeti_prepare()                        # cell types need the TP06 model
    assert e.value.code == binding.EINVAL
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_k_rule_from_the_reaction_rate(precision):
    """Reading R-k2 (k from the reaction's dV/dt at the previous step's last
    sub-step) against the oracle with the same reading; it changes the run."""
    cases = [(I.ms_square_2d(), 600, 50), (I.tp06_slab_3d(13, 11, 6), 300, 50)]
    for wl, n_steps, every in cases:
        g, ga, stab, _ = run_gpu(wl, n_steps, every, precision=precision, k_rule="reaction")
        o, oa, _ = run_oracle(wl, n_steps, every, k_rule="reaction")
        tv, ta = TOL[precision]
        assert float(np.max(np.abs(g - o))) * _mv(wl) <= tv, wl.name
        da, same, n_act = act_error(ga, oa)
        assert same and da <= ta and n_act > 0, wl.name
        if wl.model == "tp06":                   # the two readings give different TP06 runs
            o_total, _, _ = run_oracle(wl, n_steps, every)
            assert float(np.max(np.abs(o - o_total))) > 5.0


def test_conductivity_update_switches_to_per_node_rows():
    """A grid prepared with one D per layer gets per-node stencil rows when an
    update makes D vary within a layer; the run then equals one prepared with
    that D (same l).  Updating back to the per-layer D keeps per-node rows and
    agrees with the per-layer table to rounding."""
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl = I.tp06_slab_3d(13, 11, 6)
    f = np.random.default_rng(11).uniform(0.95, 1.0, wl.n_elems)
    het = (wl.d_long * f, wl.d_trans * f)

    def make(dl, dtr):
        w = I.Workload(**{**wl.__dict__})
        w.d_long, w.d_trans = dl, dtr
        return binding.solver_from_workload(w, precision="fp64")

    a, b = make(wl.d_long, wl.d_trans), make(*het)
    a.daeti_update_conductivity(het[0], het[1], wl.fibre)
    assert a.daeti_get_stability()["l"] == b.daeti_get_stability()["l"] == 1
    a.daeti_advance(10.0)
    b.daeti_advance(10.0)
    assert np.array_equal(a.daeti_read_state(), b.daeti_read_state())
    assert np.array_equal(a.daeti_read_activation(), b.daeti_read_activation())
    c = make(wl.d_long, wl.d_trans)
    b.daeti_update_conductivity(wl.d_long, wl.d_trans, wl.fibre)
    b.daeti_init_state()
    b.daeti_advance(10.0)
    c.daeti_advance(10.0)
    assert np.allclose(b.daeti_read_v(), c.daeti_read_v(), rtol=0.0, atol=1e-9)
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("scheme_name", ["ost", "ostar"])
def test_scheme_variants(scheme_name):
    wl = I.aniso_sheet_2d(n=21, length=0.2, model="ms")
    if scheme_name == "ost":
        wl.dt = 0.01
    _compare(wl, 300, 20, "fp64", scheme_name=scheme_name)


def test_bucketing_and_graphs_do_not_change_results():
    wl = I.tp06_slab_3d(15, 13, 5, t_end=10)
    ref = None
    for bucket in (True, False):
        for graph in (0, 20):
            g, ga, _, st = run_gpu(wl, 100, 50, precision="fp32_kahan", bucket_k=bucket, graph_steps=graph)
            if ref is None:
                ref = (g, ga, st)
            else:
                assert np.array_equal(g, ref[0]) and np.array_equal(ga, ref[1]) and np.array_equal(st, ref[2])


def test_checkpoint_roundtrip_is_exact():
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl = I.tp06_slab_3d(11, 11, 5)
    a = binding.solver_from_workload(wl, precision="fp32_kahan")
    a.daeti_advance(3.0)
    ck = a.daeti_save_state()
    a.daeti_advance(8.0)
    va = a.daeti_read_v()
    a.daeti_load_state(ck)
    assert abs(a.time - 3.0) < 1e-12
    a.daeti_advance(8.0)
    assert np.array_equal(a.daeti_read_v(), va)
    a.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_initial_state_from_host_array(precision):
    """A caller's initial state is stored rounded once to the state precision,
    in the chunked layout with a node count that is not a multiple of 32, and
    the published state passed explicitly runs exactly like the default."""
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl = I.tp06_slab_3d(9, 7, 3)                 # 189 nodes
    s = binding.solver_from_workload(wl, precision=precision)
    default = s.daeti_read_state()
    rng = np.random.default_rng(5)
    custom = default * (1.0 + 0.01 * rng.standard_normal(default.shape))
    s.daeti_advance(1.0)
    s.daeti_init_state(custom)
    assert s.time == 0.0
    want = custom if precision == "fp64" else custom.astype(np.float32).astype(np.float64)
    assert np.array_equal(s.daeti_read_state(), want)
    s.daeti_init_state(default)
    s.daeti_advance(5.0)
    a = s.daeti_read_state()
    s.daeti_init_state()
    s.daeti_advance(5.0)
    assert np.array_equal(s.daeti_read_state(), a)
    s.close()


def test_error_paths():
    from parity_util import ensure_lib

    binding = ensure_lib()
    s = binding.Solver()
    with pytest.raises(binding.DaetiError) as e:
        s.daeti_advance(1.0)
    assert e.value.code == binding.ESTATE
    s.close()
    wl = I.ms_square_2d(n=11)
    s = binding.solver_from_workload(wl, precision="fp64")
    with pytest.raises(binding.DaetiError) as e:
        s.daeti_advance(0.05)                    # not a whole number of steps
    assert e.value.code == binding.EINVAL
    bad = np.zeros((2, wl.n_nodes))
    bad[0, 3] = np.nan
    with pytest.raises(binding.DaetiError):
        s.daeti_init_state(bad)
    s.close()
    # a blown-up stimulus makes V non-finite: reported at synchronisation, context stays usable
    wl.stimuli[0].amplitude = 1e38
    s = binding.solver_from_workload(wl, precision="fp32")
    s.daeti_advance(2.0)
    with pytest.raises(binding.DaetiError) as e:
        s.daeti_synchronize()
    assert e.value.code == binding.ENONFINITE
    s.daeti_init_state()
    # launch shapes outside their ranges are refused and leave the tuning as it was
    before = s.daeti_get_tuning()
    for bad_shape in (dict(diff_rows=3), dict(diff_rows=-1), dict(react_block=48), dict(diff_block=512),
                      dict(react_min_blocks=7), dict(pdl=2)):
        with pytest.raises(binding.DaetiError) as e:
            s.daeti_set_tuning(**bad_shape)
        assert e.value.code == binding.EINVAL, bad_shape
    assert s.daeti_get_tuning() == before
    s.close()
    # tet meshes: an index out of range, a node in no tetrahedron
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=float) * 0.1
    for tets in (np.array([[0, 1, 2, 5]]), np.array([[0, 1, 2, 3]])):
        s = binding.Solver(precision="fp64")
        with pytest.raises(binding.DaetiError) as e:
            s.daeti_set_mesh_tet(xyz, tets)
        assert e.value.code == binding.EINVAL
        s.close()


def test_degenerate_inputs():
    from parity_util import ensure_lib

    binding = ensure_lib()
    # smallest grid, no stimulus, zero conductivity: reaction only
    wl = I.ms_square_2d(n=2)
    wl.stimuli = []
    wl.d_long[:] = 0.0
    wl.d_trans[:] = 0.0
    g, ga, stab, _ = run_gpu(wl, 20, 20, precision="fp64")
    assert stab["l"] == 1
    assert np.all(g == 0.0) and np.all(ga == -1.0)
    # advancing by zero steps is a no-op
    s = binding.solver_from_workload(I.ms_square_2d(n=5), precision="fp64")
    s.daeti_advance(0.0)
    assert s.time == 0.0
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_full_slab_bench_config_first_steps(precision):
    """The bench workload (101 x 101 x 26 TP06 slab) at full size, in the bench's
    launch configuration (graphs, bucketing), over the stimulus and first upstrokes."""
    wl = I.tp06_slab_3d()
    _compare(wl, 30, 10, precision)


@pytest.mark.parametrize("wl_name", ["slab", "slab_wide", "slab_even", "sheet2d", "sheet_l3", "sheet_l4", "hetero_slab"])
def test_launch_shapes_do_not_change_results(wl_name):
    """Fused or separate diffusion sub-step, register caps, block sizes, k lists,
    programmatic dependent launch or plain launches, graphs, and the
    diff_block = 0 kernels (2D shared-memory tiles; in 3D runs of 2 or 4 nodes
    along y per thread with packed FP32 arithmetic, and the one-thread-per-node
    kernel they fall back to in FP64) give bit-identical states (l = 1, 3
    and 4)."""
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl, opts = {"slab": (I.tp06_slab_3d(23, 19, 9, t_end=12), {}),
                "sheet2d": (I.aniso_sheet_2d(n=41, length=1.0, model="tp06"), {}),
                "sheet_l3": (I.aniso_sheet_2d(n=37, length=0.36, model="tp06"), {}),
                "sheet_l4": (I.aniso_sheet_2d(n=45, length=0.44, model="tp06"), dict(l_rounding="ceil")),
                "slab_wide": (I.tp06_slab_3d(45, 21, 7, t_end=12), {}),
                "slab_even": (I.tp06_slab_3d(24, 18, 6, t_end=12), {}),
                "hetero_slab": (_heterogeneous(I.tp06_slab_3d(23, 19, 9, t_end=12)), {})}[wl_name]
    variants = [dict(),
                dict(fuse_diffusion=0),
                dict(react_min_blocks=10),
                dict(react_min_blocks=10, react_block=64, fuse_diffusion=0),
                dict(pdl=0),
                dict(pdl=0, react_block=64, graph_steps=0),
                dict(bucket_k=0, graph_steps=0),
                dict(graph_steps=6, diff_block=128),
                dict(diff_block=256, fuse_diffusion=0, graph_steps=0),
                dict(diff_block=0),
                dict(diff_block=0, fuse_diffusion=0, graph_steps=0),
                dict(diff_block=0, bucket_k=0, pdl=0),
                dict(diff_block=0, diff_rows=2),
                dict(diff_block=0, diff_rows=4, fuse_diffusion=0, graph_steps=0),
                dict(diff_block=0, diff_rows=4, bucket_k=0, pdl=0)]
    ref = None
    for prec in ("fp32_kahan", "fp64"):
        ref = None
        for v in variants:
            s = binding.solver_from_workload(wl, precision=prec, **opts)
            if wl_name.startswith("sheet_l"):
                assert s.daeti_get_stability()["l"] == int(wl_name[-1])
            s.daeti_set_tuning(**v)
            s.daeti_advance(3.1)        # odd step count: graph segments and plain steps
            s.daeti_advance(7.0)        # two advances: prologue/epilogue of the fused path twice
            out = (s.daeti_read_state(), s.daeti_read_activation())
            s.close()
            if ref is None:
                ref = out
            else:
                assert np.array_equal(out[0], ref[0]), v
                assert np.array_equal(out[1], ref[1]), v


@pytest.mark.parametrize("model,params", [("tp06", (0.0,)), ("tp06", (1.0,)), ("tp06", (2.0,)), ("ms", ())])
def test_cell_models_fp64_tight(model, params):
    """Reaction only (zero conductivity), every node paced: FP64 GPU cell models
    against the oracle's transcription to 1e-6 mV over a full action potential."""
    wl = I.ms_square_2d(n=3) if model == "ms" else I.tp06_slab_3d(3, 3, 3)
    wl.model = model
    wl.model_params = params or wl.model_params
    wl.v_threshold = 0.5 if model == "ms" else -40.0
    wl.d_long[:] = 0.0
    wl.d_trans[:] = 0.0
    amp = 1.0 if model == "ms" else 40.0
    wl.stimuli = [I.Stimulus(np.arange(wl.n_nodes), 1.0, 2.0, amp, period=300.0, count=2)]
    g, ga, _, gs = run_gpu(wl, 4000, 100, precision="fp64")
    o, oa, sim = run_oracle(wl, 4000, 100)
    scale = 100.0 if model == "ms" else 1.0
    assert float(np.max(np.abs(g - o))) * scale <= 1e-6
    np.testing.assert_allclose(gs, sim.S, rtol=1e-9, atol=1e-12)
    assert np.all(ga >= 0) and float(np.max(np.abs(ga - oa))) <= 1e-9


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp64"])
def test_probe_reads_match_the_full_field(precision):
    """daeti_read_v_nodes returns V (Kahan term applied) at the given nodes,
    repeated and unordered indices included; bad indices are EINVAL."""
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl = I.tp06_slab_3d(13, 11, 5, t_end=10)
    s = binding.solver_from_workload(wl, precision=precision)
    s.daeti_advance(3.0)
    full = s.daeti_read_v()
    nodes = np.array([0, wl.n_nodes - 1, 17, 17, 5, 300], dtype=np.int64)
    assert np.array_equal(s.daeti_read_v_nodes(nodes), full[nodes])
    big = np.arange(wl.n_nodes, dtype=np.int64)[::-1]
    assert np.array_equal(s.daeti_read_v_nodes(big), full[big])
    assert s.daeti_read_v_nodes(np.zeros(0, dtype=np.int64)).size == 0
    for bad in ([-1], [wl.n_nodes]):
        with pytest.raises(binding.DaetiError) as e:
            s.daeti_read_v_nodes(np.array(bad, dtype=np.int64))
        assert e.value.code == binding.EINVAL
    s.close()


@pytest.mark.parametrize("graph_steps", [0, 20])
def test_substep_count_equals_the_oracle_sum_of_k(graph_steps):
    """The sub-step counter (sum over steps and nodes of the k step A used),
    kept from the per-k list lengths, from n * k when every node has one k,
    and summed per node on the step after that stops holding, equals the
    oracle's sum of k in FP64 through the stimulus and the first wavefront."""
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl = I.tp06_slab_3d(15, 13, 5, t_end=40)
    n_steps = 300
    sim = scheme.simulation_from_workload(wl)
    total = 0
    for _ in range(n_steps):
        total += int(np.sum(sim.k))
        sim.step()
    s = binding.solver_from_workload(wl, precision="fp64", graph_steps=graph_steps)
    s.daeti_advance(n_steps * wl.dt)
    got = s.daeti_get_substeps()
    s.close()
    assert total > n_steps * wl.n_nodes          # k > 1 somewhere
    assert got == total


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp64"])
def test_graph_segments_without_stimulus_keep_every_pulse(precision):
    """Graph segments in which no stimulus window is open launch the reaction
    without stimuli; a pacing train whose pulses start inside, across and
    between 20-step segments gives the same state as plain launches, which
    test every window."""
    from parity_util import ensure_lib

    binding = ensure_lib()
    wl = I.ms_square_2d(n=21)
    st = wl.stimuli[0]
    # pulses of 0.35 ms every 3.7 ms from 0.55 ms: start and end at every
    # offset against the 2 ms (20-step) segments
    st.t_start, st.duration, st.period, st.count, st.amplitude = 0.55, 0.35, 3.7, 12, 3.0
    # windows that start and end exactly on segment boundaries, one that fills
    # a whole segment, and one ending on a boundary
    edge = wl.stimuli[0].nodes[:3]
    wl.stimuli = wl.stimuli + [I.Stimulus(edge, 4.0, 2.0, 3.0), I.Stimulus(edge, 9.6, 0.4, 3.0),
                               I.Stimulus(edge, 20.0, 0.1, 3.0, period=2.0, count=5)]
    out = []
    for graph_steps in (20, 0):
        s = binding.solver_from_workload(wl, precision=precision, graph_steps=graph_steps)
        s.daeti_advance(50.0)
        out.append((s.daeti_read_state(), s.daeti_read_activation()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert (out[0][1] >= 0).any()
