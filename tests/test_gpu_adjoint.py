"""GPU discrete adjoint (through the C ABI) against the FP64 oracle adjoint and
against central differences of the GPU forward with the recorded schedule."""
import numpy as np
import pytest

import inputs as I
from parity_util import ensure_lib, gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _small(n=12, n_steps=300, seed=0, d_scale=1.0):
    from oracle import adjoint, fem

    wl = I.ms_square_2d(n=n, length=(n - 1) * 0.025)
    rng = np.random.default_rng(seed)
    d_node = d_scale * 0.001 * np.exp(0.3 * rng.standard_normal(n * n))
    conn = fem.grid_elements(2, wl.n)
    d_elem = adjoint.element_d_from_nodes(conn, d_node)
    sensors = np.sort(rng.choice(n * n, size=8, replace=False))
    target = adjoint.MSAdjointGrid(2, wl.n, wl.h, d_elem * 1.15, wl.model_params, wl.stimuli)
    _, rec = target.forward(n_steps, sensors, 10)
    prob = adjoint.MSAdjointGrid(2, wl.n, wl.h, d_elem, wl.model_params, wl.stimuli)
    return wl, prob, d_elem, sensors, rec["samples"], n_steps


def _gpu(wl, d_elem, precision, **kw):
    binding = ensure_lib()
    w = I.Workload(**{**wl.__dict__})
    w.d_long = d_elem
    w.d_trans = d_elem
    w.fibre = None
    return binding.solver_from_workload(w, precision=precision, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_kahan", 2e-3)])
def test_adjoint_matches_oracle(precision, tol):
    wl, prob, d_elem, sensors, data, n_steps = _small()
    loss_o, g_o, gt_o, _ = prob.gradient(n_steps, sensors, 10, data)
    s = _gpu(wl, d_elem, precision)
    loss, g, gt = s.daeti_adjoint(sensors, data, n_steps, 10, n_slots=6, n_elem=len(d_elem))
    t_after = s.time
    s.close()
    assert t_after == 0.0
    assert abs(loss - loss_o) <= tol * loss_o
    assert _rel(g, g_o) <= tol
    assert abs(gt - gt_o) <= tol * abs(gt_o)


@pytest.mark.parametrize("d_scale,l", [(4.0, 2), (5.0, 3)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_kahan", 2e-3)])
def test_adjoint_with_diffusion_substeps(d_scale, l, precision, tol):
    """l > 1 (several diffusion sub-steps per half step, each reversed), with one
    checkpoint slot (recomputation from the start) and with five."""
    wl, prob, d_elem, sensors, data, n_steps = _small(n_steps=200, d_scale=d_scale)
    assert prob.l == l
    loss_o, g_o, gt_o, _ = prob.gradient(n_steps, sensors, 10, data)
    for slots in (1, 5):
        s = _gpu(wl, d_elem, precision)
        assert s.daeti_get_stability()["l"] == l
        loss, g, gt = s.daeti_adjoint(sensors, data, n_steps, 10, n_slots=slots, n_elem=len(d_elem))
        v_end = s.daeti_read_v()
        s.close()
        assert abs(loss - loss_o) <= tol * loss_o
        assert _rel(g, g_o) <= tol
        assert abs(gt - gt_o) <= tol * abs(gt_o)
        assert np.all(v_end == 0.0)          # the context is back at its (resting) start


def test_checkpoint_slot_count_does_not_change_gradient():
    wl, prob, d_elem, sensors, data, n_steps = _small(n=10, n_steps=200)
    out = []
    for slots in (1, 2, 5, 32):
        s = _gpu(wl, d_elem, "fp64")
        out.append(s.daeti_adjoint(sensors, data, n_steps, 10, n_slots=slots, n_elem=len(d_elem)))
        s.close()
    for o in out[1:]:
        assert abs(o[0] - out[0][0]) <= 1e-12 * out[0][0]
        assert _rel(o[1], out[0][1]) <= 1e-12
        assert abs(o[2] - out[0][2]) <= 1e-12 * abs(out[0][2])


def test_full_adjoint_config_against_central_differences():
    """256 x 256 MS tissue, log-normal nodal D, 2000 steps, 64 sensors sampled every
    1 ms, 32 checkpoint slots: FP64 and FP32 adjoint gradients against central
    differences of the FP64 forward (recorded schedule replayed) on 20 directions."""
    from paper_2011_04747_gb300.autograd import MisfitProblem

    wl, d_node, sensors, sample_dt = I.ms_adjoint_2d()
    conn = MisfitProblem(2, wl.n, wl.h, wl.model_params, wl.stimuli, sensors, None, 0).elements()
    d_elem = d_node[conn].mean(axis=1)
    n_steps, every = 2000, 10
    # data: sensor traces of a run with a perturbed field
    g2 = I.lognormal_field_2d(wl.n[0], wl.h, seed_index=23) / 0.001
    d_target = (d_node * g2 ** (0.5))[conn].mean(axis=1)
    tgt = _gpu(wl, d_target, "fp64")
    data = []
    for j in range(n_steps // every):
        tgt.daeti_advance((j + 1) * every * 0.1)
        data.append(tgt.daeti_read_v()[sensors])
    tgt.close()
    data = np.array(data)

    s64 = _gpu(wl, d_elem, "fp64")
    loss0, _, _ = s64.daeti_adjoint(sensors, data, n_steps, every, 32, flags=1)      # record the schedule
    loss, g64, gt64 = s64.daeti_adjoint(sensors, data, n_steps, every, 32, n_elem=len(d_elem))
    assert abs(loss - loss0) <= 1e-12 * loss0
    s32 = _gpu(wl, d_elem, "fp32_kahan")
    loss32, g32, gt32 = s32.daeti_adjoint(sensors, data, n_steps, every, 32, n_elem=len(d_elem))
    s32.close()
    assert abs(loss32 - loss) <= 2e-3 * loss

    def nodal(ge):
        g = np.zeros(wl.n_nodes)
        np.add.at(g, conn, (ge / 4.0)[:, None])
        return g

    gn64, gn32 = nodal(g64), nodal(g32)
    rng = np.random.default_rng(2011047 + 4)
    worst64, worst32 = 0.0, 0.0
    for _ in range(20):
        u = rng.standard_normal(wl.n_nodes) * d_node
        eps = 1e-6
        lp = lm = None
        for sgn in (1.0, -1.0):
            de = (d_node + sgn * eps * u)[conn].mean(axis=1)
            s64.daeti_update_conductivity(de, de, None)
            val = s64.daeti_adjoint(sensors, data, n_steps, every, 32, flags=2)[0]
            if sgn > 0:
                lp = val
            else:
                lm = val
        fd = (lp - lm) / (2 * eps)
        worst64 = max(worst64, abs(gn64 @ u - fd) / abs(fd))
        worst32 = max(worst32, abs(gn32 @ u - fd) / abs(fd))
    s64.close()
    assert worst64 <= 1e-5, worst64
    assert worst32 <= 1e-3, worst32


def test_nodal_conductivity_and_nodal_gradient():
    """Per-node D (daeti_set_conductivity_nodal: element D = mean of its nodes)
    runs like the element means given directly, and the per-node gradient is
    the chain rule of the element gradient (the oracle's nodal_gradient)."""
    from oracle import adjoint, fem

    wl, prob, d_elem, sensors, data, n_steps = _small(n=10, n_steps=150)
    rng = np.random.default_rng(3)
    d_node = 0.001 * np.exp(0.3 * rng.standard_normal(wl.n_nodes))
    conn = fem.grid_elements(2, wl.n)
    de = adjoint.element_d_from_nodes(conn, d_node)
    binding = ensure_lib()
    a = _gpu(wl, de, "fp64")
    b = binding.Solver(precision="fp64", dt=wl.dt, dt0=wl.dt0, v_threshold=wl.v_threshold)
    b.daeti_set_mesh_grid(wl.dim, wl.n, wl.h)
    b.daeti_set_conductivity_nodal(d_node)
    b.daeti_set_cell_model(wl.model, tuple(wl.model_params))
    for st in wl.stimuli:
        b.daeti_add_stimulus(st.nodes, st.t_start, st.duration, st.amplitude, st.period, st.count)
    b.daeti_prepare()
    la, ga, ta = a.daeti_adjoint(sensors, data, n_steps, 10, n_slots=6, n_elem=len(de))
    lb, gb, tb = b.daeti_adjoint(sensors, data, n_steps, 10, n_slots=6, nodal=True)
    assert gb.shape == (wl.n_nodes,)
    assert abs(la - lb) <= 1e-12 * la and abs(ta - tb) <= 1e-12 * abs(ta)
    assert _rel(gb, adjoint.nodal_gradient(conn, ga, wl.n_nodes)) <= 1e-12
    a.close()
    b.close()


def test_autograd_wrapper():
    import torch

    from paper_2011_04747_gb300.autograd import MisfitProblem, MonodomainMisfit

    wl, prob, d_elem, sensors, data, n_steps = _small(n=10, n_steps=150)
    rng = np.random.default_rng(3)
    d_node = torch.tensor(0.001 * np.exp(0.3 * rng.standard_normal(wl.n_nodes)), requires_grad=True)
    tau = torch.tensor(150.0, dtype=torch.float64, requires_grad=True)
    p = MisfitProblem(2, wl.n, wl.h, wl.model_params, wl.stimuli, sensors, data, n_steps, precision="fp64")
    loss = MonodomainMisfit.apply(d_node, tau, p)
    (2.0 * loss).backward()
    from oracle import adjoint

    conn = p.elements()
    o = adjoint.MSAdjointGrid(2, wl.n, wl.h, adjoint.element_d_from_nodes(conn, d_node.detach().numpy()),
                              wl.model_params, wl.stimuli)
    lo, ge, gt, _ = o.gradient(n_steps, sensors, 10, data)
    assert abs(float(loss.detach()) - lo) <= 1e-9 * lo
    assert _rel(d_node.grad.numpy(), 2.0 * adjoint.nodal_gradient(conn, ge, wl.n_nodes)) <= 1e-8
    assert abs(float(tau.grad) - 2.0 * gt) <= 1e-8 * abs(2.0 * gt)
    # later calls reuse the prepared solver (new D and tau_close by updates) ...
    for scale, tau_v, prepares in ((1.2, 140.0, 1), (1.1, 160.0, 1), (30.0, 150.0, 2)):
        d2 = torch.tensor(d_node.detach().numpy() * scale, requires_grad=True)
        t2 = torch.tensor(tau_v, dtype=torch.float64, requires_grad=True)
        loss2 = MonodomainMisfit.apply(d2, t2, p)
        loss2.backward()
        params = list(wl.model_params)
        params[3] = tau_v
        # ... with the prepared l while it is stable (D x 30 needs a new prepare)
        assert p.prepares == prepares
        l_used = p._solver.daeti_get_stability()["l"]
        d2e = adjoint.element_d_from_nodes(conn, d2.detach().numpy())
        o2 = adjoint.MSAdjointGrid(2, wl.n, wl.h, d2e, params, wl.stimuli, l_override=l_used)
        if prepares == 2:
            assert l_used == adjoint.MSAdjointGrid(2, wl.n, wl.h, d2e, params, wl.stimuli).l > 1
        lo2, ge2, gt2, _ = o2.gradient(n_steps, sensors, 10, data)
        assert abs(float(loss2.detach()) - lo2) <= 1e-9 * lo2
        assert _rel(d2.grad.numpy(), adjoint.nodal_gradient(conn, ge2, wl.n_nodes)) <= 1e-8
        assert abs(float(t2.grad) - gt2) <= 1e-8 * abs(gt2)
    p.close()


def test_adjoint_graph_replay_repeats_exactly():
    """The gradient sweep is captured once and replayed: a second call (and a call
    after a different request) returns the same loss and gradients."""
    wl, prob, d_elem, sensors, data, n_steps = _small(n=10, n_steps=120)
    s = _gpu(wl, d_elem, "fp32_kahan")
    a = s.daeti_adjoint(sensors, data, n_steps, 10, n_slots=4, n_elem=len(d_elem))
    b = s.daeti_adjoint(sensors, data, n_steps, 10, n_slots=4, n_elem=len(d_elem))
    c = s.daeti_adjoint(sensors, data[:6], 60, 10, n_slots=4, n_elem=len(d_elem))
    d = s.daeti_adjoint(sensors, data, n_steps, 10, n_slots=4, n_elem=len(d_elem))
    s.close()
    for x in (b, d):
        assert abs(x[0] - a[0]) <= 1e-12 * a[0] and abs(x[2] - a[2]) <= 1e-9 * abs(a[2])
        assert np.allclose(x[1], a[1], rtol=1e-9, atol=1e-12 * np.abs(a[1]).max())
    assert c[0] < a[0]
