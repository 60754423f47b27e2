"""Pins of the oracle's discrete adjoint: central differences of the
frozen-schedule forward map (the schedule of the unperturbed run replayed)."""
import numpy as np
import pytest

import inputs as I
from oracle import adjoint


def _problem(n=12, n_steps=300, seed=0):
    wl = I.ms_square_2d(n=n, length=(n - 1) * 0.025)
    rng = np.random.default_rng(seed)
    d_node = 0.001 * np.exp(0.3 * rng.standard_normal(n * n))
    conn = adjoint._fem.grid_elements(2, wl.n)
    d_elem = adjoint.element_d_from_nodes(conn, d_node)
    prob = adjoint.MSAdjointGrid(2, wl.n, wl.h, d_elem, wl.model_params, wl.stimuli)
    sensors = np.sort(rng.choice(n * n, size=8, replace=False))
    # data: a run with a perturbed field
    target = adjoint.MSAdjointGrid(2, wl.n, wl.h, d_elem * 1.15, wl.model_params, wl.stimuli)
    _, rec = target.forward(n_steps, sensors, 10)
    return prob, conn, d_node, sensors, rec["samples"], n_steps


def test_adjoint_matches_central_differences_frozen_schedule():
    prob, conn, d_node, sensors, data, n_steps = _problem()
    loss, g_elem, g_tau, rec = prob.gradient(n_steps, sensors, 10, data)
    assert loss > 0
    g_node = adjoint.nodal_gradient(conn, g_elem, prob.n_nodes)
    rng = np.random.default_rng(5)
    replay = {"k": rec["k"], "branch": rec["branch"]}
    l0 = prob.l
    for _ in range(4):
        u = rng.standard_normal(prob.n_nodes)
        eps = 1e-6 * np.abs(d_node).max()
        lp, lm = [], []
        for sgn, store in ((1, lp), (-1, lm)):
            prob.set_d(adjoint.element_d_from_nodes(conn, d_node + sgn * eps * u), l_override=l0)
            store.append(prob.forward(n_steps, sensors, 10, data, replay=replay)[0])
        fd = (lp[0] - lm[0]) / (2 * eps)
        ad = float(g_node @ u)
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-12) + 1e-10, (fd, ad)
    prob.set_d(adjoint.element_d_from_nodes(conn, d_node), l_override=l0)
    tau = prob.ms_params[3]
    e = 1e-5 * tau
    fp = prob.forward(n_steps, sensors, 10, data, tau_close=tau + e, replay=replay)[0]
    fm = prob.forward(n_steps, sensors, 10, data, tau_close=tau - e, replay=replay)[0]
    fd = (fp - fm) / (2 * e)
    assert abs(fd - g_tau) <= 1e-6 * max(abs(g_tau), 1e-12) + 1e-10, (fd, g_tau)


def test_adjoint_forward_equals_scheme_forward():
    """The adjoint's recorded forward is the scheme of oracle.scheme (same V)."""
    from oracle import scheme

    prob, conn, d_node, sensors, data, n_steps = _problem(n=10, n_steps=120)
    _, rec = prob.forward(n_steps, sensors, 10)
    sim = scheme.Simulation(prob.K, prob.m, adjoint._cells.MitchellSchaeffer(*prob.ms_params), prob.stimuli)
    vals = []
    for _ in range(n_steps // 10):
        sim.run(10)
        vals.append(sim.S[0][sensors].copy())
    np.testing.assert_allclose(rec["samples"], np.array(vals), rtol=0, atol=1e-14)
