"""Pins of the oracle's time integration (Section 2, Eq. 2, Eq. 3).

Dense brute force on small meshes, closed forms, conservation laws and the
structural statements of Section 2 (k and l rules, reduction to the standard
splitting when dt/2 <= dt_s, merged diffusion halves).
"""
import math

import numpy as np
import pytest
import scipy.linalg

import inputs as I
from oracle import cells, fem, scheme


def _small_aniso(n=5):
    wl = I.tp06_slab_3d(n, n - 1, 4, h=0.02)
    K, m = fem.assemble_grid(3, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
    return wl, K, m


def test_diffusion_substeps_equal_dense_matrix_power():
    wl, K, m = _small_aniso()
    n = K.shape[0]
    assert n <= 100
    rng = np.random.default_rng(1)
    V0 = rng.standard_normal(n)
    sim = scheme.Simulation(K, m, cells.CubicBistable(), dt=0.1)
    sim.S[0] = V0
    sim.diffuse(7)
    A = np.eye(n) - sim.dt_ad * np.diag(1.0 / m) @ K.toarray()
    np.testing.assert_allclose(sim.S[0], np.linalg.matrix_power(A, 7) @ V0, rtol=0, atol=1e-13)


def test_diffusion_converges_to_matrix_exponential():
    wl, K, m = _small_aniso()
    n = K.shape[0]
    rng = np.random.default_rng(2)
    V0 = rng.standard_normal(n)
    T = 0.2
    exact = scipy.linalg.expm(-T * np.diag(1.0 / m) @ K.toarray()) @ V0
    errs = []
    for nsub in (20, 40, 80):
        sim = scheme.Simulation(K, m, cells.CubicBistable(), dt=0.1)
        sim.dt_ad = T / nsub
        sim.S[0] = V0
        sim.diffuse(nsub)
        errs.append(np.abs(sim.S[0] - exact).max())
    # forward Euler: first order
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_gershgorin_bounds_dense_spectrum_and_lambda():
    for wl in (I.tp06_slab_3d(6, 5, 4, h=0.02), I.ms_square_2d(n=9), I.aniso_sheet_2d(n=9, length=0.08)):
        K, m = fem.assemble_workload(wl)
        lam = np.linalg.eigvals(np.diag(1.0 / m) @ K.toarray()).real
        dt_s = scheme.gershgorin_dt(K, m)
        # Gershgorin: every eigenvalue lies below max_i (k_ii + sum |k_ij|) / m_ii = 0.9 / dt_s
        assert lam.max() <= 0.9 / dt_s * (1 + 1e-12)
        assert lam.min() > -1e-10
        assert abs(scheme.lambda_max(K, m) - lam.max()) < 1e-9 * lam.max()
        # Section 2's claim: explicit Euler with dt_ad <= dt_s is stable
        assert dt_s * lam.max() < 2.0


def test_diffusion_conserves_mass_and_uniform_fields():
    wl, K, m = _small_aniso(9)
    rng = np.random.default_rng(3)
    sim = scheme.Simulation(K, m, cells.CubicBistable(), dt=0.1)
    V0 = rng.standard_normal(K.shape[0])
    sim.S[0] = V0.copy()
    sim.diffuse(50)
    assert abs(m @ sim.S[0] - m @ V0) < 1e-13 * np.abs(m @ np.abs(V0))
    sim.S[0] = np.full(K.shape[0], -85.23)
    sim.diffuse(10)
    np.testing.assert_allclose(sim.S[0], -85.23, rtol=0, atol=1e-12)


def test_l_rule_section2_and_section31():
    # Section 3.1: dt = 0.1 ms, dt_s = 0.013 ms -> l = floor(0.1 / 0.026) = 3
    assert scheme.l_rule(0.1, 0.013) == 3
    assert scheme.l_rule(0.1, 0.013, "ceil") == 4
    # dt / 2 <= dt_s: l = 1 (standard splitting)
    assert scheme.l_rule(0.1, 0.05) == 1
    assert scheme.l_rule(0.1, 0.10546875) == 1
    # floor always keeps dt_ad below 2 dt_s (so below 1.8 / lambda_max)
    for dt_s in np.linspace(0.001, 0.05, 200):
        l = scheme.l_rule(0.1, dt_s)
        assert 0.1 / (2 * l) < 2 * dt_s or l == 1


def test_k_rule_section2():
    kmax = scheme.k_max_rule(0.1, 0.01)
    assert kmax == 10
    r = np.array([0.0, -0.0, 1e-12, 0.5, -0.5, -3.7, 4.9, 5.0, -9.2, 100.0, -1e9, 0.999999])
    k = scheme.k_rule(r, kmax)
    np.testing.assert_array_equal(k, [1, 1, 5, 5, 1, 4, 9, 10, 10, 10, 10, 5])
    assert scheme.k_max_rule(0.05, 0.01) == 5 and scheme.k_max_rule(0.01, 0.01) == 1


def test_stimulus_window():
    st = I.Stimulus(np.array([0]), 1.0, 1.0, 1.0, period=10.0, count=2)
    t = np.array([0.99, 1.0, 1.5, 1.99, 2.0, 10.99, 11.0, 11.999, 12.0, 21.0])
    np.testing.assert_array_equal(scheme.stimulus_on(st, t),
                                  [False, True, True, True, False, False, True, True, False, False])


def test_reduces_to_standard_splitting_when_dt_half_below_dt_s():
    # plain 2D square: dt_s = 0.105 ms > dt / 2, so DAETI == OSTAR bit for bit (Section 2)
    wl = I.ms_square_2d(n=15)
    a = scheme.simulation_from_workload(wl, scheme="daeti")
    b = scheme.simulation_from_workload(wl, scheme="ostar")
    assert a.l == b.l == 1 and a.dt == b.dt
    a.run(200)
    b.run(200)
    assert np.array_equal(a.S, b.S) and np.array_equal(a.act, b.act)


def test_merged_diffusion_halves_match_separate_halves():
    """Section 2: steps III and I of consecutive steps combine into one step B of dt.

    The synchronisation between the halves only reads V, so a fused B of 2l
    sub-steps with the synchronisation after sub-step l is the same sequence.
    """
    wl = I.ms_square_2d(n=11)
    a = scheme.simulation_from_workload(wl)
    a.run(12)
    b = scheme.simulation_from_workload(wl)
    b.run(12)
    s_before = a.S.copy()
    a.diffuse(a.l)
    a.n += 1
    a.sync()
    a.diffuse(a.l)
    b.diffuse(2 * b.l)
    assert np.array_equal(a.S, b.S)
    # the synchronisation left the state untouched
    c = scheme.simulation_from_workload(wl)
    c.run(12)
    c.sync()
    assert np.array_equal(c.S, s_before)


def test_activation_interpolation():
    # a node whose sync values go 0.2 -> 0.8 between t = 0.1 and 0.2 crosses 0.5 at 0.15
    K = np.zeros((1, 1))
    sim = scheme.Simulation(K + 1e-300, np.ones(1), cells.CubicBistable(), dt=0.1, v_threshold=0.5)
    sim.n = 2
    sim.v_sync[:] = 0.2
    sim.S[0] = 0.8
    sim.sync()
    assert abs(sim.act[0] - 0.15) < 1e-15
    sim.S[0] = 0.1
    sim.sync()
    sim.S[0] = 0.9
    sim.sync()
    assert abs(sim.act[0] - 0.15) < 1e-15      # first crossing only


def test_k_rules_on_a_linear_cell():
    """dv/dt = J (the cubic model with a_r = 0) on one node without diffusion:
    while the stimulus is on, both readings of 'dV/dt at the previous
    iteration' give 100 J = 3 mV/ms, k = 5 + 3 = 8 (k = 1 at the first step,
    rate 0).  The window ends after 4 of the 8 sub-steps of the step at
    0.5 ms: over that step the split solution rose 4 (0.0125)(0.03), a rate of
    1.5 mV/ms (k = 5 + 1 = 6), while the reaction's rate at the step's last
    sub-step is 0 (k = 1)."""
    ks = {}
    for rule in ("total", "reaction"):
        st = I.Stimulus(np.array([0]), 0.0, 0.55, 0.03)
        sim = scheme.Simulation(np.zeros((1, 1)) + 1e-300, np.ones(1), cells.CubicBistable(a_r=0.0), [st],
                                dt=0.1, dt0=0.01, k_rule=rule)
        seq = []
        for _ in range(7):
            seq.append(int(sim.k[0]))
            sim.step()
        ks[rule] = seq
        assert abs(sim.S[0, 0] - 0.55 * 0.03) < 1e-15
    assert ks["total"] == [1, 8, 8, 8, 8, 8, 6]
    assert ks["reaction"] == [1, 8, 8, 8, 8, 8, 1]


def test_ost_is_fixed_step():
    wl = I.ms_square_2d(n=9)
    a = scheme.simulation_from_workload(wl, scheme="ost", dt=0.01)
    assert a.k_max == 1 and a.l == 1 and a.dt == 0.01
    a.run(5)
    assert (a.k == 1).all()


def test_ostar_step_reduction():
    wl = I.aniso_sheet_2d(n=9, length=0.08, model="ms")        # dt_s = 0.0132 ms
    s = scheme.simulation_from_workload(wl, scheme="ostar")
    assert abs(s.dt - 0.1 / math.ceil(0.1 / s.dt_s)) < 1e-15 and s.dt <= s.dt_s and s.l == 1
    d = scheme.simulation_from_workload(wl, scheme="daeti")
    assert d.l == 3 and abs(d.dt_ad - 0.1 / 6) < 1e-15


def test_s1s2_time_is_the_scan_choice():
    """The tet slab's S2 time is the S2 time of the oracle's 10 ms scan after
    which activity persisted at 1000 ms (tests/golden/s1s2_scan_oracle.json,
    written by make_s1s2_scan.py from oracle runs), and the recorded traces
    show it re-entering: the active-node count falls and rises again."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "s1s2_scan_oracle.json")))
    assert g["s2_with_activity_at_1000ms"] == [int(I.S1S2_S2_TIME)]
    a = np.array(g["runs"][str(int(I.S1S2_S2_TIME))])
    assert a[-1] > 0 and (a[55:] < 0.6 * a[55:].max()).any()
    for s2, trace in g["runs"].items():
        if int(s2) != int(I.S1S2_S2_TIME):
            assert trace[-1] == 0, s2
