"""Pins of the oracle's cell models and reaction sub-stepping (Section 2, step A).

Mitchell-Schaeffer: closed-form threshold, upper fixed point and APD
asymptote.  Cubic bistable model in a strip: exact front speed of the split
scheme's continuum limit.  TP06: parity unpinned against its publication;
pinned by charge conservation, gate bounds, consistency of its fast-gate
steady states with its published initial state, and fine-step convergence.
"""
import math

import numpy as np
import pytest

import inputs as I
from oracle import cells, metrics, scheme


def _run_cell(model, S, dt, T, J=lambda t: 0.0):
    t = 0.0
    out = [S[0, 0]]
    for _ in range(int(round(T / dt))):
        S = model.substep(S, dt, np.array([J(t)]))
        t += dt
        out.append(S[0, 0])
    return S, np.array(out)


def test_ms_threshold_closed_form():
    ms = cells.MitchellSchaeffer()
    vth = 0.5 * (1.0 - math.sqrt(1.0 - 4.0 * ms.tau_in / ms.tau_out))   # root of h v(1-v)/tau_in = 1/tau_out
    for v0, fires in ((vth - 0.002, False), (vth + 0.002, True)):
        S = np.array([[v0], [1.0]])
        _, tr = _run_cell(ms, S, 0.002, 80.0)
        assert (tr.max() > 0.5) == fires


def test_ms_plateau_fold_and_apd_asymptote():
    """Plateau on the upper branch v*(h), h decaying with tau_close, fold at h = 4 tau_in / tau_out."""
    ms = cells.MitchellSchaeffer()
    S = np.array([[0.0], [1.0]])
    dt = 0.002
    t, hs, vs = 0.0, [], []
    for _ in range(int(400.0 / dt)):
        S = ms.substep(S, dt, np.array([0.5 if t < 1.0 else 0.0]))
        t += dt
        vs.append(S[0, 0])
        hs.append(S[1, 0])
    vs, hs = np.array(vs), np.array(hs)

    def v_star(h):
        return 0.5 * (1.0 + math.sqrt(1.0 - 4.0 * ms.tau_in / (h * ms.tau_out)))

    up = np.argmax(vs > ms.v_gate)
    for t_pl in (50.0, 100.0, 150.0):
        i = up + int(t_pl / dt)
        assert abs(vs[i] - v_star(hs[i])) < 0.005
        # h decays exactly as exp(-t / tau_close) while v > v_gate
        assert abs(hs[i] / hs[up + int(20.0 / dt)] - math.exp(-(t_pl - 20.0) / ms.tau_close)) < 1e-3
    peak = up + int(np.argmax(vs[up:]))
    fold = peak + np.argmax(vs[peak:] < 0.5)      # the branches meet at v = 1/2
    h_min = 4.0 * ms.tau_in / ms.tau_out
    assert 0.7 * h_min < hs[fold] <= h_min
    down = up + np.argmax(vs[up:] < ms.v_gate)
    apd = (down - up) * dt
    apd_asym = ms.tau_close * math.log(ms.tau_out / (4.0 * ms.tau_in))
    assert abs(apd_asym - 241.4) < 0.1
    # the asymptote is the leading-order term; the slow passage through the fold adds delay
    assert apd_asym < apd < 1.25 * apd_asym


def test_ms_adaptive_k_matches_fine_reference():
    """Step A with the k rule converges to a fine RK4 integration of the same ODE."""
    ms = cells.MitchellSchaeffer()
    # fine RK4 reference with the stimulus
    def f(S, t):
        J = 0.5 if t < 1.0 - 1e-12 else 0.0
        dv, dh = ms.rhs(S, np.array([J]))
        return np.stack([dv, dh])
    S = np.array([[0.0], [1.0]])
    dtf, T = 5e-3, 300.0
    ref = [0.0]
    t = 0.0
    for _ in range(int(T / dtf)):
        k1 = f(S, t); k2 = f(S + 0.5 * dtf * k1, t + 0.5 * dtf)
        k3 = f(S + 0.5 * dtf * k2, t + 0.5 * dtf); k4 = f(S + dtf * k3, t + dtf)
        S = S + dtf / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dtf
        ref.append(S[0, 0])
    ref = np.array(ref)
    # one-node "tissue" (no diffusion) through the Simulation's step A
    sim = scheme.Simulation(np.zeros((1, 1)) + 1e-300, np.ones(1), ms,
                            stimuli=[I.Stimulus(np.array([0]), 0.0, 1.0, 0.5)], dt=0.1, v_threshold=0.5)
    trace = [0.0]
    for _ in range(int(T / 0.1)):
        sim.step()
        trace.append(sim.S[0, 0])
    trace = np.array(trace)
    t_ref = np.arange(len(ref)) * dtf
    t_sim = np.arange(len(trace)) * 0.1
    up_ref = np.interp(0.5, ref[:600], t_ref[:600])
    assert abs(sim.act[0] - up_ref) < 0.1
    # voltage aligned on the upstroke agrees closely through the plateau and repolarisation
    dv = metrics.aligned_max_dv(t_sim, trace, np.interp(t_sim, t_ref, ref), sim.act[0], up_ref)
    assert dv * 100.0 < 5.0      # mV


def test_cubic_front_speed_closed_form():
    """Split scheme on the Nagumo strip converges to c = sqrt(a_r D / 2)(1 - 2a)."""
    errs = []
    for h, dt in ((0.01, 0.02), (0.005, 0.01)):
        wl = I.cubic_strip_2d(h=h, dt=dt, t_end=60.0)
        sim = scheme.simulation_from_workload(wl)
        sim.run(int(round(wl.t_end / dt)))
        nx = wl.n[0]
        x = np.arange(nx) * h
        sel = (x > 0.4) & (x < 0.8)
        c = metrics.conduction_velocity(x[sel], sim.act[:nx][sel])
        a_r, a = wl.model_params
        exact = math.sqrt(a_r * 0.001 / 2.0) * (1.0 - 2.0 * a)
        errs.append(abs(c - exact) / exact)
    assert errs[1] < 0.03
    assert errs[1] < errs[0]


def test_tp06_fast_gate_steady_states_match_published_initial_state():
    """At the published resting V, the fast gates sit at their steady states."""
    tp = cells.TP06(1)
    S = tp.initial_state(1)
    inf, _ = tp.gates(S[0], S[3])
    names = ("m", "h", "j", "xr1", "xr2", "xs", "r", "s", "d", "f", "f2", "fCass")
    for g in ("m", "h", "xr2", "r", "d", "s"):
        i = names.index(g)
        published = S[cells.TP06_STATES.index(g), 0]
        assert abs(inf[i][0] - published) <= 0.01 * published, g


def test_tp06_charge_conservation_converges():
    tp = cells.TP06(0)
    drifts = []
    for dt in (0.02, 0.01):
        S = tp.initial_state(1)
        q0 = tp.total_charge(S)[0]
        S, _ = _run_cell(tp, S, dt, 200.0, J=lambda t: 30.0 if t < 2.0 else 0.0)
        drifts.append(abs(tp.total_charge(S)[0] - q0) / abs(q0))
    assert drifts[1] < 2e-6
    assert 1.6 < drifts[0] / drifts[1] < 2.4


def test_tp06_action_potential_plausible_and_gates_bounded():
    tp = cells.TP06(0)
    S = tp.initial_state(1)
    dt = 0.02
    t = 0.0
    tr = []
    for _ in range(int(600 / dt)):
        S = tp.substep(S, dt, np.array([52.0 if t < 1.0 else 0.0]))
        t += dt
        tr.append(S[0, 0])
        assert (S[6:18] >= 0).all() and (S[6:18] <= 1).all()
    tr = np.array(tr)
    assert 25.0 < tr.max() < 50.0
    amp = tr.max() - tr[0]
    up = np.argmax(tr > -40.0)
    down = up + 50 + np.argmax(tr[up + 50:] < tr.max() - 0.9 * amp)
    apd90 = (down - up) * dt
    assert 250.0 < apd90 < 330.0
    assert abs(tr[-1] - (-85.23)) < 1.5


def test_tp06_ical_removable_singularity():
    tp = cells.TP06(0)
    S = tp.initial_state(3)
    S[0] = [15.0 - 1e-7, 15.0, 15.0 + 1e-7]
    S[14] = 0.5                         # d gate open
    ical = tp.currents(S)["CaL"]
    assert np.isfinite(ical).all()
    assert abs(ical[1] - 0.5 * (ical[0] + ical[2])) < 1e-9 * abs(ical[1])


def test_tp06_adaptive_k_converges_to_fine_step():
    """A TP06 node through the adaptive step A approaches a 0.001 ms integration."""
    tp = cells.TP06(0)
    stim = I.Stimulus(np.array([0]), 0.0, 2.0, 30.0)
    sim = scheme.Simulation(np.zeros((1, 1)) + 1e-300, np.ones(1), tp, stimuli=[stim], dt=0.1,
                            v_threshold=-40.0)
    tr = [sim.S[0, 0]]
    for _ in range(3200):
        sim.step()
        tr.append(sim.S[0, 0])
    S = tp.initial_state(1)
    dtf = 0.004
    _, fine = _run_cell(tp, S, dtf, 320.0, J=lambda t: 30.0 if t < 2.0 - 1e-12 else 0.0)
    t_f = np.arange(len(fine)) * dtf
    up_f = np.interp(-40.0, fine[:1500], t_f[:1500])
    assert abs(sim.act[0] - up_f) < 0.3
    t_s = np.arange(len(tr)) * 0.1
    dv = metrics.aligned_max_dv(t_s, np.array(tr), np.interp(t_s, t_f, fine), sim.act[0], up_f)
    assert dv < 8.0


def test_tp06_per_node_cell_types_match_each_type_alone():
    """Transmural heterogeneity: a per-node type array integrates every node as
    the model of that node's type alone (the reaction is local to the node),
    the three types give three different action potentials, and an array of
    one type equals the scalar model."""
    types = np.array([0, 1, 2, 2, 0, 1])
    mixed = cells.TP06(types)
    alone = [cells.TP06(int(t)) for t in types]
    S = mixed.initial_state(len(types))
    Ss = [m.initial_state(1) for m in alone]
    dt = 0.1
    gap = np.zeros(3)                      # largest V difference of type pairs (0,1), (0,2), (1,2)
    for step in range(3500):
        J = np.full(len(types), 52.0 if step * dt < 1.0 else 0.0)
        S = mixed.substep(S, dt, J)
        for q, m in enumerate(alone):
            Ss[q] = m.substep(Ss[q], dt, J[q:q + 1])
        v = S[0]
        gap = np.maximum(gap, np.abs([v[0] - v[1], v[0] - v[2], v[1] - v[2]]))
        assert abs(v[0] - v[4]) < 1e-9 and abs(v[1] - v[5]) < 1e-9 and abs(v[2] - v[3]) < 1e-9
    for q in range(len(types)):
        assert np.allclose(S[:, q], Ss[q][:, 0], rtol=1e-12, atol=1e-12)
    assert gap.min() > 5.0                 # the three types repolarise differently
    one = cells.TP06(np.zeros(3, dtype=np.int64))
    S1, S0 = one.initial_state(3), cells.TP06(0).initial_state(3)
    for _ in range(50):
        S1 = one.substep(S1, 0.1, np.full(3, 52.0))
        S0 = cells.TP06(0).substep(S0, 0.1, np.full(3, 52.0))
    assert np.allclose(S1, S0, rtol=1e-14, atol=0.0)

