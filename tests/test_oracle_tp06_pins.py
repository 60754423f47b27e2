"""Pins of the oracle's ten Tusscher-Panfilov 2006 model by what physics and
mathematics fix (the paper does not contain the model, so its published
traces cannot be compared; see the parity note in oracle/cells.py).

* RT/F of the model's constants equals k_B T / e from the SI values of the
  Boltzmann constant and the elementary charge (an independent route to the
  thermal voltage) to 1e-5 (the model's R and F are an older CODATA
  revision, 1e-6 apart); the reversal potentials below use k_B T / e, so
  "vanishes" means |I(E)| <= 1e-4 of |I(E +- 10 mV)|.
* Every current with a driving force (V - E) vanishes at its own Nernst
  potential computed here from k_B T / e, and has the sign of V - E on either
  side: I_Kr, I_K1, I_to, I_pK at E_K; I_Na, I_bNa at E_Na; I_bCa at E_Ca;
  I_Ks at the Na-permeable E_Ks.
* I_CaL (GHK flux) vanishes where 0.25 CaSS e^x = Cao, x = 2 (V - 15) F/RT,
  inward below and outward above; I_NaCa vanishes at the thermodynamic
  reversal of a 3 Na : 1 Ca exchanger, 3 E_Na - 2 E_Ca, shifted by the
  model's (RT/F) ln(alpha).
* Michaelis-Menten factors: I_NaK is half its saturated value at Nai = KmNa
  and positive at every V; I_pCa is half its maximum at Cai = KpCa.
* Gates: steady states in [0, 1], activation gates non-decreasing and
  inactivation gates non-increasing in V, time constants positive and
  finite over -100..+60 mV, for all three cell types.
* The published initial state is a resting state: the fast gates sit at their
  steady states (within 0.3 %), the net ionic current nearly vanishes
  (|dV/dt| < 0.002 mV/ms while I_K1, I_NaCa, I_NaK, I_bCa, I_bNa and I_pCa are
  0.02-0.31 pA/pF each), and an unstimulated cell stays within 0.5 mV of it
  for 1000 ms.
"""
import numpy as np
import pytest

from oracle import cells

K_B = 1.380649e-23          # J/K (exact in the SI since 2019)
Q_E = 1.602176634e-19       # C (exact)
NAMES = ("m", "h", "j", "xr1", "xr2", "xs", "r", "s", "d", "f", "f2", "fCass")


def _kt_over_e_mv(T):
    return 1e3 * K_B * T / Q_E


def _state(tp, n, **over):
    S = tp.initial_state(n)
    for k, v in over.items():
        S[cells.TP06_STATES.index(k)] = v
    return S


def test_thermal_voltage_from_boltzmann_constant():
    tp = cells.TP06(0)
    assert abs(tp.R * tp.T / tp.F - _kt_over_e_mv(tp.T)) <= 1e-5 * _kt_over_e_mv(tp.T)


@pytest.mark.parametrize("celltype", [0, 1, 2])
def test_currents_vanish_at_their_reversal_potentials(celltype):
    tp = cells.TP06(celltype)
    vt = _kt_over_e_mv(tp.T)
    rng = np.random.default_rng(5)
    for _ in range(5):
        Ki, Nai, Cai = rng.uniform(120, 150), rng.uniform(5, 15), rng.uniform(5e-5, 1e-3)
        gates = dict(m=rng.uniform(0.1, 1), h=rng.uniform(0.1, 1), j=rng.uniform(0.1, 1),
                     xr1=rng.uniform(0.1, 1), xr2=rng.uniform(0.1, 1), xs=rng.uniform(0.1, 1),
                     r=rng.uniform(0.1, 1), s=rng.uniform(0.1, 1))
        E = {"K": vt * np.log(tp.Ko / Ki), "Na": vt * np.log(tp.Nao / Nai), "Ca": 0.5 * vt * np.log(tp.Cao / Cai),
             "Ks": vt * np.log((tp.Ko + tp.pKNa * tp.Nao) / (Ki + tp.pKNa * Nai))}
        which = {"Kr": "K", "K1": "K", "to": "K", "pK": "K", "Na": "Na", "bNa": "Na", "bCa": "Ca", "Ks": "Ks"}
        for cur, e in which.items():
            V = E[e] + np.array([-10.0, 0.0, 10.0])
            S = _state(tp, 3, V=V, Ki=Ki, Nai=Nai, Cai=Cai, **gates)
            I = tp.currents(S)[cur]
            scale = np.abs(I).max()
            assert scale > 0, cur
            assert abs(I[1]) <= 1e-4 * scale, (cur, I)
            assert I[0] < 0 < I[2], (cur, I)


def test_ical_vanishes_at_the_ghk_reversal():
    tp = cells.TP06(0)
    vt = _kt_over_e_mv(tp.T)
    for CaSS in (1e-4, 3.6e-4, 2e-3):
        v_rev = 15.0 + 0.5 * vt * np.log(4.0 * tp.Cao / CaSS)
        V = v_rev + np.array([-5.0, 0.0, 5.0])
        S = _state(tp, 3, V=V, CaSS=CaSS, d=0.8, f=0.9, f2=0.9, fCass=0.9)
        I = tp.currents(S)["CaL"]
        assert abs(I[1]) <= 1e-4 * np.abs(I).max()
        assert I[0] < 0 < I[2]
        # inward over the physiological range
        S = _state(tp, 4, V=np.array([-40.0, 0.0, 15.0, 40.0]), CaSS=CaSS, d=0.8, f=0.9, f2=0.9, fCass=0.9)
        assert (tp.currents(S)["CaL"] < 0).all()


def test_naca_vanishes_at_the_exchanger_reversal():
    tp = cells.TP06(0)
    vt = _kt_over_e_mv(tp.T)
    for Nai, Cai in ((8.6, 1.26e-4), (12.0, 5e-4), (6.0, 2e-4)):
        e_na, e_ca = vt * np.log(tp.Nao / Nai), 0.5 * vt * np.log(tp.Cao / Cai)
        v_rev = 3.0 * e_na - 2.0 * e_ca + vt * np.log(tp.alf)
        S = _state(tp, 3, V=v_rev + np.array([-5.0, 0.0, 5.0]), Nai=Nai, Cai=Cai)
        I = tp.currents(S)["NaCa"]
        assert abs(I[1]) <= 1e-4 * np.abs(I).max()
        assert I[0] < 0 < I[2]


def test_pump_michaelis_menten_factors():
    tp = cells.TP06(0)
    V = np.linspace(-100.0, 60.0, 9)
    half = tp.currents(_state(tp, 9, V=V, Nai=tp.KmNa))["NaK"]
    sat = tp.currents(_state(tp, 9, V=V, Nai=1e12))["NaK"]
    np.testing.assert_allclose(half, 0.5 * sat, rtol=1e-9)
    assert (tp.currents(_state(tp, 9, V=V))["NaK"] > 0).all()
    pca_half = tp.currents(_state(tp, 1, Cai=tp.KpCa))["pCa"]
    assert abs(pca_half[0] - 0.5 * tp.GpCa) <= 1e-12


@pytest.mark.parametrize("celltype", [0, 1, 2])
def test_gates_bounded_monotone_with_positive_time_constants(celltype):
    tp = cells.TP06(celltype)
    V = np.linspace(-100.0, 60.0, 3201)
    inf, tau = tp.gates(V, np.full_like(V, 3.6e-4))
    rising = ("m", "xr1", "xs", "r", "d")
    falling = ("h", "j", "xr2", "s", "f", "f2")
    for name, i, t in zip(NAMES, inf, tau):
        i = np.broadcast_to(i, V.shape)
        t = np.broadcast_to(t, V.shape)
        assert (i >= 0).all() and (i <= 1).all(), name
        assert np.isfinite(t).all() and (t > 0).all(), name
        if name in rising:
            assert (np.diff(i) >= 0).all() and i[-1] - i[0] > 0.5, name
        if name in falling:
            assert (np.diff(i) <= 0).all() and i[0] - i[-1] > 0.5, name
    ca = np.logspace(-5, -1, 200)
    inf_c, tau_c = tp.gates(np.full_like(ca, -80.0), ca)
    assert (np.diff(inf_c[11]) <= 0).all() and (np.diff(tau_c[11]) <= 0).all()
    assert inf_c[11][0] < 1.0 and inf_c[11][-1] > 0.4


@pytest.mark.parametrize("celltype", [0, 1, 2])
def test_published_initial_state_is_a_resting_state(celltype):
    tp = cells.TP06(celltype)
    S = tp.initial_state(1)
    inf, _ = tp.gates(S[0], S[3])
    for g in ("m", "h", "xr2", "r", "s", "d"):
        published = S[cells.TP06_STATES.index(g), 0]
        assert abs(np.ravel(inf[NAMES.index(g)])[0] - published) <= 0.003 * published, g
    I = tp.currents(S)
    for cur in ("K1", "NaCa", "NaK", "bCa", "bNa", "pCa"):
        assert abs(I[cur][0]) > 0.02, cur           # each carries a resting current ...
    assert abs(tp.dvdt(S, np.zeros(1))[0]) < 0.002  # ... and they balance


def test_unstimulated_cells_stay_at_rest_for_1000_ms():
    tp = cells.TP06(np.array([0, 1, 2]))            # the three types side by side
    S = tp.initial_state(3)
    V0 = S[0].copy()
    for _ in range(20000):                           # 1000 ms, Rush-Larsen gates, 0.05 ms steps
        S = tp.substep(S, 0.05, np.zeros(3))
        assert np.abs(S[0] - V0).max() < 0.5
    assert (S[6:18] >= 0).all() and (S[6:18] <= 1).all()
