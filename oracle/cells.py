"""Cell models of the reaction sub-problem (Eq. 2a) and their explicit sub-steps.

Each model holds its state as a (n_states, n_nodes) float64 array, row 0 = V.
``substep(S, dt, J)`` advances every column by one explicit sub-step of length
``dt`` (scalar or per-column array) with the stimulus term J added to dV/dt,
evaluating every right-hand side at the state at the start of the sub-step.
Section 2 integrates the reaction with forward Euler; for the ten
Tusscher-Panfilov model the gating variables use the Rush-Larsen exponential
update (reading R-int) because forward Euler on its fast gates is unstable at
0.1 ms sub-steps.

``vscale`` converts the model's dV/dt to mV/ms for the reaction sub-step rule
of Section 2 (k = k0 + floor(|dV/dt|)): the Mitchell-Schaeffer and cubic
models are normalised (V_mV = 100 v - 80, reading R-MS).
"""
from __future__ import annotations

import numpy as np


class MitchellSchaeffer:
    """Mitchell-Schaeffer two-variable model (v in [0, 1], gate h)."""

    name = "ms"
    n_states = 2
    vscale = 100.0
    state_names = ("v", "h")

    def __init__(self, tau_in=0.3, tau_out=6.0, tau_open=120.0, tau_close=150.0, v_gate=0.13):
        self.tau_in, self.tau_out = float(tau_in), float(tau_out)
        self.tau_open, self.tau_close, self.v_gate = float(tau_open), float(tau_close), float(v_gate)

    def initial_state(self, n):
        S = np.zeros((2, n))
        S[1] = 1.0
        return S

    def rhs(self, S, J):
        v, h = S[0], S[1]
        dv = h * v * v * (1.0 - v) / self.tau_in - v / self.tau_out + J
        dh = np.where(v < self.v_gate, (1.0 - h) / self.tau_open, -h / self.tau_close)
        return dv, dh

    def substep(self, S, dt, J):
        dv, dh = self.rhs(S, J)
        return np.stack([S[0] + dt * dv, S[1] + dt * dh])

    def dvdt(self, S, J):
        """dv/dt of a forward-Euler sub-step from S (model units per ms)."""
        return self.rhs(S, J)[0]


class CubicBistable:
    """Test-only Nagumo model dv/dt = a_r v (1 - v)(v - a) (exact front speed known)."""

    name = "cubic"
    n_states = 1
    vscale = 100.0
    state_names = ("v",)

    def __init__(self, a_r=1.0, a=0.1):
        self.a_r, self.a = float(a_r), float(a)

    def initial_state(self, n):
        return np.zeros((1, n))

    def substep(self, S, dt, J):
        v = S[0]
        return (v + dt * self.dvdt(S, J))[None, :]

    def dvdt(self, S, J):
        v = S[0]
        return self.a_r * v * (1.0 - v) * (v - self.a) + J


# ---------------------------------------------------------------------------
# ten Tusscher & Panfilov (2006) human ventricular model.
# State order (shared convention of the library and the oracle):
TP06_STATES = ("V", "Cai", "CaSR", "CaSS", "Nai", "Ki", "m", "h", "j", "xr1", "xr2", "xs",
               "r", "s", "d", "f", "f2", "fCass", "RR")
# Initial state published with the model (its table of initial values).
TP06_INIT = (-85.23, 0.000126, 3.64, 0.00036, 8.604, 136.89, 0.00172, 0.7444, 0.7045,
             0.00621, 0.4712, 0.0095, 2.42e-8, 0.999998, 3.373e-5, 0.7888, 0.9755, 0.9953,
             0.9073)


class TP06:
    """ten Tusscher-Panfilov 2006; celltype 0 = endo, 1 = epi, 2 = mid-myocardial.

    Units: mV, ms, mM, pA/pF (C = 1 uF/cm^2 per unit area).  The stimulus J
    (mV/ms, added to dV/dt) is carried by K+ (it enters dKi/dt as -I_stim),
    which makes the total charge of the cell an exact invariant of the ODEs.
    The I_CaL factor (V-15)/(exp(2(V-15)F/RT) - 1) is evaluated through
    x / expm1(x) with its limit 1 at x = 0 (removable singularity at 15 mV).

    Parity: unpinned against the model's publication (the paper does not
    contain it).  What pins each part (tests/test_oracle_tp06_pins.py,
    tests/test_oracle_cells.py):

    * constants R, T, F: the thermal voltage k_B T / e from SI constants;
    * ``gates``: steady states in [0, 1] and monotone in V, time constants
      positive and finite (a sign or offset typo in an exponent fails), the
      published resting state holding m, h, xr2, r, s, d at their steady
      states within 0.3 %; the slow gates' time constants only by the AP
      plausibility test (peak, APD90);
    * ``currents``: each (V - E) current vanishes at its Nernst potential
      with the sign of V - E (E_K, E_Na, E_Ca, E_Ks); I_CaL at its GHK zero;
      I_NaCa at 3 E_Na - 2 E_Ca + (RT/F) ln(alf); the I_NaK and I_pCa
      half-saturation points; the resting balance of the published state
      (|dV/dt| < 0.002 mV/ms), which fails for a change of a few per cent in
      GK1, knaca, knak, GbNa, GbCa, GpCa, KmNa, KpCa, alf, Ko or GCaL;
      GNa, GKr, GKs, Gto and GpK (currents that are ~0 at rest) only by the AP
      plausibility test;
    * ``rates``: charge conservation converging with dt (the stoichiometry
      of Na, K and Ca fluxes and the Cm/(V F) factors); the SR and buffer
      constants (Vmaxup, Vrel, Vleak, Vxfer, k1p..., Vc, Vsr, Vss) only by
      the AP plausibility test and the 1000 ms resting drift (< 0.5 mV);
    * ``substep``: the adaptive step A against a 0.004 ms integration
      (self-convergence) and gates kept in [0, 1] through an AP.
    """

    name = "tp06"
    n_states = 19
    vscale = 1.0
    state_names = TP06_STATES

    # physical constants
    R = 8314.472
    T = 310.0
    F = 96485.3415
    Ko, Cao, Nao = 5.4, 2.0, 140.0
    Vc, Vsr, Vss, Cm = 0.016404, 0.001094, 0.00005468, 0.185
    Bufc, Kbufc, Bufsr, Kbufsr, Bufss, Kbufss = 0.2, 0.001, 10.0, 0.3, 0.4, 0.00025
    Vmaxup, Kup, Vrel, Vleak, Vxfer = 0.006375, 0.00025, 0.102, 0.00036, 0.0038
    k1p, k2p, k3, k4, EC, maxsr, minsr = 0.15, 0.045, 0.060, 0.005, 1.5, 2.5, 1.0
    GKr, pKNa, GK1, GNa, GbNa = 0.153, 0.03, 5.405, 14.838, 0.00029
    KmK, KmNa, knak = 1.0, 40.0, 2.724
    GCaL, GbCa = 3.980e-5, 0.000592
    knaca, KmNai, KmCa, ksat, gam, alf = 1000.0, 87.5, 1.38, 0.1, 0.35, 2.5
    GpCa, KpCa, GpK = 0.1238, 0.0005, 0.0146

    def __init__(self, celltype=0):
        # one cell type for every node, or one per node (an integer array:
        # transmural heterogeneity); the published per-type constants either way
        ct = np.asarray(celltype)
        if ct.ndim == 0:
            self.celltype = int(ct)
            self.Gks = 0.098 if self.celltype == 2 else 0.392
            self.Gto = 0.073 if self.celltype == 0 else 0.294
        else:
            self.celltype = ct.astype(np.int64)
            self.Gks = np.where(self.celltype == 2, 0.098, 0.392)
            self.Gto = np.where(self.celltype == 0, 0.073, 0.294)

    def initial_state(self, n):
        return np.tile(np.asarray(TP06_INIT, dtype=np.float64)[:, None], (1, n))

    def for_nodes(self, idx):
        """The model of the node subset idx (per-node types follow their nodes)."""
        if np.ndim(self.celltype) == 0:
            return self
        return TP06(self.celltype[idx])

    # -- gate steady states and time constants --------------------------------
    def gates(self, V, CaSS):
        """(inf, tau) for m, h, j, xr1, xr2, xs, r, s, d, f, f2, fCass."""
        e = np.exp
        hi = V >= -40.0
        m_inf = 1.0 / (1.0 + e((-56.86 - V) / 9.03)) ** 2
        a_m = 1.0 / (1.0 + e((-60.0 - V) / 5.0))
        b_m = 0.1 / (1.0 + e((V + 35.0) / 5.0)) + 0.10 / (1.0 + e((V - 50.0) / 200.0))
        tau_m = a_m * b_m
        h_inf = 1.0 / (1.0 + e((V + 71.55) / 7.43)) ** 2
        a_h = np.where(hi, 0.0, 0.057 * e(-(V + 80.0) / 6.8))
        b_h = np.where(hi, 0.77 / (0.13 * (1.0 + e(-(V + 10.66) / 11.1))),
                       2.7 * e(0.079 * V) + 3.1e5 * e(0.3485 * V))
        tau_h = 1.0 / (a_h + b_h)
        j_inf = h_inf
        a_j = np.where(hi, 0.0, (-2.5428e4 * e(0.2444 * V) - 6.948e-6 * e(-0.04391 * V))
                       * (V + 37.78) / (1.0 + e(0.311 * (V + 79.23))))
        b_j = np.where(hi, 0.6 * e(0.057 * V) / (1.0 + e(-0.1 * (V + 32.0))),
                       0.02424 * e(-0.01052 * V) / (1.0 + e(-0.1378 * (V + 40.14))))
        tau_j = 1.0 / (a_j + b_j)
        xr1_inf = 1.0 / (1.0 + e((-26.0 - V) / 7.0))
        tau_xr1 = (450.0 / (1.0 + e((-45.0 - V) / 10.0))) * (6.0 / (1.0 + e((V + 30.0) / 11.5)))
        xr2_inf = 1.0 / (1.0 + e((V + 88.0) / 24.0))
        tau_xr2 = (3.0 / (1.0 + e((-60.0 - V) / 20.0))) * (1.12 / (1.0 + e((V - 60.0) / 20.0)))
        xs_inf = 1.0 / (1.0 + e((-5.0 - V) / 14.0))
        tau_xs = (1400.0 / np.sqrt(1.0 + e((5.0 - V) / 6.0))) * (1.0 / (1.0 + e((V - 35.0) / 15.0))) + 80.0
        r_inf = 1.0 / (1.0 + e((20.0 - V) / 6.0))
        tau_r = 9.5 * e(-(V + 40.0) ** 2 / 1800.0) + 0.8
        # s gate: endocardial form for type 0, the other form for types 1 and 2
        s_inf_endo = 1.0 / (1.0 + e((V + 28.0) / 5.0))
        tau_s_endo = 1000.0 * e(-(V + 67.0) ** 2 / 1000.0) + 8.0
        s_inf_other = 1.0 / (1.0 + e((V + 20.0) / 5.0))
        tau_s_other = 85.0 * e(-(V + 45.0) ** 2 / 320.0) + 5.0 / (1.0 + e((V - 20.0) / 5.0)) + 3.0
        if np.ndim(self.celltype) == 0:
            s_inf, tau_s = (s_inf_endo, tau_s_endo) if self.celltype == 0 else (s_inf_other, tau_s_other)
        else:
            endo = self.celltype == 0
            s_inf = np.where(endo, s_inf_endo, s_inf_other)
            tau_s = np.where(endo, tau_s_endo, tau_s_other)
        d_inf = 1.0 / (1.0 + e((-8.0 - V) / 7.5))
        tau_d = ((1.4 / (1.0 + e((-35.0 - V) / 13.0)) + 0.25) * (1.4 / (1.0 + e((V + 5.0) / 5.0)))
                 + 1.0 / (1.0 + e((50.0 - V) / 20.0)))
        f_inf = 1.0 / (1.0 + e((V + 20.0) / 7.0))
        tau_f = (1102.5 * e(-(V + 27.0) ** 2 / 225.0) + 200.0 / (1.0 + e((13.0 - V) / 10.0))
                 + 180.0 / (1.0 + e((V + 30.0) / 10.0)) + 20.0)
        f2_inf = 0.67 / (1.0 + e((V + 35.0) / 7.0)) + 0.33
        tau_f2 = (562.0 * e(-(V + 27.0) ** 2 / 240.0) + 31.0 / (1.0 + e((25.0 - V) / 10.0))
                  + 80.0 / (1.0 + e((V + 30.0) / 10.0)))
        q = (CaSS / 0.05) ** 2
        fcass_inf = 0.6 / (1.0 + q) + 0.4
        tau_fcass = 80.0 / (1.0 + q) + 2.0
        inf = (m_inf, h_inf, j_inf, xr1_inf, xr2_inf, xs_inf, r_inf, s_inf, d_inf, f_inf, f2_inf, fcass_inf)
        tau = (tau_m, tau_h, tau_j, tau_xr1, tau_xr2, tau_xs, tau_r, tau_s, tau_d, tau_f, tau_f2, tau_fcass)
        return inf, tau

    # -- currents and concentration rates --------------------------------------
    def currents(self, S):
        V, Cai, CaSR, CaSS, Nai, Ki = S[0], S[1], S[2], S[3], S[4], S[5]
        m, h, j, xr1, xr2, xs, r, s, d, f, f2, fcass, RR = S[6:19]
        RTF = self.R * self.T / self.F
        FRT = 1.0 / RTF
        e = np.exp
        EK = RTF * np.log(self.Ko / Ki)
        ENa = RTF * np.log(self.Nao / Nai)
        EKs = RTF * np.log((self.Ko + self.pKNa * self.Nao) / (Ki + self.pKNa * Nai))
        ECa = 0.5 * RTF * np.log(self.Cao / Cai)
        a_k1 = 0.1 / (1.0 + e(0.06 * (V - EK - 200.0)))
        b_k1 = (3.0 * e(0.0002 * (V - EK + 100.0)) + e(0.1 * (V - EK - 10.0))) / (1.0 + e(-0.5 * (V - EK)))
        xk1 = a_k1 / (a_k1 + b_k1)
        I = {}
        I["Na"] = self.GNa * m ** 3 * h * j * (V - ENa)
        x = 2.0 * (V - 15.0) * FRT
        x_over_expm1 = np.where(np.abs(x) < 1e-12, 1.0 - 0.5 * x, x / np.where(x == 0.0, 1.0, np.expm1(x)))
        # 4 (V-15) F^2/(RT) (0.25 CaSS e^x - Cao)/(e^x - 1) = 2 F (0.25 CaSS e^x - Cao) x/(e^x - 1)
        I["CaL"] = self.GCaL * d * f * f2 * fcass * 2.0 * self.F * (0.25 * CaSS * e(x) - self.Cao) * x_over_expm1
        I["to"] = self.Gto * r * s * (V - EK)
        I["Kr"] = self.GKr * np.sqrt(self.Ko / 5.4) * xr1 * xr2 * (V - EK)
        I["Ks"] = self.Gks * xs * xs * (V - EKs)
        I["K1"] = self.GK1 * np.sqrt(self.Ko / 5.4) * xk1 * (V - EK)
        I["NaCa"] = (self.knaca / ((self.KmNai ** 3 + self.Nao ** 3) * (self.KmCa + self.Cao)
                                   * (1.0 + self.ksat * e((self.gam - 1.0) * V * FRT)))
                     * (e(self.gam * V * FRT) * Nai ** 3 * self.Cao
                        - e((self.gam - 1.0) * V * FRT) * self.Nao ** 3 * Cai * self.alf))
        I["NaK"] = (self.knak * self.Ko / (self.Ko + self.KmK) * Nai / (Nai + self.KmNa)
                    / (1.0 + 0.1245 * e(-0.1 * V * FRT) + 0.0353 * e(-V * FRT)))
        I["pCa"] = self.GpCa * Cai / (self.KpCa + Cai)
        I["pK"] = self.GpK * (V - EK) / (1.0 + e((25.0 - V) / 5.98))
        I["bNa"] = self.GbNa * (V - ENa)
        I["bCa"] = self.GbCa * (V - ECa)
        return I

    def rates(self, S, J):
        """dV/dt, concentration and RR rates (forward-Euler part of the sub-step)."""
        V, Cai, CaSR, CaSS, Nai, Ki = S[0], S[1], S[2], S[3], S[4], S[5]
        RR = S[18]
        I = self.currents(S)
        Iion = (I["Kr"] + I["Ks"] + I["K1"] + I["to"] + I["Na"] + I["bNa"] + I["CaL"] + I["bCa"]
                + I["NaK"] + I["NaCa"] + I["pCa"] + I["pK"])
        dV = -Iion + J
        kcasr = self.maxsr - (self.maxsr - self.minsr) / (1.0 + (self.EC / CaSR) ** 2)
        k1 = self.k1p / kcasr
        k2 = self.k2p * kcasr
        dRR = -k2 * CaSS * RR + self.k4 * (1.0 - RR)
        O = k1 * CaSS ** 2 * RR / (self.k3 + k1 * CaSS ** 2)
        Irel = self.Vrel * O * (CaSR - CaSS)
        Iup = self.Vmaxup / (1.0 + self.Kup ** 2 / Cai ** 2)
        Ileak = self.Vleak * (CaSR - Cai)
        Ixfer = self.Vxfer * (CaSS - Cai)
        bi = 1.0 / (1.0 + self.Bufc * self.Kbufc / (Cai + self.Kbufc) ** 2)
        bsr = 1.0 / (1.0 + self.Bufsr * self.Kbufsr / (CaSR + self.Kbufsr) ** 2)
        bss = 1.0 / (1.0 + self.Bufss * self.Kbufss / (CaSS + self.Kbufss) ** 2)
        dCai = bi * ((Ileak - Iup) * self.Vsr / self.Vc + Ixfer
                     - (I["bCa"] + I["pCa"] - 2.0 * I["NaCa"]) * self.Cm / (2.0 * self.Vc * self.F))
        dCaSR = bsr * (Iup - Irel - Ileak)
        dCaSS = bss * (-I["CaL"] * self.Cm / (2.0 * self.Vss * self.F) + Irel * self.Vsr / self.Vss
                       - Ixfer * self.Vc / self.Vss)
        dNai = -(I["Na"] + I["bNa"] + 3.0 * I["NaK"] + 3.0 * I["NaCa"]) * self.Cm / (self.Vc * self.F)
        dKi = -(I["K1"] + I["to"] + I["Kr"] + I["Ks"] - 2.0 * I["NaK"] + I["pK"] - J) * self.Cm / (self.Vc * self.F)
        return dV, dCai, dCaSR, dCaSS, dNai, dKi, dRR

    def substep(self, S, dt, J, gate_rl=True):
        dV, dCai, dCaSR, dCaSS, dNai, dKi, dRR = self.rates(S, J)
        inf, tau = self.gates(S[0], S[3])
        out = np.empty_like(S)
        out[0] = S[0] + dt * dV
        out[1] = S[1] + dt * dCai
        out[2] = S[2] + dt * dCaSR
        out[3] = S[3] + dt * dCaSS
        out[4] = S[4] + dt * dNai
        out[5] = S[5] + dt * dKi
        for gi in range(12):
            g = S[6 + gi]
            if gate_rl:
                out[6 + gi] = inf[gi] - (inf[gi] - g) * np.exp(-dt / tau[gi])
            else:
                out[6 + gi] = g + dt * (inf[gi] - g) / tau[gi]
        out[18] = S[18] + dt * dRR
        return out

    def dvdt(self, S, J):
        """dV/dt of a sub-step from S (mV/ms)."""
        return self.rates(S, J)[0]

    def total_charge(self, S):
        """Cm V / F minus the cell's ion content (Na, K, buffered Ca): constant along the ODEs."""
        V, Cai, CaSR, CaSS, Nai, Ki = S[0], S[1], S[2], S[3], S[4], S[5]
        ca_i = Cai + self.Bufc * Cai / (Cai + self.Kbufc)
        ca_sr = CaSR + self.Bufsr * CaSR / (CaSR + self.Kbufsr)
        ca_ss = CaSS + self.Bufss * CaSS / (CaSS + self.Kbufss)
        ions = self.Vc * (Nai + Ki) + 2.0 * (self.Vc * ca_i + self.Vsr * ca_sr + self.Vss * ca_ss)
        return self.Cm * V / self.F - ions


def make_model(name, params=(), cell_type=None):
    """cell_type: TP06 type per node (overrides params[0]) or None."""
    if name == "ms":
        return MitchellSchaeffer(*params)
    if name == "tp06":
        if cell_type is not None:
            return TP06(np.asarray(cell_type))
        return TP06(int(params[0]) if len(params) else 0)
    if name == "cubic":
        return CubicBistable(*params)
    raise ValueError(f"unknown cell model {name!r}")
