// Cell models of the reaction sub-problem (Eq. 2a) as per-node register
// code: Mitchell-Schaeffer (forward Euler, the integrator of Section 2) and
// ten Tusscher-Panfilov 2006 (forward Euler for V, concentrations and the RyR
// state; Rush-Larsen for the twelve gates, since forward Euler on its fast
// gates is unstable at 0.1 ms sub-steps).  Every right-hand side of a
// sub-step is evaluated at the state at the start of that sub-step.
#pragma once

#include "common.cuh"

namespace daeti {

struct MSParams {
    double tau_in, tau_out, tau_open, tau_close, v_gate;
};

// One Mitchell-Schaeffer forward-Euler sub-step: v' = h v^2 (1-v)/tau_in -
// v/tau_out + J; h' = (1-h)/tau_open if v < v_gate else -h/tau_close.
template <typename R>
__device__ __forceinline__ void ms_substep(R& v, float* cv, R& h, R dt, R J, R r_in, R r_out,
                                           R r_open, R r_close, R v_gate) {
    R dv = h * v * v * ((R)1 - v) * r_in - v * r_out + J;
    R dh = (v < v_gate) ? ((R)1 - h) * r_open : -h * r_close;
    add_comp(v, cv, dt * dv);
    h += dt * dh;
}

// ------------------------------------------------------------------ TP06
// State order: V, Cai, CaSR, CaSS, Nai, Ki, m, h, j, xr1, xr2, xs, r, s, d,
// f, f2, fCass, RR.  Units mV, ms, mM, pA/pF; the stimulus J (mV/ms) is
// carried by K+.
struct TP06Consts {
    static constexpr double R_ = 8314.472, T_ = 310.0, F_ = 96485.3415;
    static constexpr double Ko = 5.4, Cao = 2.0, Nao = 140.0;
    static constexpr double Vc = 0.016404, Vsr = 0.001094, Vss = 0.00005468, Cm = 0.185;
    static constexpr double Bufc = 0.2, Kbufc = 0.001, Bufsr = 10.0, Kbufsr = 0.3;
    static constexpr double Bufss = 0.4, Kbufss = 0.00025;
    static constexpr double Vmaxup = 0.006375, Kup = 0.00025, Vrel = 0.102;
    static constexpr double Vleak = 0.00036, Vxfer = 0.0038;
    static constexpr double k1p = 0.15, k2p = 0.045, k3 = 0.060, k4 = 0.005;
    static constexpr double EC = 1.5, maxsr = 2.5, minsr = 1.0;
    static constexpr double GKr = 0.153, pKNa = 0.03, GK1 = 5.405, GNa = 14.838, GbNa = 0.00029;
    static constexpr double KmK = 1.0, KmNa = 40.0, knak = 2.724;
    static constexpr double GCaL = 3.980e-5, GbCa = 0.000592;
    static constexpr double knaca = 1000.0, KmNai = 87.5, KmCa = 1.38, ksat = 0.1;
    static constexpr double gam = 0.35, alf = 2.5;
    static constexpr double GpCa = 0.1238, KpCa = 0.0005, GpK = 0.0146;
};

struct TP06Params {
    int celltype;  // 0 endo, 1 epi, 2 mid
    int gate_rl;   // 1 Rush-Larsen, 0 forward Euler gates
};

template <typename R>
struct TP06State {
    R V, Cai, CaSR, CaSS, Nai, Ki, m, h, j, xr1, xr2, xs, r, s, d, f, f2, fcass, RR;
};

// Gate update toward g_inf with time constant tau over dt.
template <typename R>
__device__ __forceinline__ R gate_step(R g, R ginf, R tau, R dt, int rl) {
    typedef Fm<R> M;
    if (rl) return ginf - (ginf - g) * M::ex(-M::dv(dt, tau));
    return g + dt * M::dv(ginf - g, tau);
}

template <typename R>
__device__ __forceinline__ void tp06_substep(TP06State<R>& x, float* cv, R dt, R J,
                                             const TP06Params& prm) {
    typedef TP06Consts C;
    typedef Fm<R> M;
    const R one = (R)1;
    const R RTF = (R)(C::R_ * C::T_ / C::F_);
    const R FRT = (R)(C::F_ / (C::R_ * C::T_));
    const R V = x.V;

    // reversal potentials
    const R EK = RTF * M::lg(M::dv((R)C::Ko, x.Ki));
    const R ENa = RTF * M::lg(M::dv((R)C::Nao, x.Nai));
    const R EKs = RTF * M::lg(M::dv((R)(C::Ko + C::pKNa * C::Nao), x.Ki + (R)C::pKNa * x.Nai));
    const R ECa = (R)0.5 * RTF * M::lg(M::dv((R)C::Cao, x.Cai));

    // inward rectifier
    const R vek = V - EK;
    const R ak1 = M::dv((R)0.1, one + M::ex((R)0.06 * (vek - (R)200)));
    const R bk1 = M::dv((R)3 * M::ex((R)0.0002 * (vek + (R)100)) + M::ex((R)0.1 * (vek - (R)10)),
                        one + M::ex((R)-0.5 * vek));
    const R xk1 = M::dv(ak1, ak1 + bk1);

    const R Gks = prm.celltype == 2 ? (R)0.098 : (R)0.392;
    const R Gto = prm.celltype == 0 ? (R)0.073 : (R)0.294;
    const R sqk = (R)1;  // sqrt(Ko / 5.4) with Ko = 5.4

    const R INa = (R)C::GNa * x.m * x.m * x.m * x.h * x.j * (V - ENa);
    // I_CaL with (V-15)/(exp(2(V-15)F/RT) - 1) written as (RT/2F) x/expm1(x)
    const R xc = (R)2 * (V - (R)15) * FRT;
    const R exc = M::ex(xc);
    R xq;
    if (fabs(xc) < (R)1e-4) {
        xq = one - (R)0.5 * xc + xc * xc * (R)(1.0 / 12.0);
    } else {
        xq = M::dv(xc, M::em1(xc));
    }
    const R ICaL = (R)C::GCaL * x.d * x.f * x.f2 * x.fcass * (R)(2.0 * C::F_) *
                   ((R)0.25 * x.CaSS * exc - (R)C::Cao) * xq;
    const R Ito = Gto * x.r * x.s * vek;
    const R IKr = (R)C::GKr * sqk * x.xr1 * x.xr2 * vek;
    const R IKs = Gks * x.xs * x.xs * (V - EKs);
    const R IK1 = (R)C::GK1 * sqk * xk1 * vek;
    const R e_g = M::ex((R)C::gam * V * FRT);
    const R e_g1 = M::ex((R)(C::gam - 1.0) * V * FRT);
    const R INaCa = M::dv((R)C::knaca * (e_g * x.Nai * x.Nai * x.Nai * (R)C::Cao -
                                         e_g1 * (R)(C::Nao * C::Nao * C::Nao) * x.Cai * (R)C::alf),
                          (R)((C::KmNai * C::KmNai * C::KmNai + C::Nao * C::Nao * C::Nao) *
                              (C::KmCa + C::Cao)) * (one + (R)C::ksat * e_g1));
    const R INaK = M::dv((R)(C::knak * C::Ko / (C::Ko + C::KmK)) * x.Nai,
                         (x.Nai + (R)C::KmNa) *
                             (one + (R)0.1245 * M::ex((R)-0.1 * V * FRT) + (R)0.0353 * M::ex(-V * FRT)));
    const R IpCa = M::dv((R)C::GpCa * x.Cai, (R)C::KpCa + x.Cai);
    const R IpK = M::dv((R)C::GpK * vek, one + M::ex(((R)25 - V) * (R)(1.0 / 5.98)));
    const R IbNa = (R)C::GbNa * (V - ENa);
    const R IbCa = (R)C::GbCa * (V - ECa);

    const R Iion = IKr + IKs + IK1 + Ito + INa + IbNa + ICaL + IbCa + INaK + INaCa + IpCa + IpK;
    const R dV = -Iion + J;

    // calcium handling
    const R ecs = M::dv((R)C::EC, x.CaSR);
    const R kcasr = (R)C::maxsr - M::dv((R)(C::maxsr - C::minsr), one + ecs * ecs);
    const R k1 = M::dv((R)C::k1p, kcasr);
    const R k2 = (R)C::k2p * kcasr;
    const R dRR = -k2 * x.CaSS * x.RR + (R)C::k4 * (one - x.RR);
    const R css2 = x.CaSS * x.CaSS;
    const R O = M::dv(k1 * css2 * x.RR, (R)C::k3 + k1 * css2);
    const R Irel = (R)C::Vrel * O * (x.CaSR - x.CaSS);
    const R kc = M::dv((R)C::Kup, x.Cai);
    const R Iup = M::dv((R)C::Vmaxup, one + kc * kc);
    const R Ileak = (R)C::Vleak * (x.CaSR - x.Cai);
    const R Ixfer = (R)C::Vxfer * (x.CaSS - x.Cai);
    const R ci = x.Cai + (R)C::Kbufc;
    const R csr = x.CaSR + (R)C::Kbufsr;
    const R css = x.CaSS + (R)C::Kbufss;
    const R bi = M::dv(ci * ci, ci * ci + (R)(C::Bufc * C::Kbufc));
    const R bsr = M::dv(csr * csr, csr * csr + (R)(C::Bufsr * C::Kbufsr));
    const R bss = M::dv(css * css, css * css + (R)(C::Bufss * C::Kbufss));
    const R dCai = bi * ((Ileak - Iup) * (R)(C::Vsr / C::Vc) + Ixfer -
                         (IbCa + IpCa - (R)2 * INaCa) * (R)(C::Cm / (2.0 * C::Vc * C::F_)));
    const R dCaSR = bsr * (Iup - Irel - Ileak);
    const R dCaSS = bss * (-ICaL * (R)(C::Cm / (2.0 * C::Vss * C::F_)) + Irel * (R)(C::Vsr / C::Vss) -
                           Ixfer * (R)(C::Vc / C::Vss));
    const R dNai = -(INa + IbNa + (R)3 * INaK + (R)3 * INaCa) * (R)(C::Cm / (C::Vc * C::F_));
    const R dKi = -(IK1 + Ito + IKr + IKs - (R)2 * INaK + IpK - J) * (R)(C::Cm / (C::Vc * C::F_));

    // gates: steady states and time constants at the start-of-sub-step V
    const bool hi = V >= (R)-40;
    const int rl = prm.gate_rl;
    {
        const R em = one + M::ex(((R)-56.86 - V) * (R)(1.0 / 9.03));
        const R minf = M::dv(one, em * em);
        const R am = M::dv(one, one + M::ex(((R)-60 - V) * (R)0.2));
        const R bm = M::dv((R)0.1, one + M::ex((V + (R)35) * (R)0.2)) +
                     M::dv((R)0.1, one + M::ex((V - (R)50) * (R)0.005));
        x.m = gate_step(x.m, minf, am * bm, dt, rl);
    }
    {
        const R eh = one + M::ex((V + (R)71.55) * (R)(1.0 / 7.43));
        const R hinf = M::dv(one, eh * eh);
        R ah, bh, aj, bj;
        if (hi) {
            ah = (R)0;
            bh = M::dv((R)0.77, (R)0.13 * (one + M::ex(-(V + (R)10.66) * (R)(1.0 / 11.1))));
            aj = (R)0;
            bj = M::dv((R)0.6 * M::ex((R)0.057 * V), one + M::ex((R)-0.1 * (V + (R)32)));
        } else {
            ah = (R)0.057 * M::ex(-(V + (R)80) * (R)(1.0 / 6.8));
            bh = (R)2.7 * M::ex((R)0.079 * V) + (R)3.1e5 * M::ex((R)0.3485 * V);
            aj = M::dv(((R)-2.5428e4 * M::ex((R)0.2444 * V) - (R)6.948e-6 * M::ex((R)-0.04391 * V)) *
                           (V + (R)37.78),
                       one + M::ex((R)0.311 * (V + (R)79.23)));
            bj = M::dv((R)0.02424 * M::ex((R)-0.01052 * V), one + M::ex((R)-0.1378 * (V + (R)40.14)));
        }
        x.h = gate_step(x.h, hinf, M::dv(one, ah + bh), dt, rl);
        x.j = gate_step(x.j, hinf, M::dv(one, aj + bj), dt, rl);
    }
    {
        const R inf = M::dv(one, one + M::ex(((R)-26 - V) * (R)(1.0 / 7.0)));
        const R tau = M::dv((R)450, one + M::ex(((R)-45 - V) * (R)0.1)) *
                      M::dv((R)6, one + M::ex((V + (R)30) * (R)(1.0 / 11.5)));
        x.xr1 = gate_step(x.xr1, inf, tau, dt, rl);
    }
    {
        const R inf = M::dv(one, one + M::ex((V + (R)88) * (R)(1.0 / 24.0)));
        const R tau = M::dv((R)3, one + M::ex(((R)-60 - V) * (R)0.05)) *
                      M::dv((R)1.12, one + M::ex((V - (R)60) * (R)0.05));
        x.xr2 = gate_step(x.xr2, inf, tau, dt, rl);
    }
    {
        const R inf = M::dv(one, one + M::ex(((R)-5 - V) * (R)(1.0 / 14.0)));
        const R tau = (R)1400 * M::rsq(one + M::ex(((R)5 - V) * (R)(1.0 / 6.0))) *
                          M::dv(one, one + M::ex((V - (R)35) * (R)(1.0 / 15.0))) +
                      (R)80;
        x.xs = gate_step(x.xs, inf, tau, dt, rl);
    }
    {
        const R inf = M::dv(one, one + M::ex(((R)20 - V) * (R)(1.0 / 6.0)));
        const R v40 = V + (R)40;
        const R tau = (R)9.5 * M::ex(-v40 * v40 * (R)(1.0 / 1800.0)) + (R)0.8;
        x.r = gate_step(x.r, inf, tau, dt, rl);
    }
    {
        R inf, tau;
        if (prm.celltype == 0) {
            inf = M::dv(one, one + M::ex((V + (R)28) * (R)0.2));
            const R v67 = V + (R)67;
            tau = (R)1000 * M::ex(-v67 * v67 * (R)0.001) + (R)8;
        } else {
            inf = M::dv(one, one + M::ex((V + (R)20) * (R)0.2));
            const R v45 = V + (R)45;
            tau = (R)85 * M::ex(-v45 * v45 * (R)(1.0 / 320.0)) +
                  M::dv((R)5, one + M::ex((V - (R)20) * (R)0.2)) + (R)3;
        }
        x.s = gate_step(x.s, inf, tau, dt, rl);
    }
    {
        const R inf = M::dv(one, one + M::ex(((R)-8 - V) * (R)(1.0 / 7.5)));
        const R ad = M::dv((R)1.4, one + M::ex(((R)-35 - V) * (R)(1.0 / 13.0))) + (R)0.25;
        const R bd = M::dv((R)1.4, one + M::ex((V + (R)5) * (R)0.2));
        const R cd = M::dv(one, one + M::ex(((R)50 - V) * (R)0.05));
        x.d = gate_step(x.d, inf, ad * bd + cd, dt, rl);
    }
    {
        const R inf = M::dv(one, one + M::ex((V + (R)20) * (R)(1.0 / 7.0)));
        const R v27 = V + (R)27;
        const R tau = (R)1102.5 * M::ex(-v27 * v27 * (R)(1.0 / 225.0)) +
                      M::dv((R)200, one + M::ex(((R)13 - V) * (R)0.1)) +
                      M::dv((R)180, one + M::ex((V + (R)30) * (R)0.1)) + (R)20;
        x.f = gate_step(x.f, inf, tau, dt, rl);
        const R inf2 = M::dv((R)0.67, one + M::ex((V + (R)35) * (R)(1.0 / 7.0))) + (R)0.33;
        const R tau2 = (R)562 * M::ex(-v27 * v27 * (R)(1.0 / 240.0)) +
                       M::dv((R)31, one + M::ex(((R)25 - V) * (R)0.1)) +
                       M::dv((R)80, one + M::ex((V + (R)30) * (R)0.1));
        x.f2 = gate_step(x.f2, inf2, tau2, dt, rl);
    }
    {
        const R q = x.CaSS * (R)20;  // CaSS / 0.05
        const R den = one + q * q;
        const R inf = M::dv((R)0.6, den) + (R)0.4;
        const R tau = M::dv((R)80, den) + (R)2;
        x.fcass = gate_step(x.fcass, inf, tau, dt, rl);
    }

    // forward Euler for V, concentrations and RR
    add_comp(x.V, cv, dt * dV);
    x.Cai += dt * dCai;
    x.CaSR += dt * dCaSR;
    x.CaSS += dt * dCaSS;
    x.Nai += dt * dNai;
    x.Ki += dt * dKi;
    x.RR += dt * dRR;
}

}  // namespace daeti
