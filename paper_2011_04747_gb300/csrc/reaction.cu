// Step A of Section 2: every node integrates its cell model over dt with k
// explicit sub-steps of dt_ar = dt/k, k fixed for the step (chosen at the
// last synchronisation from dV/dt).  One thread per node, all state in
// registers for the whole step; the node order may come from the k buckets
// so that warps run a uniform number of sub-steps.
#include "cells.cuh"
#include "kernels.h"

namespace daeti {

template <typename R>
struct ReactArgs {
    int n;
    R* V;
    float* C;            // Kahan compensation or null
    R* S;                // states 1.. (state-major, stride ld)
    size_t ld;
    const uint8_t* kk;
    const int* perm;     // null: node = thread
    const unsigned* stim_mask;
    const StimDev* stims;
    int n_stims;
    double dt;
    StepRef step;
    R ms_r_in, ms_r_out, ms_r_open, ms_r_close, ms_vgate;
    TP06Params tp;
};

// Sum of the amplitudes of the stimuli in `mask` that are on at time t.
template <typename R>
__device__ __forceinline__ R stim_current(unsigned mask, const StimDev* stims, double t) {
    R J = (R)0;
    while (mask) {
        int b = __ffs(mask) - 1;
        mask &= mask - 1;
        if (stim_on(stims[b], t)) J += (R)stims[b].amp;
    }
    return J;
}

template <typename R, int MODEL, bool KAHAN>
__global__ void __launch_bounds__(256) reaction_kernel(ReactArgs<R> a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const long long nstep = step_index(a.step);
    const double tn = (double)nstep * a.dt;
    bool any_stim = false;
    for (int s = 0; s < a.n_stims; ++s) any_stim |= stim_overlaps(a.stims[s], tn, tn + a.dt);

    const int i = a.perm ? a.perm[t] : t;
    const int k = a.kk[i];
    const unsigned smask = any_stim ? a.stim_mask[i] : 0u;
    const double dt_ar = a.dt / (double)k;
    const R h = (R)dt_ar;
    float c = KAHAN ? a.C[i] : 0.f;
    float* cp = KAHAN ? &c : nullptr;
    const size_t ld = a.ld;

    if (MODEL == M_MS) {
        R v = a.V[i];
        R g = a.S[i];
        for (int s = 0; s < k; ++s) {
            R J = smask ? stim_current<R>(smask, a.stims, tn + (double)s * dt_ar) : (R)0;
            ms_substep(v, cp, g, h, J, a.ms_r_in, a.ms_r_out, a.ms_r_open, a.ms_r_close, a.ms_vgate);
        }
        a.V[i] = v;
        a.S[i] = g;
    } else {
        TP06State<R> x;
        const R* S = a.S;
        x.V = a.V[i];
        x.Cai = S[0 * ld + i];
        x.CaSR = S[1 * ld + i];
        x.CaSS = S[2 * ld + i];
        x.Nai = S[3 * ld + i];
        x.Ki = S[4 * ld + i];
        x.m = S[5 * ld + i];
        x.h = S[6 * ld + i];
        x.j = S[7 * ld + i];
        x.xr1 = S[8 * ld + i];
        x.xr2 = S[9 * ld + i];
        x.xs = S[10 * ld + i];
        x.r = S[11 * ld + i];
        x.s = S[12 * ld + i];
        x.d = S[13 * ld + i];
        x.f = S[14 * ld + i];
        x.f2 = S[15 * ld + i];
        x.fcass = S[16 * ld + i];
        x.RR = S[17 * ld + i];
        for (int s = 0; s < k; ++s) {
            R J = smask ? stim_current<R>(smask, a.stims, tn + (double)s * dt_ar) : (R)0;
            tp06_substep(x, cp, h, J, a.tp);
        }
        R* W = a.S;
        a.V[i] = x.V;
        W[0 * ld + i] = x.Cai;
        W[1 * ld + i] = x.CaSR;
        W[2 * ld + i] = x.CaSS;
        W[3 * ld + i] = x.Nai;
        W[4 * ld + i] = x.Ki;
        W[5 * ld + i] = x.m;
        W[6 * ld + i] = x.h;
        W[7 * ld + i] = x.j;
        W[8 * ld + i] = x.xr1;
        W[9 * ld + i] = x.xr2;
        W[10 * ld + i] = x.xs;
        W[11 * ld + i] = x.r;
        W[12 * ld + i] = x.s;
        W[13 * ld + i] = x.d;
        W[14 * ld + i] = x.f;
        W[15 * ld + i] = x.f2;
        W[16 * ld + i] = x.fcass;
        W[17 * ld + i] = x.RR;
    }
    if (KAHAN) a.C[i] = c;
}

template <typename R, bool KAHAN>
static void launch_typed(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool use_perm,
                         int buf, int block, cudaStream_t st) {
    ReactArgs<R> a;
    a.n = (int)s.n;
    a.V = (R*)s.V[buf];
    a.C = KAHAN ? s.C[buf] : nullptr;
    a.S = (R*)s.S;
    a.ld = (size_t)s.n;
    a.kk = s.kk;
    a.perm = use_perm ? s.perm : nullptr;
    a.stim_mask = s.stim_mask;
    a.stims = s.stims;
    a.n_stims = s.stim_mask ? s.n_stims : 0;
    a.dt = dt;
    a.step = step;
    a.ms_r_in = (R)(1.0 / m.ms[0]);
    a.ms_r_out = (R)(1.0 / m.ms[1]);
    a.ms_r_open = (R)(1.0 / m.ms[2]);
    a.ms_r_close = (R)(1.0 / m.ms[3]);
    a.ms_vgate = (R)m.ms[4];
    a.tp.celltype = m.celltype;
    a.tp.gate_rl = m.gate_rl;
    if (block <= 0) block = 128;
    int grid = (int)((s.n + block - 1) / block);
    if (grid == 0) return;
    if (m.model == M_MS)
        reaction_kernel<R, M_MS, KAHAN><<<grid, block, 0, st>>>(a);
    else
        reaction_kernel<R, M_TP06, KAHAN><<<grid, block, 0, st>>>(a);
}

void launch_reaction(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool use_perm,
                     int buf, int block, cudaStream_t st) {
    if (s.prec == P_F64)
        launch_typed<double, false>(s, m, dt, step, use_perm, buf, block, st);
    else if (s.kahan)
        launch_typed<float, true>(s, m, dt, step, use_perm, buf, block, st);
    else
        launch_typed<float, false>(s, m, dt, step, use_perm, buf, block, st);
}

}  // namespace daeti
