// Step A of Section 2 (implementation shared by the reaction translation
// units): every node integrates its cell model over dt with k explicit
// sub-steps of dt_ar = dt/k, k fixed for the step (chosen at the last
// synchronisation from dV/dt).  One thread per node, all state in registers
// for the whole step.  Nodes are taken from the per-k lists, largest k first,
// so warps run uniform sub-step counts.  Optionally the launch first applies
// the last diffusion sub-step of step I to the node (from the V field of the
// previous launch), so that step I's last sub-step and step II cost one
// launch.
#pragma once

#include "cells.cuh"
#include "diffops.cuh"

namespace daeti {

template <typename R>
struct ReactArgs {
    int n;
    R* V;                // V of this step A (written; also read when no diffusion is fused)
    float* C;            // Kahan compensation or null
    const R* vsrc;       // fused diffusion: V before the sub-step (other buffer)
    const float* csrc;
    R* S;                // states 1.. (state-major, stride ld)
    size_t ld;
    const uint8_t* kk;
    const int* lists;    // per-k node lists (list k at lists + k*n), null: node = item
    const int* counts;   // list lengths of this step A
    int* counts_next;    // list lengths of the next step A, cleared here
    unsigned long long* substeps;
    int kmax;
    const unsigned* stim_mask;
    const StimDev* stims;
    int n_stims;
    double dt;
    double dtk[DAETI_MAX_K];   // dt / k, computed on the host (no FP64 division per node)
    R dtkr[DAETI_MAX_K];       // the same in the state precision
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

// Integrate the k sub-steps of one node (state loaded, advanced, stored).
template <typename R, int MODEL, bool KAHAN>
__device__ __forceinline__ void react_node(const ReactArgs<R>& a, int i, int k, double tn, bool any_stim, R v0,
                                           float c0) {
    const unsigned smask = any_stim ? a.stim_mask[i] : 0u;
    const double dt_ar = a.dtk[k];     // used in FP64 only for stimulus times
    const R h = a.dtkr[k];
    float c = c0;
    float* cp = KAHAN ? &c : nullptr;
    const size_t ld = a.ld;
    if (MODEL == M_MS) {
        R v = v0;
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
        x.V = v0;
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

// One item per thread.  Items are taken largest k first (list kmax, ...,
// list 1), so that every warp but those at the list boundaries runs one
// uniform sub-step count.  MINB caps registers (minimum resident blocks of
// 128 threads) to trade spills against occupancy.  DIM >= 0 fuses one
// diffusion sub-step before the reaction (0: SELL-32, 2/3: stencil).
template <typename R, int MODEL, bool KAHAN, int MINB, int DIM>
__global__ void __launch_bounds__(128, MINB) reaction_kernel(ReactArgs<R> a, OpView<R> op) {
    __shared__ int off[DAETI_MAX_K];
    __shared__ int cnt[DAETI_MAX_K];
    __shared__ double sh_tn;
    __shared__ int sh_stim;
    // step time and stimulus window once per block (FP64 is slow on this part)
    if (threadIdx.x == 0) {
        const double t0 = (double)step_index(a.step) * a.dt;
        int on = 0;
        for (int s = 0; s < a.n_stims; ++s) on |= stim_overlaps(a.stims[s], t0, t0 + a.dt) ? 1 : 0;
        sh_tn = t0;
        sh_stim = on;
    }
    if (threadIdx.x < DAETI_MAX_K)
        cnt[threadIdx.x] = (a.lists && threadIdx.x >= 1 && threadIdx.x <= a.kmax) ? a.counts[threadIdx.x] : 0;
    __syncthreads();
    const double tn = sh_tn;
    const bool any_stim = sh_stim != 0;
    int total = a.n;
    if (a.lists) {
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int k = DAETI_MAX_K - 1; k >= 1; --k) {
                off[k] = acc;
                acc += cnt[k];
            }
            off[0] = acc;
        }
        if (blockIdx.x == 0 && threadIdx.x < DAETI_MAX_K) a.counts_next[threadIdx.x] = 0;
        if (blockIdx.x == 0 && threadIdx.x == 32 && a.substeps) {
            unsigned long long tot = 0;
            for (int k = 1; k < DAETI_MAX_K; ++k) tot += (unsigned long long)k * cnt[k];
            atomicAdd(a.substeps, tot);
        }
        __syncthreads();
        total = off[0];
    }
    // Item warps are dealt to blocks round-robin (item warp u = j * gridDim.x +
    // block, j the warp within the block), so the few heavy (large k) warps at
    // the head of the list land on different SMs instead of a handful of blocks.
    const int u = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int t = a.lists ? u * 32 + (threadIdx.x & 31) : blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total) {
        int i, k;
        if (a.lists) {
            // buckets are laid out largest k first: walk down to the one holding t
            k = a.kmax;
            while (k > 1 && t >= off[k] + cnt[k]) --k;
            i = a.lists[(size_t)k * a.n + (t - off[k])];
        } else {
            i = t;
            k = a.kk[i];
        }
        R v0;
        float c0 = 0.f;
        if (DIM >= 0) {
            diffuse_node<R, (DIM < 0 ? 0 : DIM), KAHAN>(op, a.vsrc, a.csrc, i, v0, c0);
        } else {
            v0 = a.V[i];
            if (KAHAN) c0 = a.C[i];
        }
        react_node<R, MODEL, KAHAN>(a, i, k, tn, any_stim, v0, c0);
    }
}

template <typename R, bool KAHAN>
ReactArgs<R> react_args(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par,
                        int src, bool fused, const ReactTuning& tune) {
    ReactArgs<R> a;
    const int dst = fused ? 1 - src : src;
    a.n = (int)s.n;
    a.V = (R*)s.V[dst];
    a.C = KAHAN ? s.C[dst] : nullptr;
    a.vsrc = (const R*)s.V[src];
    a.csrc = KAHAN ? s.C[src] : nullptr;
    a.S = (R*)s.S;
    a.ld = (size_t)s.n;
    a.kk = s.kk;
    a.lists = lists ? s.lists : nullptr;
    a.counts = s.counts + par * DAETI_MAX_K;
    a.counts_next = s.counts + (1 - par) * DAETI_MAX_K;
    a.substeps = s.substeps;
    a.kmax = tune.kmax;
    a.stim_mask = s.stim_mask;
    a.stims = s.stims;
    a.n_stims = s.stim_mask ? s.n_stims : 0;
    a.dt = dt;
    for (int k = 0; k < DAETI_MAX_K; ++k) {
        a.dtk[k] = k > 0 ? dt / (double)k : dt;
        a.dtkr[k] = (R)a.dtk[k];
    }
    a.step = step;
    a.ms_r_in = (R)(1.0 / m.ms[0]);
    a.ms_r_out = (R)(1.0 / m.ms[1]);
    a.ms_r_open = (R)(1.0 / m.ms[2]);
    a.ms_r_close = (R)(1.0 / m.ms[3]);
    a.ms_vgate = (R)m.ms[4];
    a.tp.celltype = m.celltype;
    a.tp.gate_rl = m.gate_rl;
    return a;
}

// Launch of one (model, precision, register cap) over the four operator cases.
template <typename R, int MODEL, bool KAHAN, int MINB>
void launch_react_dims(const ReactArgs<R>& a, const DiffOp& dop, bool fused, int grid, int block, cudaStream_t st) {
    const OpView<R> op = op_view<R>(dop);
    if (!fused) reaction_kernel<R, MODEL, KAHAN, MINB, -1><<<grid, block, 0, st>>>(a, op);
    else if (dop.kind == 1) reaction_kernel<R, MODEL, KAHAN, MINB, 0><<<grid, block, 0, st>>>(a, op);
    else if (dop.dim == 2) reaction_kernel<R, MODEL, KAHAN, MINB, 2><<<grid, block, 0, st>>>(a, op);
    else reaction_kernel<R, MODEL, KAHAN, MINB, 3><<<grid, block, 0, st>>>(a, op);
}

// Per-TU entry points (explicitly instantiated in reaction_*.cu).
template <typename R, bool KAHAN>
void launch_tp06(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par, int src,
                 bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st);
template <typename R, bool KAHAN>
void launch_ms(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par, int src,
               bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st);

inline int react_block(const ReactTuning& t) {
    int b = t.block > 0 ? t.block : 128;
    return b > 128 ? 128 : b;
}

}  // namespace daeti
