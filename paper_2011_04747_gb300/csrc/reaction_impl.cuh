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
    R* S;                // states 1.. in chunks of 32 nodes: state s of node i at ((i/32)*ns + s)*32 + i%32
    const uint8_t* kk;
    const int* lists;    // per-k node lists (list k at lists + k*n), null: node = item
    const int* counts;   // list lengths of this step A (counts[k], k >= 1)
    int* counts_next;    // list lengths of the next step A, cleared here; [0] = its bucketing mode
    const int* uflag;    // with mode -K: set if some node's k is not K
    int* uflag_next;     // the same for the next step A, cleared here
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
    const uint8_t* ctype;   // TP06 cell type per node, or null (tp.celltype everywhere)
    R* rrate;               // dV/dt of each node's last sub-step (k rule from the reaction rate), or null
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
// EXT: per-node TP06 cell types and the reaction-rate record are possible
// (compiled out of the plain instance).
template <typename R, int MODEL, bool KAHAN, bool EXT>
__device__ __forceinline__ void react_node(const ReactArgs<R>& a, int i, int k, double tn, bool any_stim, R v0,
                                           float c0) {
    const unsigned smask = any_stim ? a.stim_mask[i] : 0u;
    const double dt_ar = a.dtk[k];     // used in FP64 only for stimulus times
    const R h = a.dtkr[k];
    float c = c0;
    float* cp = KAHAN ? &c : nullptr;
    if (MODEL == M_MS) {
        R v = v0;
        R g = a.S[i];
        for (int s = 0; s < k; ++s) {
            R J = smask ? stim_current<R>(smask, a.stims, tn + (double)s * dt_ar) : (R)0;
            const R dv = ms_substep(v, cp, g, h, J, a.ms_r_in, a.ms_r_out, a.ms_r_open, a.ms_r_close, a.ms_vgate);
            if (EXT && a.rrate && s == k - 1) a.rrate[i] = dv;
        }
        a.V[i] = v;
        a.S[i] = g;
    } else {
        // the node's 18 cell states in its chunk of 32 nodes: base + 32 s
        TP06State<R> x;
        R* const S = a.S + (size_t)(i >> 5) * (18 * 32) + (i & 31);
        x.V = v0;
        x.Cai = S[0 * 32];
        x.CaSR = S[1 * 32];
        x.CaSS = S[2 * 32];
        x.Nai = S[3 * 32];
        x.Ki = S[4 * 32];
        x.m = S[5 * 32];
        x.h = S[6 * 32];
        x.j = S[7 * 32];
        x.xr1 = S[8 * 32];
        x.xr2 = S[9 * 32];
        x.xs = S[10 * 32];
        x.r = S[11 * 32];
        x.s = S[12 * 32];
        x.d = S[13 * 32];
        x.f = S[14 * 32];
        x.f2 = S[15 * 32];
        x.fcass = S[16 * 32];
        x.RR = S[17 * 32];
        TP06Params tp = a.tp;
        if (EXT && a.ctype) tp.celltype = a.ctype[i];
        if (tp.gate_rl) {
            for (int s = 0; s < k; ++s) {
                R J = smask ? stim_current<R>(smask, a.stims, tn + (double)s * dt_ar) : (R)0;
                const R dv = tp06_substep<R, true>(x, cp, h, J, tp);
                if (EXT && a.rrate && s == k - 1) a.rrate[i] = dv;
            }
        } else {
            for (int s = 0; s < k; ++s) {
                R J = smask ? stim_current<R>(smask, a.stims, tn + (double)s * dt_ar) : (R)0;
                const R dv = tp06_substep<R, false>(x, cp, h, J, tp);
                if (EXT && a.rrate && s == k - 1) a.rrate[i] = dv;
            }
        }
        a.V[i] = x.V;
        S[0 * 32] = x.Cai;
        S[1 * 32] = x.CaSR;
        S[2 * 32] = x.CaSS;
        S[3 * 32] = x.Nai;
        S[4 * 32] = x.Ki;
        S[5 * 32] = x.m;
        S[6 * 32] = x.h;
        S[7 * 32] = x.j;
        S[8 * 32] = x.xr1;
        S[9 * 32] = x.xr2;
        S[10 * 32] = x.xs;
        S[11 * 32] = x.r;
        S[12 * 32] = x.s;
        S[13 * 32] = x.d;
        S[14 * 32] = x.f;
        S[15 * 32] = x.f2;
        S[16 * 32] = x.fcass;
        S[17 * 32] = x.RR;
    }
    if (KAHAN) a.C[i] = c;
}

// Node of item t.  Buckets are laid out largest k first: bucket k holds the
// items off[k] <= t < off[k-1], with off[k] = sum of the lengths of buckets
// j > k non-increasing in k and off[j] = 0 for j >= kmax, so k is the
// smallest j >= 1 with off[j] <= t (branch-free binary search over 1..15).
__device__ __forceinline__ int item_node(const int* __restrict__ lists, int n, const int* off, int t, int& k) {
    int lo = 0;   // off[lo] > t holds for lo = 0 (t < total = off[0])
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1)
        if (off[lo + step] > t) lo += step;
    k = lo + 1;
    return lists[(size_t)k * n + (t - off[k])];
}

// One item: the optional fused diffusion sub-step, then step A of node i.
template <typename R, int MODEL, bool KAHAN, int DIM, bool PAD, bool EXT>
__device__ __forceinline__ void react_item(const ReactArgs<R>& a, const OpView<R>& op, int i, int k, double tn,
                                           bool any_stim) {
    R v0;
    float c0 = 0.f;
    if (DIM >= 0) {
        diffuse_node<R, (DIM < 0 ? 0 : DIM), KAHAN, PAD, EXT>(op, a.vsrc, a.csrc, i, v0, c0);
    } else {
        v0 = a.V[i];
        if (KAHAN) c0 = a.C[i];
    }
    react_node<R, MODEL, KAHAN, EXT>(a, i, k, tn, any_stim, v0, c0);
}

// Items are the entries of the per-k lists taken largest k first (list
// kmax, ..., list 1), one per thread, so that every warp but those at list
// boundaries runs one uniform sub-step count.  Item-warp u goes to warp
// u / gridDim.x of block u % gridDim.x, so the few heavy (large k) warps at
// the head of the list land on different SMs instead of a handful of
// blocks.  MINB caps registers (minimum resident blocks of 128 threads) to
// trade spills against occupancy.  DIM >= 0 fuses one diffusion sub-step
// before the reaction (0: SELL-32, 2/3: stencil; PAD: V buffers with a ghost
// margin, no per-neighbour boundary tests).
template <typename R, int MODEL, bool KAHAN, int MINB, int DIM, bool PAD, bool EXT>
__global__ void __launch_bounds__(128, MINB) reaction_kernel(ReactArgs<R> a, OpView<R> op) {
    __shared__ int off[DAETI_MAX_K];
    __shared__ double sh_tn;
    __shared__ int sh_stim;
    __shared__ int sh_uni;
    __shared__ int sh_listed;
    __shared__ int sh_total;
    pdl_wait();
    pdl_trigger();
    // Warp 0: step time, stimulus window and list offsets, with the loads of
    // the step counter, the stimuli and the list lengths in flight together.
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const double t0 = a.n_stims ? (double)step_index(a.step) * a.dt : 0.0;   // only stimuli need it
        const bool on = lane < a.n_stims && stim_overlaps(a.stims[lane], t0, t0 + a.dt);
        const unsigned any = __ballot_sync(0xffffffffu, on);
        const int c = (a.lists && lane >= 1 && lane <= a.kmax) ? a.counts[lane] : 0;
        // inclusive suffix sum of the bucket lengths c over lanes 0..15:
        // off[k] = sum of c_j, j > k; off[0] = total number of items
        int sfx = c;
#pragma unroll
        for (int d = 1; d < DAETI_MAX_K; d <<= 1) {
            const int y = __shfl_down_sync(0xffffffffu, sfx, d);
            if (lane + d < DAETI_MAX_K) sfx += y;
        }
        if (lane < DAETI_MAX_K) off[lane] = sfx - c;
        // Bucketing mode of this step (counts[0], chosen by the previous step
        // A): 1 = lists built, counts valid; -K = k expected to be K at every
        // node, confirmed unless *uflag is set.  uni = the k every node has,
        // else 0.
        const int mode = a.lists ? a.counts[0] : 1;
        const int uflag = a.lists ? *a.uflag : 0;   // loaded with the mode, not after it
        const int broken = mode < 0 ? uflag : 0;
        const unsigned full = __ballot_sync(0xffffffffu, c == a.n && c > 0);
        const int uni = mode < 0 ? (broken ? 0 : -mode) : (full ? __ffs(full) - 1 : 0);
        const int listed_total = __shfl_sync(0xffffffffu, sfx, 0);
        if (lane == 0) {
            sh_tn = t0;
            sh_stim = any != 0u;
            sh_uni = uni;
            sh_listed = mode > 0;
            sh_total = mode < 0 ? a.n : listed_total;
        }
        if (a.lists && blockIdx.x == 0) {
            // next step's mode: expect this step's uniform k again, else lists
            if (lane < DAETI_MAX_K) a.counts_next[lane] = lane == 0 ? (uni ? -uni : 1) : 0;
            if (lane == 0) *a.uflag_next = 0;
            if (a.substeps && (mode > 0 || uni)) {
                unsigned long long tot = mode > 0 ? (unsigned long long)lane * (unsigned long long)c : 0ull;
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, d);
                if (mode < 0) tot = (unsigned long long)a.n * (unsigned long long)uni;
                if (lane == 0) atomicAdd(a.substeps, tot);
            }
        }
    }
    __syncthreads();
    const double tn = sh_tn;
    const bool any_stim = sh_stim != 0;
    if (!a.lists) {
        // no bucketing: node t with its own k (the sub-step count summed per warp)
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        const int kt = t < a.n ? (int)a.kk[t] : 0;
        if (a.substeps) {
            unsigned long long w = (unsigned long long)kt;
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
            if ((threadIdx.x & 31) == 0 && w) atomicAdd(a.substeps, w);
        }
        if (t < a.n) react_item<R, MODEL, KAHAN, DIM, PAD, EXT>(a, op, t, kt, tn, any_stim);
        return;
    }
    const int total = sh_total;
    const int t = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
    if (sh_uni) {
        // every node has the same k (common away from wavefronts): item t is
        // node t, no list indirection
        if (t < total) react_item<R, MODEL, KAHAN, DIM, PAD, EXT>(a, op, t, sh_uni, tn, any_stim);
    } else if (!sh_listed) {
        // k became mixed after a step with the same k everywhere, so no lists
        // were built: item t is node t with its own k (and the sub-step count
        // is summed here)
        const int kt = t < total ? (int)a.kk[t] : 0;
        if (a.substeps) {
            unsigned long long w = (unsigned long long)kt;
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
            if ((threadIdx.x & 31) == 0 && w) atomicAdd(a.substeps, w);
        }
        if (t < total) react_item<R, MODEL, KAHAN, DIM, PAD, EXT>(a, op, t, kt, tn, any_stim);
    } else if (t < total) {
        int k;
        const int i = item_node(a.lists, a.n, off, t, k);
        react_item<R, MODEL, KAHAN, DIM, PAD, EXT>(a, op, i, k, tn, any_stim);
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
    a.kk = s.kk;
    a.lists = lists ? s.lists : nullptr;
    a.counts = s.counts + par * DAETI_MAX_K;
    a.counts_next = s.counts + (1 - par) * DAETI_MAX_K;
    a.uflag = s.flags + 2 + par;
    a.uflag_next = s.flags + 2 + (1 - par);
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
    a.ctype = s.ctype;
    a.rrate = (R*)s.rrate;
    return a;
}

template <typename R, int MODEL, bool KAHAN, int MINB, int DIM, bool PAD = false, bool EXT = false>
void launch_react_one(const ReactArgs<R>& a, const OpView<R>& op, int grid, int block, bool pdl, cudaStream_t st) {
    launch_ex(reaction_kernel<R, MODEL, KAHAN, MINB, DIM, PAD, EXT>, grid, block, st, pdl, a, op);
}

// The extended instances (per-node operator rows, per-node cell types or the
// reaction-rate k rule), with 8 resident blocks per SM whatever the tuning.
template <typename R, int MODEL, bool KAHAN>
void launch_react_ext(const ReactArgs<R>& a, const OpView<R>& op, const DiffOp& dop, bool fused, bool pad, int grid,
                      int block, bool pdl, cudaStream_t st) {
    if (!fused) launch_react_one<R, MODEL, KAHAN, 8, -1, false, true>(a, op, grid, block, pdl, st);
    else if (dop.kind == 1) launch_react_one<R, MODEL, KAHAN, 8, 0, false, true>(a, op, grid, block, pdl, st);
    else if (dop.dim == 2 && pad) launch_react_one<R, MODEL, KAHAN, 8, 2, true, true>(a, op, grid, block, pdl, st);
    else if (dop.dim == 2) launch_react_one<R, MODEL, KAHAN, 8, 2, false, true>(a, op, grid, block, pdl, st);
    else if (pad) launch_react_one<R, MODEL, KAHAN, 8, 3, true, true>(a, op, grid, block, pdl, st);
    else launch_react_one<R, MODEL, KAHAN, 8, 3, false, true>(a, op, grid, block, pdl, st);
}

// Launch of one (model, precision, register cap) over the four operator cases.
template <typename R, int MODEL, bool KAHAN, int MINB>
void launch_react_dims(const ReactArgs<R>& a, const DevState& s, const DiffOp& dop, bool fused, int grid, int block,
                       const ReactTuning& tune, cudaStream_t st) {
    const OpView<R> op = op_view<R>(dop);
    const bool pdl = tune.pdl != 0;
    const bool pad = s.vpad >= stencil_reach(dop);
    if (s.ctype || s.rrate || dop.per_node) {
        launch_react_ext<R, MODEL, KAHAN>(a, op, dop, fused, pad, grid, block, pdl, st);
        return;
    }
    if (!fused) launch_react_one<R, MODEL, KAHAN, MINB, -1>(a, op, grid, block, pdl, st);
    else if (dop.kind == 1) launch_react_one<R, MODEL, KAHAN, MINB, 0>(a, op, grid, block, pdl, st);
    else if (dop.dim == 2 && pad) launch_react_one<R, MODEL, KAHAN, MINB, 2, true>(a, op, grid, block, pdl, st);
    else if (dop.dim == 2) launch_react_one<R, MODEL, KAHAN, MINB, 2>(a, op, grid, block, pdl, st);
    else if (pad) launch_react_one<R, MODEL, KAHAN, MINB, 3, true>(a, op, grid, block, pdl, st);
    else launch_react_one<R, MODEL, KAHAN, MINB, 3>(a, op, grid, block, pdl, st);
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
