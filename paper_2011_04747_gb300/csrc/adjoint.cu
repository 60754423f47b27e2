// Discrete adjoint of the split step (Section 2's scheme, Mitchell-Schaeffer
// cells, structured grids with isotropic per-element D): gradients of
//   L = sum_j sum_s (v_s(t_j) - d_js)^2
// with respect to the element conductivities D_e and tau_close, for the
// schedule the forward run chose (k per node and step, gate branch per
// sub-step; these discrete choices are held fixed).
//
// Reverse sweep per step (costate of v kept as mu = M_L^-1 lambda while it
// crosses diffusion, because (I - dt_ad M^-1 K)^T = M (I - dt_ad M^-1 K) M^-1
// for symmetric K: the transposed sub-step is the forward sub-step on mu):
//   step III^T: for each sub-step, dL/dD_e += -dt_ad mu_out^T K_e v_in, mu <- D mu
//   step II^T : per node, the k forward-Euler sub-steps are recomputed in
//               registers and reversed (reaction Jacobian-transpose products),
//               dL/dtau_close accumulated
//   step I^T  : as step III^T.
// States are recomputed from device checkpoints placed by a binomial
// (revolve-type) schedule: with s free slots and t steps, the next checkpoint
// goes d = max(1, t - C(s-1+r, s-1)) steps ahead, r the least repetition
// number with C(s+r, s) >= t.  A save or a restore costs no launch of its
// own: the next forward step's combined diffusion-reaction launch writes
// the step-start state of each node to the slot (save), or takes V, h and k
// from the slot and copies its vsync and activation times to the live state
// (restore).  The whole sweep is one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cells.cuh"
#include "context.h"
#include "diffops.cuh"

using namespace daeti_host;

struct AdjointBuffers {
    int64_t n = 0, n_elem = 0, n_steps_hist = 0;
    int n_slots = 0, l = 0, n_sensors = 0, n_samples = 0;
    bool kahan = false;
    int prec = 0;
    std::vector<void*> allocs;
    // snapshots: V, C, h, vsync, act, kk per slot
    std::vector<void*> sV, sC, sH, sVs, sA, sK;
    std::vector<int64_t> slot_step;
    // per-step intermediates: the forward of a step being reversed writes every
    // sub-step's result to its own buffer (pools P, CP), so no copies are needed
    std::vector<void*> P;               // 2l + 1 V buffers
    std::vector<float*> CP;             // 2l + 1 Kahan buffers (FP32 + Kahan)
    void* Hout = nullptr;               // reaction output h (the state h is its input)
    uint8_t* kk_next = nullptr;         // k written by the synchronisation of that step
    std::vector<const void*> d1, d2;    // inputs of the diffusion sub-steps (aliases)
    const void *rv = nullptr, *rh = nullptr, *vend = nullptr;
    const float* rc = nullptr;
    const uint8_t* kused = nullptr;
    // costate and gradients
    void* mu[2] = {nullptr, nullptr};
    void* lamh = nullptr;
    void* mR = nullptr;                  // lumped mass in the state precision
    double* g_elem = nullptr;
    double* acc = nullptr;               // [0] loss, [1] dL/dtau_close
    int* sensors = nullptr;
    void* data = nullptr;
    // recorded schedule
    uint8_t* hist_k = nullptr;
    uint16_t* hist_b = nullptr;
    // the whole gradient sweep as one CUDA graph (the binomial schedule is
    // fixed by n_steps, n_slots and the sampling), keyed by those and the start step
    cudaGraphExec_t graph = nullptr;
    int64_t gkey[5] = {-1, -1, -1, -1, -1};
};

namespace daeti_host {
void drop_adjoint_graph(daeti_ctx* c) {
    if (c->adj && c->adj->graph) {
        cudaGraphExecDestroy(c->adj->graph);
        c->adj->graph = nullptr;
    }
}

void free_adjoint(daeti_ctx* c) {
    if (!c->adj) return;
    if (c->adj->graph) cudaGraphExecDestroy(c->adj->graph);
    for (void* p : c->adj->allocs) cudaFree(p);
    delete c->adj;
    c->adj = nullptr;
}
}  // namespace daeti_host

namespace {

// --------------------------------------------------------------- kernels
template <typename R>
struct AdjReactArgs {
    int n;
    R* V;
    float* C;
    R* H;
    R* Vo;        // outputs (equal to the inputs for in-place steps)
    float* Co;
    R* Ho;
    const uint8_t* kk;
    uint8_t* hist_k;
    uint16_t* hist_b;
    const unsigned* stim_mask;
    const StimDev* stims;
    int n_stims;
    double t_n, dt;
    double dtk[DAETI_MAX_K];
    R dtkr[DAETI_MAX_K];
    R r_in, r_out, r_open, r_close, vgate;
};

template <typename R>
__device__ __forceinline__ R adj_stim(unsigned mask, const StimDev* stims, double t) {
    R J = (R)0;
    while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        if (stim_on(stims[b], t)) J += (R)stims[b].amp;
    }
    return J;
}

// Step A of the adjoint's forward at node i on (v, c): MODE 0 decide, 1 decide
// and record, 2 replay.  h is read from a.H and written to a.Ho.
template <typename R, bool KAHAN, int MODE>
__device__ __forceinline__ void react_node(const AdjReactArgs<R>& a, int i, R& v, float& c) {
    const int k = MODE == 2 ? a.hist_k[i] : a.kk[i];
    const unsigned smask = a.n_stims ? a.stim_mask[i] : 0u;
    const uint16_t rb = MODE == 2 ? a.hist_b[i] : 0;
    R h = a.H[i];
    float* cp = KAHAN ? &c : nullptr;
    uint16_t bits = 0;
    for (int s = 0; s < k; ++s) {
        const R J = smask ? adj_stim<R>(smask, a.stims, a.t_n + (double)s * a.dtk[k]) : (R)0;
        const bool low = MODE == 2 ? ((rb >> s) & 1) != 0 : v < a.vgate;
        bits |= (uint16_t)(low ? 1u << s : 0u);
        ms_substep_b(v, cp, h, a.dtkr[k], J, a.r_in, a.r_out, a.r_open, a.r_close, low);
    }
    a.Ho[i] = h;
    if (MODE == 1) {
        a.hist_k[i] = (uint8_t)k;
        a.hist_b[i] = bits;
    }
}

// Checkpoint traffic carried by the first forward launch after a save or a
// restore, node by node.  Save: the step-start state (v0, c0, a.H, a.kk and the
// live vs, act) is copied to the slot arrays s*.  Restore: the launch reads V,
// the compensation, h and k from the slot directly, and copies the slot's
// vsync and activation times (rVs, rA) to the live vs, act before the
// synchronising sub-step reads them.
template <typename R>
struct CkSide {
    R *sV = nullptr, *sH = nullptr, *sVs = nullptr, *sA = nullptr;
    float* sC = nullptr;
    uint8_t* sK = nullptr;
    const R* v0 = nullptr;
    const float* c0 = nullptr;
    const R *rVs = nullptr, *rA = nullptr;
    R *vs = nullptr, *act = nullptr;
};

// The last step-I diffusion sub-step and step A in one launch: node i's
// diffused value feeds its own reaction directly.  With vmid the diffused
// value (the reaction's input) is stored as well.
template <typename R, bool KAHAN, int MODE, int DIM>
__global__ void __launch_bounds__(128) adj_diff_react_fwd(OpView<R> op, AdjReactArgs<R> a, const R* __restrict__ vin,
                                                          const float* __restrict__ cin, R* vmid, float* cmid,
                                                          CkSide<R> ck) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (ck.sV) {
        ck.sV[i] = ck.v0[i];
        if (KAHAN) ck.sC[i] = ck.c0[i];
        ck.sH[i] = a.H[i];
        ck.sK[i] = a.kk[i];
        ck.sVs[i] = ck.vs[i];
        ck.sA[i] = ck.act[i];
    }
    if (ck.rVs) {
        ck.vs[i] = ck.rVs[i];
        ck.act[i] = ck.rA[i];
    }
    R v;
    float c;
    diffuse_node<R, DIM, KAHAN, false, true>(op, vin, cin, i, v, c);
    if (!KAHAN) c = 0.f;
    if (vmid) {
        vmid[i] = v;
        if (KAHAN) cmid[i] = c;
    }
    react_node<R, KAHAN, MODE>(a, i, v, c);
    a.Vo[i] = v;
    if (KAHAN) a.Co[i] = c;
}

// Reverse of step A at node i: recompute the sub-steps from the stored input
// (rv, rc, rh), then transpose them on the costate (mu_i = lambda_v / m_i and
// lamh[i]).  Returns the new mu_i; gn gets the node's dL/dtau_close share.
template <typename R, bool KAHAN>
__device__ __forceinline__ R react_bwd_node(const AdjReactArgs<R>& a, int i, const R* __restrict__ rv,
                                            const float* __restrict__ rc, const R* __restrict__ rh,
                                            const uint8_t* __restrict__ kused, R mu_i, R* lamh,
                                            const R* __restrict__ m, R& gn) {
    const int k = kused[i];
    const unsigned smask = a.n_stims ? a.stim_mask[i] : 0u;
    R vs[DAETI_MAX_K], hs[DAETI_MAX_K];
    bool lows[DAETI_MAX_K];
    R v = rv[i], h = rh[i];
    float c = KAHAN ? rc[i] : 0.f;
    float* cp = KAHAN ? &c : nullptr;
    const R dt = a.dtkr[k];
#pragma unroll 1
    for (int s = 0; s < k; ++s) {
        const R J = smask ? adj_stim<R>(smask, a.stims, a.t_n + (double)s * a.dtk[k]) : (R)0;
        const bool low = v < a.vgate;
        vs[s] = v;
        hs[s] = h;
        lows[s] = low;
        ms_substep_b(v, cp, h, dt, J, a.r_in, a.r_out, a.r_open, a.r_close, low);
    }
    const R mi = m[i];
    R lv = mu_i * mi;
    R lh = lamh[i];
    // this node's share of dL/dtau_close in the state precision (at most
    // k_max terms), added to the double block sum once
    const R tau_fac = dt * a.r_close * a.r_close;
    gn = (R)0;
#pragma unroll 1
    for (int s = k - 1; s >= 0; --s) {
        const R vi = vs[s], hi = hs[s];
        const R fv = hi * ((R)2 * vi - (R)3 * vi * vi) * a.r_in - a.r_out;
        const R fh = vi * vi * ((R)1 - vi) * a.r_in;
        const R gh = lows[s] ? -a.r_open : -a.r_close;
        if (!lows[s]) gn += lh * hi * tau_fac;
        const R nlv = ((R)1 + dt * fv) * lv;
        lh = dt * fh * lv + ((R)1 + dt * gh) * lh;
        lv = nlv;
    }
    lamh[i] = lh;
    return lv / mi;
}

template <typename R>
struct KrefR {
    R k[64];
};

// dL/dD_e += -dt_ad mu_out^T K_e v_in on element e of a structured grid (the
// element product in the state precision, the sum over steps in double).
template <typename R>
__device__ __forceinline__ void elem_dgrad(int64_t e, int dim, int nx, int ny, const R* __restrict__ mu,
                                           const R* __restrict__ vin, double dt_ad, const KrefR<R>& kr, double* g) {
    const int ex = (int)(e % (nx - 1));
    const int64_t t = e / (nx - 1);
    const int ey = (int)(t % (ny - 1));
    const int ez = (int)(t / (ny - 1));
    const int nl = 1 << dim;
    int node[8];
    for (int a = 0; a < nl; ++a)
        node[a] = (ex + (a & 1)) + nx * ((ey + ((a >> 1) & 1)) + ny * (ez + ((a >> 2) & 1)));
    R s = (R)0;
    for (int a = 0; a < nl; ++a) {
        R r = (R)0;
        for (int b = 0; b < nl; ++b) r = fma(kr.k[a * nl + b], vin[node[b]], r);
        s = fma(mu[node[a]], r, s);
    }
    g[e] += -dt_ad * (double)s;
}

// One transposed diffusion sub-step on the costate, mu_out = (I - dt_ad M^-1 K) mu_in
// (thread t: node t), and in the same launch the element products of that
// sub-step (thread t: element t); both read mu_in only.
template <typename R, int DIM>
__global__ void __launch_bounds__(256) adj_mu_dgrad(OpView<R> op, int n, const R* __restrict__ mu_in,
                                                    R* __restrict__ mu_out, int64_t n_elem, int dim, int nx,
                                                    int ny, const R* __restrict__ vin, double dt_ad, KrefR<R> kr,
                                                    double* g) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) {
        R v;
        float cc;
        diffuse_node<R, DIM, false, false, true>(op, mu_in, nullptr, (int)t, v, cc);
        mu_out[t] = v;
    }
    if (t < n_elem) elem_dgrad<R>(t, dim, nx, ny, mu_in, vin, dt_ad, kr, g);
}

// As adj_mu_dgrad for the first sub-step of step III, followed at each node by
// the reverse of its step A (which needs only that node's costate).
template <typename R, bool KAHAN, int DIM>
__global__ void __launch_bounds__(256) adj_mu_react_bwd(OpView<R> op, AdjReactArgs<R> a, const R* __restrict__ mu_in,
                                                        R* __restrict__ mu_out, int64_t n_elem, int dim, int nx,
                                                        int ny, const R* __restrict__ vin, double dt_ad, KrefR<R> kr,
                                                        double* g, const R* __restrict__ rv,
                                                        const float* __restrict__ rc, const R* __restrict__ rh,
                                                        const uint8_t* __restrict__ kused, R* lamh,
                                                        const R* __restrict__ m, double* g_tau) {
    __shared__ double red[32];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double gt = 0.0;
    if (t < a.n) {
        R v, gn;
        float cc;
        diffuse_node<R, DIM, false, false, true>(op, mu_in, nullptr, (int)t, v, cc);
        mu_out[t] = react_bwd_node<R, KAHAN>(a, (int)t, rv, rc, rh, kused, v, lamh, m, gn);
        gt = (double)gn;
    }
    if (t < n_elem) elem_dgrad<R>(t, dim, nx, ny, mu_in, vin, dt_ad, kr, g);
    for (int o = 16; o > 0; o >>= 1) gt += __shfl_xor_sync(0xffffffffu, gt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gt;
    __syncthreads();
    if (threadIdx.x < 32) {
        gt = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) gt += __shfl_xor_sync(0xffffffffu, gt, o);
        if (threadIdx.x == 0 && gt != 0.0) atomicAdd(g_tau, gt);
    }
}

template <typename R>
__global__ void adj_loss_inject(int n_s, const int* __restrict__ sensors, const R* __restrict__ v,
                                const R* __restrict__ d, const R* __restrict__ m, R* mu, double* loss, int inject) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int q = threadIdx.x; q < n_s; q += blockDim.x) {
        const int i = sensors[q];
        const double r = (double)v[i] - (double)d[q];
        acc += r * r;
        if (inject) mu[i] += (R)(2.0 * r) / m[i];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) loss[0] += acc;
    }
}

// Checkpoint save / restore: up to six arrays copied in one launch, each in
// the widest word (16, 8, 4 or 1 bytes) its addresses and length allow.
struct CopyList {
    void* dst[6];
    const void* src[6];
    int64_t words[6];
    int width[6];
    int n;
};

template <typename W>
__device__ __forceinline__ void copy_words(void* d, const void* s, int64_t n, int64_t t, int64_t stride) {
    W* dw = (W*)d;
    const W* sw = (const W*)s;
    for (int64_t i = t; i < n; i += stride) dw[i] = sw[i];
}

__global__ void adj_copy_arrays(CopyList L) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int q = 0; q < L.n; ++q) {
        switch (L.width[q]) {
            case 16: copy_words<uint4>(L.dst[q], L.src[q], L.words[q], t, stride); break;
            case 8: copy_words<uint2>(L.dst[q], L.src[q], L.words[q], t, stride); break;
            case 4: copy_words<unsigned>(L.dst[q], L.src[q], L.words[q], t, stride); break;
            default: copy_words<uint8_t>(L.dst[q], L.src[q], L.words[q], t, stride); break;
        }
    }
}

// --------------------------------------------------------------- host side
struct CopyBuilder {
    CopyList L{};
    int64_t max_words = 0;
    void add(void* dst, const void* src, size_t bytes) {
        if (!dst || !src || !bytes) return;
        const uintptr_t a = (uintptr_t)dst | (uintptr_t)src | (uintptr_t)bytes;
        const int w = (a & 15) == 0 ? 16 : (a & 7) == 0 ? 8 : (a & 3) == 0 ? 4 : 1;
        const int q = L.n++;
        L.dst[q] = dst;
        L.src[q] = src;
        L.width[q] = w;
        L.words[q] = (int64_t)(bytes / (size_t)w);
        max_words = std::max(max_words, L.words[q]);
    }
    void launch(cudaStream_t st) const {
        if (!L.n) return;
        const int64_t blocks = std::min<int64_t>((max_words + 255) / 256, 4 * 152);
        adj_copy_arrays<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(L);
    }
};

template <typename R>
AdjReactArgs<R> react_args(daeti_ctx* c, int buf, int64_t step, uint8_t* hk, uint16_t* hb) {
    AdjReactArgs<R> a;
    a.n = (int)c->n_nodes;
    a.V = (R*)c->s.V[buf];
    a.C = c->s.kahan ? c->s.C[buf] : nullptr;
    a.H = (R*)c->s.S;
    a.Vo = a.V;
    a.Co = a.C;
    a.Ho = a.H;
    a.kk = c->s.kk;
    a.hist_k = hk;
    a.hist_b = hb;
    a.stim_mask = c->s.stim_mask;
    a.stims = c->s.stims;
    a.n_stims = c->s.stim_mask ? c->s.n_stims : 0;
    a.dt = c->dt_eff;
    a.t_n = (double)step * c->dt_eff;
    for (int k = 0; k < DAETI_MAX_K; ++k) {
        a.dtk[k] = k ? c->dt_eff / k : c->dt_eff;
        a.dtkr[k] = (R)a.dtk[k];
    }
    a.r_in = (R)(1.0 / c->margs.ms[0]);
    a.r_out = (R)(1.0 / c->margs.ms[1]);
    a.r_open = (R)(1.0 / c->margs.ms[2]);
    a.r_close = (R)(1.0 / c->margs.ms[3]);
    a.vgate = (R)c->margs.ms[4];
    return a;
}

struct Adj {
    daeti_ctx* c;
    AdjointBuffers* b;
    cudaStream_t st;
    int64_t n0;          // absolute step index of the adjoint's step 0
    int sample_every;
    int mode;            // 0 decide, 1 record, 2 replay
    int mu_cur = 0;
    int64_t fwd_steps = 0;
    int live_slot = -1;  // checkpoint slot the live state stands for (-1: none)
    // Saves and restores are carried out by the next forward step's combined
    // diffusion-reaction launch (CkSide); pend_save / pend_restore name the slot.
    int pend_save = -1, pend_restore = -1;
    size_t R() const { return rsize(c); }

    void copy_state(bool to_slot, int slot) {
        const size_t N = c->n_nodes, r = R();
        void* live[6] = {c->s.V[c->cur], b->kahan ? (void*)c->s.C[c->cur] : nullptr, c->s.S, c->s.vsync, c->s.act, c->s.kk};
        void* sl[6] = {b->sV[slot], b->kahan ? b->sC[slot] : nullptr, b->sH[slot], b->sVs[slot], b->sA[slot],
                       b->sK[slot]};
        const size_t bytes[6] = {N * r, N * 4, N * r, N * r, N * r, N};
        CopyBuilder cb;
        for (int q = 0; q < 6; ++q) cb.add(to_slot ? sl[q] : live[q], to_slot ? live[q] : sl[q], bytes[q]);
        cb.launch(st);
    }
    // Carry out pending copies with a copy launch (where no forward step follows).
    void flush() {
        if (pend_save >= 0) copy_state(true, pend_save);
        if (pend_restore >= 0) copy_state(false, pend_restore);
        pend_save = pend_restore = -1;
    }
    void save(int slot, int64_t step) {
        flush();
        pend_save = slot;
        b->slot_step[slot] = step;
        live_slot = slot;
    }
    // The binomial recursion restores a checkpoint right after saving it; the
    // live state then still stands for it and nothing is done.
    void restore(int slot) {
        if (live_slot == slot) return;
        flush();
        pend_restore = slot;
        live_slot = slot;
    }

    // The last step-I diffusion sub-step (vin, cin -> the reaction's input,
    // stored to vmid, cmid when given) and step A of step j in one launch;
    // h and k from hin, kin; ck: the pending checkpoint copy.
    template <typename T, bool K>
    void diff_react(int64_t j, const void* vin, const float* cin, void* vmid, float* cmid, void* vout, float* cout,
                    void* hout, const void* hin, const uint8_t* kin, int save_slot, int restore_slot) {
        const int n = (int)c->n_nodes;
        uint8_t* hk = b->hist_k ? b->hist_k + (size_t)j * n : nullptr;
        uint16_t* hb = b->hist_b ? b->hist_b + (size_t)j * n : nullptr;
        AdjReactArgs<T> a = react_args<T>(c, c->cur, n0 + j, hk, hb);
        a.V = nullptr;
        a.C = nullptr;
        a.H = (T*)const_cast<void*>(hin);
        a.kk = kin;
        a.Vo = (T*)vout;
        a.Co = cout;
        a.Ho = (T*)hout;
        CkSide<T> ck;
        ck.vs = (T*)c->s.vsync;
        ck.act = (T*)c->s.act;
        if (save_slot >= 0) {
            ck.sV = (T*)b->sV[save_slot];
            ck.sC = b->kahan ? (float*)b->sC[save_slot] : nullptr;
            ck.sH = (T*)b->sH[save_slot];
            ck.sVs = (T*)b->sVs[save_slot];
            ck.sA = (T*)b->sA[save_slot];
            ck.sK = (uint8_t*)b->sK[save_slot];
            ck.v0 = (const T*)c->s.V[c->cur];
            ck.c0 = b->kahan ? c->s.C[c->cur] : nullptr;
        }
        if (restore_slot >= 0) {
            ck.rVs = (const T*)b->sVs[restore_slot];
            ck.rA = (const T*)b->sA[restore_slot];
        }
        const int dim = c->op.kind == 1 ? 0 : c->op.dim;
        if (dim == 0) diff_react_dim<T, K, 0>(a, vin, cin, vmid, cmid, ck);
        else if (dim == 2) diff_react_dim<T, K, 2>(a, vin, cin, vmid, cmid, ck);
        else diff_react_dim<T, K, 3>(a, vin, cin, vmid, cmid, ck);
    }
    template <typename T, bool K, int DIM>
    void diff_react_dim(const AdjReactArgs<T>& a, const void* vin, const float* cin, void* vmid, float* cmid,
                        const CkSide<T>& ck) {
        const OpView<T> op = op_view<T>(c->op);
        const int grid = (a.n + 127) / 128;
        const T* vi = (const T*)vin;
        T* vm = (T*)vmid;
        if (mode == 2) adj_diff_react_fwd<T, K, 2, DIM><<<grid, 128, 0, st>>>(op, a, vi, cin, vm, cmid, ck);
        else if (mode == 1) adj_diff_react_fwd<T, K, 1, DIM><<<grid, 128, 0, st>>>(op, a, vi, cin, vm, cmid, ck);
        else adj_diff_react_fwd<T, K, 0, DIM><<<grid, 128, 0, st>>>(op, a, vi, cin, vm, cmid, ck);
    }
    void diff_react_any(int64_t j, const void* vin, const float* cin, void* vmid, float* cmid, void* vout,
                        float* cout, void* hout, const void* hin, const uint8_t* kin, int sv, int rs) {
        if (c->s.prec == P_F64)
            diff_react<double, false>(j, vin, nullptr, vmid, nullptr, vout, nullptr, hout, hin, kin, sv, rs);
        else if (c->s.kahan) diff_react<float, true>(j, vin, cin, vmid, cmid, vout, cout, hout, hin, kin, sv, rs);
        else diff_react<float, false>(j, vin, nullptr, vmid, nullptr, vout, nullptr, hout, hin, kin, sv, rs);
    }

    // One diffusion sub-step from `in` to `out` (and the Kahan terms), with the
    // synchronisation epilogue when `sync` (k written to `kk_out`).
    void diffuse_view(const void* in, void* out, const float* cin, float* cout, bool sync, StepRef ref,
                      uint8_t* kk_out) {
        DevState v = c->s;
        v.vpad = 0;
        v.V[0] = const_cast<void*>(in);
        v.V[1] = out;
        v.C[0] = const_cast<float*>(cin);
        v.C[1] = cout;
        if (kk_out) v.kk = kk_out;
        launch_diffusion(v, c->op, 0, sync, 0, c->sargs, ref, false, 256, st);
    }

    // One forward step j (from the synchronisation at t_j).  With `store`, every
    // sub-step writes a fresh buffer so that all intermediates the reverse of
    // this step needs stay in place (the state itself is restored from a
    // checkpoint afterwards).  A pending restore makes the step read its
    // start state from the slot; a pending save is written by its combined
    // launch (with l >= 3 and no store, the step-I sub-steps before that
    // launch overwrite the live V, so the save is copied first).
    void fwd_step(int64_t j, bool store) {
        const StepRef ref{nullptr, (long long)(n0 + j)};
        const int l = c->l;
        if (pend_save >= 0 && !store && l >= 3) {
            copy_state(true, pend_save);
            pend_save = -1;
        }
        const int sv = pend_save, rs = pend_restore;
        pend_save = pend_restore = -1;
        live_slot = -1;
        const void* v0 = rs >= 0 ? b->sV[rs] : c->s.V[c->cur];
        const float* c0 = b->kahan ? (rs >= 0 ? (const float*)b->sC[rs] : c->s.C[c->cur]) : nullptr;
        const void* h0 = rs >= 0 ? b->sH[rs] : c->s.S;
        const uint8_t* k0 = rs >= 0 ? (const uint8_t*)b->sK[rs] : c->s.kk;
        if (!store) {
            int buf = c->cur;
            const void* x = v0;
            const float* cx = c0;
            for (int i = 0; i < l - 1; ++i) {
                if (i == 0 && rs >= 0) {
                    // from the slot (no ghost margin) into the live buffer
                    DevState v = c->s;
                    v.vpad = 0;
                    v.V[buf] = const_cast<void*>(v0);
                    v.C[buf] = const_cast<float*>(c0);
                    launch_diffusion(v, c->op, buf, false, 0, c->sargs, ref, false, 256, st);
                } else {
                    launch_diffusion(c->s, c->op, buf, false, 0, c->sargs, ref, false, 256, st);
                }
                buf ^= 1;
                x = c->s.V[buf];
                cx = c->s.C[buf];
            }
            diff_react_any(j, x, cx, nullptr, nullptr, c->s.V[buf ^ 1], c->s.C[buf ^ 1], c->s.S, h0, k0, sv, rs);
            buf ^= 1;
            for (int i = 0; i < l; ++i) {
                launch_diffusion(c->s, c->op, buf, i == l - 1, 0, c->sargs, ref, false, 256, st);
                buf ^= 1;
            }
            ++fwd_steps;
            return;
        }
        const void* x = v0;
        const float* cx = c0;
        for (int i = 0; i < l - 1; ++i) {
            b->d1[i] = x;
            diffuse_view(x, b->P[i], cx, b->kahan ? b->CP[i] : nullptr, false, ref, nullptr);
            x = b->P[i];
            cx = b->kahan ? b->CP[i] : nullptr;
        }
        b->d1[l - 1] = x;
        b->rv = b->P[l - 1];
        b->rc = b->kahan ? b->CP[l - 1] : nullptr;
        b->rh = h0;
        b->kused = k0;
        void* y = b->P[l];
        float* cy = b->kahan ? b->CP[l] : nullptr;
        diff_react_any(j, x, cx, b->P[l - 1], b->kahan ? b->CP[l - 1] : nullptr, y, cy, b->Hout, h0, k0, sv, rs);
        const void* yi = y;
        const float* cyi = cy;
        for (int i = 0; i < l; ++i) {
            b->d2[i] = yi;
            void* o = b->P[l + 1 + i];
            float* co = b->kahan ? b->CP[l + 1 + i] : nullptr;
            diffuse_view(yi, o, cyi, co, i == l - 1, ref, b->kk_next);
            yi = o;
            cyi = co;
        }
        b->vend = yi;
        ++fwd_steps;
    }

    // Loss term of the sample taken at the end of step j (and, with inject, its adjoint source).
    template <typename T>
    void loss_at(int64_t j, const void* v, bool inject) {
        if ((j + 1) % sample_every) return;
        const int64_t q = (j + 1) / sample_every - 1;
        if (q >= b->n_samples) return;
        adj_loss_inject<T><<<1, 256, 0, st>>>(b->n_sensors, b->sensors, (const T*)v,
                                              (const T*)b->data + (size_t)q * b->n_sensors, (const T*)b->mR,
                                              (T*)b->mu[mu_cur], b->acc, inject ? 1 : 0);
    }

    // Reverse of one diffusion sub-step whose input was vin: gradient products, then mu <- D mu.
    template <typename T>
    void mu_step(const void* vin) {
        KrefR<T> kr;
        for (int q = 0; q < 64; ++q) kr.k[q] = (T)c->kref[q];
        const OpView<T> op = op_view<T>(c->op);
        const int n = (int)c->n_nodes;
        const int64_t ne = c->n_elem;
        const unsigned grid = (unsigned)((std::max<int64_t>(n, ne) + 255) / 256);
        const int nx = (int)c->n[0], ny = (int)c->n[1];
        const T* mi = (const T*)b->mu[mu_cur];
        T* mo = (T*)b->mu[mu_cur ^ 1];
        if (c->op.kind == 1)
            adj_mu_dgrad<T, 0><<<grid, 256, 0, st>>>(op, n, mi, mo, ne, c->dim, nx, ny, (const T*)vin, c->dt_ad, kr,
                                                     b->g_elem);
        else if (c->op.dim == 2)
            adj_mu_dgrad<T, 2><<<grid, 256, 0, st>>>(op, n, mi, mo, ne, c->dim, nx, ny, (const T*)vin, c->dt_ad, kr,
                                                     b->g_elem);
        else
            adj_mu_dgrad<T, 3><<<grid, 256, 0, st>>>(op, n, mi, mo, ne, c->dim, nx, ny, (const T*)vin, c->dt_ad, kr,
                                                     b->g_elem);
        mu_cur ^= 1;
    }

    // The first sub-step of step III reversed (input vin) and then step A of step j reversed.
    template <typename T, bool K>
    void mu_react_bwd(int64_t j, const void* vin) {
        KrefR<T> kr;
        for (int q = 0; q < 64; ++q) kr.k[q] = (T)c->kref[q];
        const OpView<T> op = op_view<T>(c->op);
        AdjReactArgs<T> a = react_args<T>(c, c->cur, n0 + j, nullptr, nullptr);
        const int64_t ne = c->n_elem;
        const unsigned grid = (unsigned)((std::max<int64_t>(a.n, ne) + 255) / 256);
        const int nx = (int)c->n[0], ny = (int)c->n[1];
        const T* mi = (const T*)b->mu[mu_cur];
        T* mo = (T*)b->mu[mu_cur ^ 1];
        const int dim = c->op.kind == 1 ? 0 : c->op.dim;
        auto go = [&](auto kern) {
            kern<<<grid, 256, 0, st>>>(op, a, mi, mo, ne, c->dim, nx, ny, (const T*)vin, c->dt_ad, kr, b->g_elem,
                                       (const T*)b->rv, b->rc, (const T*)b->rh, b->kused, (T*)b->lamh,
                                       (const T*)b->mR, b->acc + 1);
        };
        if (dim == 0) go(adj_mu_react_bwd<T, K, 0>);
        else if (dim == 2) go(adj_mu_react_bwd<T, K, 2>);
        else go(adj_mu_react_bwd<T, K, 3>);
        mu_cur ^= 1;
    }

    // Reverse of step j (the intermediates of fwd_step(j, true) are in place).
    template <typename T, bool K>
    void rev_step_t(int64_t j) {
        loss_at<T>(j, b->vend, true);
        for (int i = c->l - 1; i >= 1; --i) mu_step<T>(b->d2[i]);
        mu_react_bwd<T, K>(j, b->d2[0]);
        for (int i = c->l - 1; i >= 0; --i) mu_step<T>(b->d1[i]);
    }
    void rev_step(int64_t j) {
        if (c->s.prec == P_F64) rev_step_t<double, false>(j);
        else if (c->s.kahan) rev_step_t<float, true>(j);
        else rev_step_t<float, false>(j);
    }

    static double beta(int s, int r) {   // C(s + r, s), saturating
        double v = 1.0;
        for (int i = 1; i <= s; ++i) {
            v = v * (double)(r + i) / (double)i;
            if (v > 1e18) return 1e18;
        }
        return v;
    }

    int free_slot() {
        for (int q = 0; q < b->n_slots; ++q)
            if (b->slot_step[q] < 0) return q;
        return -1;
    }

    // Reverse steps [a, e) given a checkpoint of step a in slot sa.
    void reverse(int64_t a, int64_t e, int sa) {
        const int64_t t = e - a;
        if (t == 1) {
            restore(sa);
            fwd_step(a, true);
            rev_step(a);
            return;
        }
        const int q = free_slot();
        if (q < 0) {
            for (int64_t j = e - 1; j >= a; --j) {
                restore(sa);
                for (int64_t p = a; p < j; ++p) fwd_step(p, false);
                fwd_step(j, true);
                rev_step(j);
            }
            return;
        }
        int free = 0;
        for (int p = 0; p < b->n_slots; ++p) free += b->slot_step[p] < 0;
        int r = 0;
        while (beta(free, r) < (double)t) ++r;
        int64_t d = t - (int64_t)beta(free - 1, r);
        if (d < 1) d = 1;
        if (d > t - 1) d = t - 1;
        restore(sa);
        for (int64_t p = a; p < a + d; ++p) fwd_step(p, false);
        save(q, a + d);
        reverse(a + d, e, q);
        b->slot_step[q] = -1;
        reverse(a, a + d, sa);
    }
};

int ensure_buffers(daeti_ctx* c, int n_slots, int n_sensors, int n_samples, int64_t hist_steps, bool keep) {
    AdjointBuffers* b = c->adj;
    const int64_t N = c->n_nodes;
    const bool same = b && b->n == N && b->n_slots == n_slots && b->l == c->l && b->n_sensors == n_sensors &&
                      b->n_samples == n_samples && b->n_steps_hist >= hist_steps && b->prec == c->s.prec &&
                      b->kahan == c->s.kahan;
    if (same) return DAETI_OK;
    if (keep) return fail(c, DAETI_ESTATE, "replay must use the sensors, samples and slots of the recording");
    free_adjoint(c);
    b = c->adj = new AdjointBuffers();
    b->n = N;
    b->n_elem = c->n_elem;
    b->n_slots = n_slots;
    b->l = c->l;
    b->n_sensors = n_sensors;
    b->n_samples = n_samples;
    b->n_steps_hist = hist_steps;
    b->prec = c->s.prec;
    b->kahan = c->s.kahan;
    const size_t r = rsize(c);
    auto al = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
        b->allocs.push_back(p);
        return p;
    };
    bool ok = true;
    for (int q = 0; q < n_slots; ++q) {
        b->sV.push_back(al(N * r));
        b->sC.push_back(b->kahan ? al(N * 4) : nullptr);
        b->sH.push_back(al(N * r));
        b->sVs.push_back(al(N * r));
        b->sA.push_back(al(N * r));
        b->sK.push_back(al(N));
        ok = ok && b->sV.back() && b->sH.back() && b->sVs.back() && b->sA.back() && b->sK.back() &&
             (!b->kahan || b->sC.back());
    }
    b->slot_step.assign(n_slots, -1);
    b->d1.assign(c->l, nullptr);
    b->d2.assign(c->l, nullptr);
    for (int i = 0; i < 2 * c->l + 1; ++i) {
        b->P.push_back(al(N * r));
        b->CP.push_back(b->kahan ? (float*)al(N * 4) : nullptr);
        ok = ok && b->P.back() && (!b->kahan || b->CP.back());
    }
    b->Hout = al(N * r);
    b->kk_next = (uint8_t*)al(N);
    b->mu[0] = al(N * r);
    b->mu[1] = al(N * r);
    b->lamh = al(N * r);
    b->mR = al(N * r);
    b->g_elem = (double*)al(8 * c->n_elem);
    b->acc = (double*)al(16);
    b->sensors = (int*)al(4 * (size_t)std::max(1, n_sensors));
    b->data = al(r * (size_t)std::max(1, n_sensors) * std::max(1, n_samples));
    if (hist_steps > 0) {
        b->hist_k = (uint8_t*)al((size_t)hist_steps * N);
        b->hist_b = (uint16_t*)al((size_t)hist_steps * N * 2);
        ok = ok && b->hist_k && b->hist_b;
    }
    ok = ok && b->Hout && b->kk_next && b->mu[0] && b->mu[1] && b->lamh && b->mR && b->g_elem && b->acc &&
         b->sensors && b->data;
    if (!ok) {
        free_adjoint(c);
        return fail(c, DAETI_ENOMEM, "adjoint buffers");
    }
    return DAETI_OK;
}

}  // namespace

extern "C" int daeti_adjoint(daeti_ctx* c, const int64_t* sensors, int n_sensors, int sample_every, const double* data,
                             int64_t n_steps, int n_slots, int flags, double* loss, double* grad_d,
                             double* grad_tau_close) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (c->model != DAETI_MODEL_MS || c->mesh_kind != 1)
        return fail(c, DAETI_EUNSUPPORTED, "the adjoint supports Mitchell-Schaeffer on structured grids");
    if (c->s.rrate) return fail(c, DAETI_EUNSUPPORTED, "the adjoint takes the k rule DAETI_K_TOTAL");
    for (int64_t e = 0; e < c->n_elem; ++e)
        if (c->dl[e] != c->dtr[e]) return fail(c, DAETI_EUNSUPPORTED, "the adjoint needs isotropic elements");
    if (n_steps < 1 || n_sensors < 1 || n_sensors > 65536 || sample_every < 1 || !sensors || !data || n_slots < 1)
        return fail(c, DAETI_EINVAL, "bad adjoint arguments");
    const bool record = (flags & DAETI_ADJ_RECORD) != 0, replay = (flags & DAETI_ADJ_REPLAY) != 0;
    const bool no_grad = (flags & DAETI_ADJ_NO_GRADIENT) != 0 || replay || record;
    if (record && replay) return fail(c, DAETI_EINVAL, "record and replay are exclusive");
    for (int q = 0; q < n_sensors; ++q)
        if (sensors[q] < 0 || sensors[q] >= c->n_nodes) return fail(c, DAETI_EINVAL, "sensor out of range");
    const int n_samples = (int)(n_steps / sample_every);
    if (replay && (!c->adj || !c->adj->hist_k || c->adj->n_steps_hist < n_steps))
        return fail(c, DAETI_ESTATE, "replay needs a recorded schedule of at least n_steps");
    int rc = daeti_synchronize(c);
    if (rc) return rc;
    const int64_t hist = (record || replay) ? std::max<int64_t>(n_steps, c->adj ? c->adj->n_steps_hist : 0) : 0;
    if ((rc = ensure_buffers(c, n_slots, n_sensors, n_samples, replay ? c->adj->n_steps_hist : hist, replay)))
        return rc;
    AdjointBuffers* b = c->adj;
    const int64_t N = c->n_nodes;
    const size_t r = rsize(c);
    cudaStream_t st = c->stream;
    // inputs in the state precision
    std::vector<int> hs(sensors, sensors + n_sensors);
    CK(cpy_(c, b->sensors, hs.data(), 4 * (size_t)n_sensors, cudaMemcpyHostToDevice));
    if (n_samples > 0) {
        int e2 = upload_real(c, b->data, data, (int64_t)n_samples * n_sensors);
        if (e2) return e2;
    }
    if ((rc = upload_real(c, b->mR, c->mass.data(), N))) return rc;
    CK(cudaMemsetAsync(b->acc, 0, 16, st));

    Adj A{c, b, st, c->nstep, sample_every, record ? 1 : (replay ? 2 : 0)};
    if (no_grad) {
        std::fill(b->slot_step.begin(), b->slot_step.end(), -1);
        A.save(0, 0);
        for (int64_t j = 0; j < n_steps; ++j) {
            A.fwd_step(j, false);
            if (c->s.prec == P_F64) A.loss_at<double>(j, c->s.V[c->cur], false);
            else A.loss_at<float>(j, c->s.V[c->cur], false);
        }
        A.restore(0);   // the context keeps its starting state
        A.flush();
    } else {
        const int64_t key[5] = {n_steps, n_slots, sample_every, n_samples, c->nstep * 2 + c->cur};
        if (!b->graph || std::memcmp(key, b->gkey, sizeof(key)) != 0) {
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
            // record the sweep on the capture stream: costates and gradients
            // cleared, start saved, binomial reverse sweep, start restored
            Adj G{c, b, c->cap_stream, c->nstep, sample_every, 0};
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaMemsetAsync(b->acc, 0, 16, c->cap_stream);
            cudaMemsetAsync(b->mu[0], 0, N * r, c->cap_stream);
            cudaMemsetAsync(b->mu[1], 0, N * r, c->cap_stream);
            cudaMemsetAsync(b->lamh, 0, N * r, c->cap_stream);
            cudaMemsetAsync(b->g_elem, 0, 8 * (size_t)c->n_elem, c->cap_stream);
            std::fill(b->slot_step.begin(), b->slot_step.end(), -1);
            G.save(0, 0);
            G.reverse(0, n_steps, 0);
            G.restore(0);
            G.flush();
            cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
            if (e != cudaSuccess) return fail(c, DAETI_ECUDA, std::string("adjoint capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->graph = nullptr;
                return fail(c, DAETI_ECUDA, std::string("adjoint graph: ") + cudaGetErrorString(e));
            }
            std::memcpy(b->gkey, key, sizeof(key));
            A.fwd_steps = G.fwd_steps;
        } else {
            A.fwd_steps = c->adj_fwd_steps;
        }
        CK(cudaGraphLaunch(b->graph, st));
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    double acc[2];
    CK(cpy_(c, acc, b->acc, 16, cudaMemcpyDeviceToHost));
    if (loss) *loss = acc[0];
    if (!no_grad) {
        if (grad_tau_close) *grad_tau_close = acc[1];
        if (grad_d && (flags & DAETI_ADJ_NODAL_GRADIENT)) {
            // chain rule of D_e = mean of its nodes' D
            std::vector<double> ge(c->n_elem);
            CK(cpy_(c, ge.data(), b->g_elem, 8 * (size_t)c->n_elem, cudaMemcpyDeviceToHost));
            std::fill(grad_d, grad_d + c->n_nodes, 0.0);
            int64_t nd[8];
            for (int64_t e = 0; e < c->n_elem; ++e) {
                const int nl = elem_nodes(c, e, nd);
                for (int a = 0; a < nl; ++a) grad_d[nd[a]] += ge[e] / nl;
            }
        } else if (grad_d) {
            CK(cpy_(c, grad_d, b->g_elem, 8 * (size_t)c->n_elem, cudaMemcpyDeviceToHost));
        }
    }
    c->adj_fwd_steps = A.fwd_steps;
    return DAETI_OK;
}
