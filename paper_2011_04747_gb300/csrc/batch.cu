// Many independent tissues advanced together: every phase of the split step
// (Section 2) is one launch over the nodes of all tissues, and a CUDA graph
// replays a run of steps.  Tissues are 2D/3D structured grids of any size
// with their own conductivity (constant per z layer), cell model and stimuli.
// The nodes of all tissues form one index space, Mitchell-Schaeffer tissues
// first, then TP06 tissues, so each cell model's reaction is one launch over
// a contiguous range.  The diffusion launch finds each node's tissue from a
// per-node tissue id and applies that tissue's stencil table; the arithmetic
// per node is the single-tissue kernels' (results are bit-identical to
// advancing each tissue alone with the same options).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "assembly.h"
#include "context.h"
#include "diffops.cuh"

using namespace daeti_host;

struct BatchTissue {
    int dim;
    int64_t n[3];
    double h;
    std::vector<double> dl, dtr, fib;
    bool fib_null;
    int model;
    std::vector<double> params;
    std::vector<StimHost> stims;
};

struct TissueInfoDev {
    long long off;
    int nx, ny, nz, dim;
    int coef_off;     // first class row of this tissue in the coefficient table
    double rate_scale, vth;   // (model units -> mV) / dt, activation threshold
};

struct daeti_batch {
    daeti_options opt;
    std::string err;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    std::vector<BatchTissue> tissues;
    bool prepared = false;
    int64_t n_total = 0, n_ms = 0, n_tp = 0;
    std::vector<int64_t> off;        // node offset per tissue (in the batch index space)
    int l = 1, kmax = 10;
    double dt = 0.1, dt_ad = 0.05;
    DevState s_all;                  // V, C, vsync, kk, act, stim mask over all nodes
    void* S_ms = nullptr;
    void* S_tp = nullptr;
    void* coef = nullptr;
    int* tid = nullptr;
    uint32_t* rows = nullptr;        // stencil table row of each node (tissue offset included)
    TissueInfoDev* info = nullptr;
    ModelArgs ms_args, tp_args;
    SyncArgs sargs;
    ReactTuning rtune;
    int64_t nstep = 0;
    int cur = 0;
    // per-k node lists of each model pool (0 MS, 1 TP06), as for a single
    // tissue: list k of pool p at plists[p] + k * n_p (pool-local indices),
    // lengths [2 parities][DAETI_MAX_K], uniform-k flags at pflags[p] + 2 + parity
    int* plists[2] = {nullptr, nullptr};
    int* pcounts[2] = {nullptr, nullptr};
    int* pflags[2] = {nullptr, nullptr};
    int par = 0;
    // lists in use per pool: the TP06 pool with bucket_k (its sub-steps are
    // long enough for warp-uniform k to pay for the bucketing); the
    // Mitchell-Schaeffer pool takes each node's own k
    bool listed[2] = {false, false};
    cudaGraphExec_t graph[2][2] = {};   // [list parity][steps with / without an open stimulus window]
    std::vector<StimDev> stim_dev;                     // host copy of the stimulus slots
    int graph_steps = 20;
    std::vector<void*> allocs;
};

namespace {

int bfail(daeti_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? DAETI_ENOMEM : DAETI_ECUDA,          \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

// One node's sub-step (and synchronisation): returns k of the next step A.
template <typename R, bool KAHAN, bool SYNC>
__device__ __forceinline__ int batch_node(const TissueInfoDev* __restrict__ info, const int* __restrict__ tid,
                                          const uint32_t* __restrict__ rows, int i, const R* __restrict__ vin,
                                          R* vout, const float* cin, float* cout, const R* __restrict__ coef,
                                          const SyncParams<R>& sp) {
    const TissueInfoDev t = info[tid[i]];
    const R* crow = coef + (size_t)rows[i] * DAETI_ROW;
    const int nx = t.nx, nxy = t.nx * t.ny;
    auto fetch = [&](int dx, int dy, int dz) { return vin[i + dx + dy * nx + dz * nxy]; };
    R v;
    float cc;
    if (t.dim == 3)
        stencil_update<R, 3, KAHAN, true>(crow, 1, 1, 1, 3, vin[i], KAHAN ? cin[i] : 0.f, fetch, v, cc);
    else
        stencil_update<R, 2, KAHAN, true>(crow, 1, 1, 0, 1, vin[i], KAHAN ? cin[i] : 0.f, fetch, v, cc);
    vout[i] = v;
    if (KAHAN) cout[i] = cc;
    if (SYNC) {
        SyncParams<R> p = sp;
        p.rate_scale = (R)t.rate_scale;
        p.vth = (R)t.vth;
        return sync_node<R, false>(p, i, v);
    }
    return 1;
}

// Bucketing of one model pool at a synchronisation (pool-local node indices).
struct PoolBuckets {
    int* counts;   // lengths of the next step A's lists (null: no lists)
    int* lists;
    int* uflag;
    int n;         // nodes in the pool
    int off;       // first node of the pool in the batch index space
};

// One diffusion sub-step of every tissue.  V buffers carry a zeroed ghost
// margin wider than the largest tissue's stencil reach, and out-of-tissue
// offsets have coefficient 0 in each tissue's table, so a neighbour read past
// a tissue's edge (the next tissue or the margin) adds exactly 0 and no
// boundary test is needed; the node's table row is precomputed.  The
// synchronising sub-step also files each node into its model pool's per-k
// lists for the next step A (or votes that k is still uniform).
template <typename R, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(256) batch_substep_kernel(const TissueInfoDev* __restrict__ info,
                                                           const int* __restrict__ tid,
                                                           const uint32_t* __restrict__ rows, int n,
                                                           const R* __restrict__ vin, R* vout, const float* cin,
                                                           float* cout, const R* __restrict__ coef, SyncParams<R> sp,
                                                           PoolBuckets pb0, PoolBuckets pb1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    int k = 1;
    if (valid) k = batch_node<R, KAHAN, SYNC>(info, tid, rows, i, vin, vout, cin, cout, coef, sp);
    // every thread of the block takes part in each listed pool's bucketing
    if (SYNC && pb0.counts) bucket_nodes(pb0.counts, pb0.lists, pb0.uflag, pb0.n, i - pb0.off, k, valid && i < pb1.off);
    if (SYNC && pb1.counts) bucket_nodes(pb1.counts, pb1.lists, pb1.uflag, pb1.n, i - pb1.off, k, valid && i >= pb1.off);
}

// par: list parity of the step whose synchronisation this is (the lists
// filed are those of parity par ^ 1, the next step's).
template <typename R, bool KAHAN>
void batch_diffuse(daeti_batch* b, int src, bool sync, StepRef ref, cudaStream_t st, int par) {
    SyncParams<R> sp;
    sp.vsync = (R*)b->s_all.vsync;
    sp.kk = b->s_all.kk;
    sp.act = (R*)b->s_all.act;
    sp.counts = nullptr;
    sp.lists = nullptr;
    sp.n = (int)b->n_total;
    sp.flags = b->s_all.flags;
    sp.dt = b->dt;
    sp.rate_scale = (R)(1.0 / b->dt);
    sp.rrate = nullptr;
    sp.vth = (R)0;
    sp.kmax = b->kmax;
    sp.adaptive = b->sargs.adaptive;
    sp.step = ref;
    const int n = (int)b->n_total;
    const int grid = (n + 255) / 256;
    const R* vin = (const R*)b->s_all.V[src];
    R* vout = (R*)b->s_all.V[1 - src];
    const float* cin = KAHAN ? b->s_all.C[src] : nullptr;
    float* cout = KAHAN ? b->s_all.C[1 - src] : nullptr;
    PoolBuckets pb[2];
    const int nxt = par ^ 1;
    for (int q = 0; q < 2; ++q) {
        pb[q].counts = b->listed[q] ? b->pcounts[q] + nxt * DAETI_MAX_K : nullptr;
        pb[q].lists = b->plists[q];
        pb[q].uflag = b->pflags[q] + 2 + nxt;
        pb[q].n = (int)(q ? b->n_tp : b->n_ms);
        pb[q].off = q ? (int)b->n_ms : 0;
    }
    if (sync)
        batch_substep_kernel<R, KAHAN, true><<<grid, 256, 0, st>>>(b->info, b->tid, b->rows, n, vin, vout, cin,
                                                                  cout, (const R*)b->coef, sp, pb[0], pb[1]);
    else
        batch_substep_kernel<R, KAHAN, false><<<grid, 256, 0, st>>>(b->info, b->tid, b->rows, n, vin, vout, cin,
                                                                   cout, (const R*)b->coef, sp, pb[0], pb[1]);
}

void batch_diffuse_any(daeti_batch* b, int src, bool sync, StepRef ref, cudaStream_t st, int par) {
    if (b->s_all.prec == P_F64) batch_diffuse<double, false>(b, src, sync, ref, st, par);
    else if (b->s_all.kahan) batch_diffuse<float, true>(b, src, sync, ref, st, par);
    else batch_diffuse<float, false>(b, src, sync, ref, st, par);
}

// View of one model's contiguous node range as a single-tissue state.
DevState pool_view(daeti_batch* b, bool ms) {
    DevState v = b->s_all;
    const int64_t o = ms ? 0 : b->n_ms;
    const size_t r = v.prec == P_F64 ? 8 : 4;
    v.n = ms ? b->n_ms : b->n_tp;
    v.n_states = ms ? 2 : 19;
    for (int q = 0; q < 2; ++q) {
        v.V[q] = (char*)b->s_all.V[q] + o * r;
        v.C[q] = b->s_all.C[q] ? b->s_all.C[q] + o : nullptr;
    }
    v.S = ms ? b->S_ms : b->S_tp;
    v.vsync = (char*)b->s_all.vsync + o * r;
    v.act = (char*)b->s_all.act + o * r;
    v.kk = b->s_all.kk + o;
    v.stim_mask = b->s_all.stim_mask ? b->s_all.stim_mask + o : nullptr;
    v.lists = b->plists[ms ? 0 : 1];
    v.counts = b->pcounts[ms ? 0 : 1];
    v.flags = b->pflags[ms ? 0 : 1];
    v.substeps = nullptr;
    return v;
}

// One step of every tissue (quiet: no stimulus window is open during it, so
// the reaction launches are told there are no stimuli) with the lists of
// parity par; returns the parity of the next step.
int batch_step(daeti_batch* b, StepRef ref, cudaStream_t st, int par, bool quiet = false) {
    int buf = b->cur;
    for (int i = 0; i < b->l; ++i) {
        batch_diffuse_any(b, buf, false, ref, st, par);
        buf ^= 1;
    }
    DiffOp none;
    DevState ms = pool_view(b, true), tp = pool_view(b, false);
    if (quiet) ms.n_stims = tp.n_stims = 0;
    if (b->n_ms) launch_reaction(ms, b->ms_args, b->dt, ref, b->listed[0], par, buf, false, none, b->rtune, st);
    if (b->n_tp) launch_reaction(tp, b->tp_args, b->dt, ref, b->listed[1], par, buf, false, none, b->rtune, st);
    for (int i = 0; i < b->l; ++i) {
        batch_diffuse_any(b, buf, i == b->l - 1, ref, st, par);
        buf ^= 1;
    }
    return par ^ 1;
}

int balloc(daeti_batch* b, void** p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
        *p = nullptr;
        return bfail(b, DAETI_ENOMEM, "cudaMalloc failed (" + std::to_string(bytes) + " bytes)");
    }
    b->allocs.push_back(*p);
    return DAETI_OK;
}

int bupload(daeti_batch* b, void* dst, const double* src, int64_t count) {
    if (b->s_all.prec == P_F64) {
        BCK(cudaMemcpyAsync(dst, src, 8 * count, cudaMemcpyHostToDevice, b->stream));
    } else {
        std::vector<float> t(count);
        for (int64_t i = 0; i < count; ++i) t[i] = (float)src[i];
        BCK(cudaMemcpyAsync(dst, t.data(), 4 * count, cudaMemcpyHostToDevice, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    return DAETI_OK;
}

}  // namespace

extern "C" {

int daeti_batch_create(daeti_batch** out, const daeti_options* opt) {
    if (!out) return DAETI_EINVAL;
    *out = nullptr;
    daeti_options o;
    daeti_default_options(&o);
    if (opt) {
        if (opt->struct_size != (int32_t)sizeof(daeti_options)) return DAETI_EINVAL;
        o = *opt;
    }
    if (!(o.dt > 0) || !(o.dt0 > 0) || o.precision < 0 || o.precision > 2 || o.scheme != DAETI_SCHEME_DAETI ||
        o.graph_steps < 0 || o.k_rule != DAETI_K_TOTAL)
        return DAETI_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return DAETI_ECUDA;
    daeti_batch* b = new daeti_batch();
    b->opt = o;
    b->graph_steps = o.graph_steps;
    if (o.react_block > 0) b->rtune.block = o.react_block;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return DAETI_ECUDA;
    }
    b->own_stream = true;
    *out = b;
    return DAETI_OK;
}

int daeti_batch_destroy(daeti_batch* b) {
    if (!b) return DAETI_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int q = 0; q < 4; ++q)
        if (b->graph[q / 2][q % 2]) cudaGraphExecDestroy(b->graph[q / 2][q % 2]);
    for (void* p : b->allocs) cudaFree(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return DAETI_OK;
}

const char* daeti_batch_last_error(const daeti_batch* b) { return b ? b->err.c_str() : "null batch"; }

int daeti_batch_set_stream(daeti_batch* b, void* stream) {
    if (!b) return DAETI_EINVAL;
    if (b->own_stream && b->stream) {
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    b->own_stream = false;
    b->stream = (cudaStream_t)stream;
    return DAETI_OK;
}

int daeti_batch_add(daeti_batch* b, const daeti_ctx* t) {
    if (!b || !t) return DAETI_EINVAL;
    if (b->prepared) return bfail(b, DAETI_ESTATE, "batch already prepared");
    if (t->mesh_kind != 1 || !t->have_cond || !t->model)
        return bfail(b, DAETI_EINVAL, "a batch tissue needs a structured grid, conductivity and a cell model");
    BatchTissue bt;
    bt.dim = t->dim;
    for (int d = 0; d < 3; ++d) bt.n[d] = t->n[d];
    bt.h = t->h;
    bt.dl = t->dl;
    bt.dtr = t->dtr;
    bt.fib = t->fib;
    bt.fib_null = t->fib_null;
    bt.model = t->model;
    bt.params = t->params;
    bt.stims = t->stims;
    b->tissues.push_back(std::move(bt));
    return DAETI_OK;
}

int daeti_batch_prepare(daeti_batch* b) {
    if (!b) return DAETI_EINVAL;
    if (b->prepared) return bfail(b, DAETI_ESTATE, "already prepared");
    const int T = (int)b->tissues.size();
    if (T < 1) return bfail(b, DAETI_ESTATE, "empty batch");
    // node order: Mitchell-Schaeffer tissues, then TP06 tissues
    std::vector<int> order;
    for (int pass = 0; pass < 2; ++pass)
        for (int t = 0; t < T; ++t)
            if ((b->tissues[t].model == DAETI_MODEL_MS) == (pass == 0)) order.push_back(t);
    b->off.assign(T, 0);
    int64_t acc = 0;
    b->n_ms = b->n_tp = 0;
    for (int t : order) {
        const BatchTissue& bt = b->tissues[t];
        const int64_t nn = bt.n[0] * bt.n[1] * (bt.dim == 3 ? bt.n[2] : 1);
        b->off[t] = acc;
        acc += nn;
        if (bt.model == DAETI_MODEL_MS) b->n_ms += nn;
        else b->n_tp += nn;
    }
    b->n_total = acc;
    if (acc >= ((int64_t)1 << 31)) return bfail(b, DAETI_EINVAL, "more than 2^31 - 1 nodes");
    // one parameter set per cell model
    const BatchTissue *ms0 = nullptr, *tp0 = nullptr;
    for (const BatchTissue& bt : b->tissues) {
        const BatchTissue*& ref = bt.model == DAETI_MODEL_MS ? ms0 : tp0;
        if (!ref) ref = &bt;
        else if (ref->params != bt.params)
            return bfail(b, DAETI_EUNSUPPORTED, "tissues of one cell model must share its parameters");
    }
    // per-tissue stencil tables, Gershgorin dt_s (Eq. 3) and l
    std::vector<double> A;
    std::vector<TissueInfoDev> info(T);
    b->dt = b->opt.dt;
    b->kmax = std::max(1, (int)std::floor(b->dt / b->opt.dt0 + 1e-9));
    if (b->kmax >= DAETI_MAX_K) return bfail(b, DAETI_EINVAL, "k_max = floor(dt/dt0) must be < 16");
    int l_all = -1;
    std::vector<GridTable> tabs(T);
    for (int t = 0; t < T; ++t) {
        const BatchTissue& bt = b->tissues[t];
        if (!build_grid_table(bt.dim, bt.n, bt.h, bt.dl.data(), bt.dtr.data(), bt.fib_null ? nullptr : bt.fib.data(),
                              tabs[t]))
            return bfail(b, DAETI_EUNSUPPORTED, "batch tissues need conductivity constant on each z layer");
        const GridTable& g = tabs[t];
        double mn = 1e300;
        const int self = 13;   // the centre entry (2D rows use entries 9..17)
        for (size_t cls = 0; cls < g.m.size(); ++cls) {
            double s = g.K[cls * 27 + self];
            for (int j = 0; j < 27; ++j)
                if (j != self) s += std::fabs(g.K[cls * 27 + j]);
            if (s > 0) mn = std::min(mn, g.m[cls] / s);
        }
        const double dts = 0.9 * mn;
        int l = 1;
        if (dts < 1e299 && b->dt / 2.0 > dts) {
            const double x = b->dt / (2.0 * dts);
            l = b->opt.l_rounding == DAETI_L_FLOOR ? (int)std::floor(x) : (int)std::ceil(x);
        }
        if (l_all < 0) l_all = l;
        else if (l != l_all) return bfail(b, DAETI_EUNSUPPORTED, "tissues of one batch must share l");
    }
    b->l = l_all;
    b->dt_ad = b->dt / (2.0 * b->l);
    for (int t = 0; t < T; ++t) {
        const BatchTissue& bt = b->tissues[t];
        const GridTable& g = tabs[t];
        info[t].off = b->off[t];
        info[t].nx = (int)bt.n[0];
        info[t].ny = (int)bt.n[1];
        info[t].nz = bt.dim == 3 ? (int)bt.n[2] : 1;
        info[t].dim = bt.dim;
        info[t].coef_off = (int)(A.size() / DAETI_ROW);
        info[t].rate_scale = (bt.model == DAETI_MODEL_MS ? 100.0 : 1.0) / b->dt;
        info[t].vth = std::isnan(b->opt.v_threshold) ? (bt.model == DAETI_MODEL_MS ? 0.5 : -40.0) : b->opt.v_threshold;
        const int self = 13;
        const size_t base = A.size();
        A.resize(base + g.m.size() * DAETI_ROW, 0.0);
        for (size_t cls = 0; cls < g.m.size(); ++cls)
            for (int j = 0; j < 27; ++j)
                if (j != self) A[base + cls * DAETI_ROW + j] = b->dt_ad * g.K[cls * 27 + j] / g.m[cls];
    }
    // stimuli: identical (t0, duration, amplitude, period, count) share one slot
    // (identical stimuli within one tissue keep separate slots: they add up)
    std::map<std::tuple<double, double, double, double, int, int>, int> slot;
    std::vector<StimDev> sd;
    std::vector<unsigned> mask(b->n_total, 0u);
    for (int t = 0; t < T; ++t) {
        std::map<std::tuple<double, double, double, double, int>, int> seen;
        for (const StimHost& st : b->tissues[t].stims) {
            const int occ = seen[std::make_tuple(st.t0, st.dur, st.amp, st.period, st.count)]++;
            auto key = std::make_tuple(st.t0, st.dur, st.amp, st.period, st.count, occ);
            auto it = slot.find(key);
            int q;
            if (it == slot.end()) {
                q = (int)sd.size();
                if (q >= DAETI_MAX_STIM) return bfail(b, DAETI_EUNSUPPORTED, "more than 32 distinct stimuli");
                slot[key] = q;
                StimDev d{st.t0, st.dur, st.amp, st.period, st.count, 0};
                sd.push_back(d);
            } else {
                q = it->second;
            }
            for (int64_t v : st.nodes) mask[b->off[t] + v] |= 1u << q;
        }
    }
    // device state
    const int64_t N = b->n_total;
    DevState& s = b->s_all;
    s = DevState();
    s.prec = b->opt.precision == DAETI_FP64 ? P_F64 : P_F32;
    s.kahan = b->opt.precision == DAETI_FP32_KAHAN;
    s.n = N;
    const size_t R = s.prec == P_F64 ? 8 : 4;
    int rc;
    void* p;
    // V with a zeroed ghost margin of the largest stencil reach on both sides
    int64_t pad = 0;
    for (const BatchTissue& bt : b->tissues)
        pad = std::max<int64_t>(pad, 1 + bt.n[0] + (bt.dim == 3 ? bt.n[0] * bt.n[1] : 0));
    for (int q = 0; q < 2; ++q) {
        if ((rc = balloc(b, &p, R * (N + 2 * pad)))) return rc;
        BCK(cudaMemsetAsync(p, 0, R * (N + 2 * pad), b->stream));
        s.V[q] = (char*)p + R * pad;
    }
    s.vpad = pad;
    if (s.kahan) {
        if ((rc = balloc(b, &p, 4 * N))) return rc;
        s.C[0] = (float*)p;
        if ((rc = balloc(b, &p, 4 * N))) return rc;
        s.C[1] = (float*)p;
    }
    if ((rc = balloc(b, &s.vsync, R * N)) || (rc = balloc(b, &s.act, R * N))) return rc;
    if ((rc = balloc(b, &p, N))) return rc;
    s.kk = (uint8_t*)p;
    if ((rc = balloc(b, &p, 16))) return rc;
    s.flags = (int*)p;
    if ((rc = balloc(b, &p, 8))) return rc;
    s.step_ctr = (long long*)p;
    for (int q = 0; q < 2; ++q) {
        const int64_t np = q ? b->n_tp : b->n_ms;
        if ((rc = balloc(b, &p, sizeof(int) * (size_t)(b->kmax + 1) * (size_t)std::max<int64_t>(1, np)))) return rc;
        b->plists[q] = (int*)p;
        if ((rc = balloc(b, &p, sizeof(int) * 2 * DAETI_MAX_K))) return rc;
        b->pcounts[q] = (int*)p;
        if ((rc = balloc(b, &p, 16))) return rc;
        b->pflags[q] = (int*)p;
    }
    if ((rc = balloc(b, &b->S_ms, R * std::max<int64_t>(1, b->n_ms)))) return rc;
    if ((rc = balloc(b, &b->S_tp, R * state_elems(std::max<int64_t>(1, b->n_tp), 18)))) return rc;
    if (!sd.empty()) {
        if ((rc = balloc(b, &p, 4 * N))) return rc;
        s.stim_mask = (unsigned*)p;
        BCK(cudaMemcpyAsync(p, mask.data(), 4 * N, cudaMemcpyHostToDevice, b->stream));
        if ((rc = balloc(b, &p, sizeof(StimDev) * sd.size()))) return rc;
        s.stims = (StimDev*)p;
        BCK(cudaMemcpyAsync(p, sd.data(), sizeof(StimDev) * sd.size(), cudaMemcpyHostToDevice, b->stream));
        s.n_stims = (int)sd.size();
        b->stim_dev = sd;
    }
    if ((rc = balloc(b, &b->coef, R * A.size()))) return rc;
    if ((rc = bupload(b, b->coef, A.data(), (int64_t)A.size()))) return rc;
    std::vector<int> tid(N);
    std::vector<uint32_t> rows(N);
    for (int t = 0; t < T; ++t) {
        const BatchTissue& bt = b->tissues[t];
        const int64_t nx = bt.n[0], ny = bt.n[1], nz = bt.dim == 3 ? bt.n[2] : 1;
        std::fill(tid.begin() + b->off[t], tid.begin() + b->off[t] + nx * ny * nz, t);
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int cx = x == 0 ? 0 : (x == nx - 1 ? 2 : 1);
                    const int cy = y == 0 ? 0 : (y == ny - 1 ? 2 : 1);
                    rows[b->off[t] + (z * ny + y) * nx + x] = (uint32_t)(info[t].coef_off + (z * 3 + cy) * 3 + cx);
                }
    }
    if ((rc = balloc(b, &p, 4 * N))) return rc;
    b->tid = (int*)p;
    BCK(cudaMemcpyAsync(p, tid.data(), 4 * N, cudaMemcpyHostToDevice, b->stream));
    if ((rc = balloc(b, &p, 4 * N))) return rc;
    b->rows = (uint32_t*)p;
    BCK(cudaMemcpyAsync(p, rows.data(), 4 * N, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if ((rc = balloc(b, &p, sizeof(TissueInfoDev) * T))) return rc;
    b->info = (TissueInfoDev*)p;
    BCK(cudaMemcpyAsync(p, info.data(), sizeof(TissueInfoDev) * T, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    // model arguments
    b->ms_args = ModelArgs();
    b->ms_args.model = M_MS;
    if (ms0 && ms0->params.size() == 5)
        for (int i = 0; i < 5; ++i) b->ms_args.ms[i] = ms0->params[i];
    b->tp_args = ModelArgs();
    b->tp_args.model = M_TP06;
    if (tp0 && tp0->params.size() == 1) b->tp_args.celltype = (int)tp0->params[0];
    b->ms_args.gate_rl = b->tp_args.gate_rl = b->opt.gate_rush_larsen ? 1 : 0;
    b->sargs.adaptive = 1;
    b->rtune.kmax = b->kmax;
    b->prepared = true;
    // initial state: published defaults
    std::vector<double> v(N), h_ms(std::max<int64_t>(1, b->n_ms), 1.0),
        tp(state_elems(std::max<int64_t>(1, b->n_tp), 18));
    for (int64_t i = 0; i < N; ++i) v[i] = i < b->n_ms ? 0.0 : TP06_INIT[0];
    // TP06 cell states in chunks of 32 pool nodes (state_index)
    for (size_t q = 0; q < tp.size(); ++q) tp[q] = TP06_INIT[1 + (q / 32) % 18];
    if ((rc = bupload(b, s.V[0], v.data(), N)) || (rc = bupload(b, s.vsync, v.data(), N))) return rc;
    if (b->n_ms && (rc = bupload(b, b->S_ms, h_ms.data(), b->n_ms))) return rc;
    if (b->n_tp && (rc = bupload(b, b->S_tp, tp.data(), (int64_t)tp.size()))) return rc;
    std::vector<double> neg(N, -1.0);
    if ((rc = bupload(b, s.act, neg.data(), N))) return rc;
    if (s.kahan) {
        BCK(cudaMemsetAsync(s.C[0], 0, 4 * N, b->stream));
        BCK(cudaMemsetAsync(s.C[1], 0, 4 * N, b->stream));
    }
    BCK(cudaMemsetAsync(s.kk, 1, N, b->stream));
    BCK(cudaMemsetAsync(s.flags, 0, 16, b->stream));
    // every node of a listed pool in the k = 1 list of parity 0
    b->listed[0] = false;
    b->listed[1] = b->opt.bucket_k != 0 && b->n_tp > 0;
    for (int q = 0; q < 2; ++q) {
        BCK(cudaMemsetAsync(b->pcounts[q], 0, sizeof(int) * 2 * DAETI_MAX_K, b->stream));
        BCK(cudaMemsetAsync(b->pflags[q], 0, 16, b->stream));
        if (b->listed[q]) launch_rebuild_lists(pool_view(b, q == 0), 0, b->stream);
    }
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->stream));
    b->nstep = 0;
    b->cur = 0;
    b->par = 0;
    return DAETI_OK;
}

int daeti_batch_advance(daeti_batch* b, double t_end) {
    if (!b) return DAETI_EINVAL;
    if (!b->prepared) return bfail(b, DAETI_ESTATE, "not prepared");
    const int64_t target = (int64_t)std::llround(t_end / b->dt);
    if (!std::isfinite(t_end) || std::fabs((double)target * b->dt - t_end) > 1e-9 * std::max(1.0, std::fabs(t_end)))
        return bfail(b, DAETI_EINVAL, "t_end is not a whole number of steps");
    if (target < b->nstep) return bfail(b, DAETI_EINVAL, "t_end is before the current time");
    int64_t remaining = target - b->nstep;
    const int G = b->graph_steps;
    if (G > 0 && remaining >= G) {
        launch_set_counter(b->s_all.step_ctr, b->nstep, b->stream);
        while (remaining >= G) {
            const int quiet =
                !stimulus_in_steps(b->stim_dev.data(), (int)b->stim_dev.size(), b->dt, b->nstep, G) ? 1 : 0;
            cudaGraphExec_t& ge = b->graph[b->par][quiet];
            int par = b->par;
            if (!ge) {
                cudaGraph_t g = nullptr;
                BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
                for (int j = 0; j < G; ++j)
                    par = batch_step(b, StepRef{b->s_all.step_ctr, (long long)j}, b->cap_stream, par, quiet != 0);
                launch_tick(b->s_all.step_ctr, G, b->cap_stream);
                BCK(cudaStreamEndCapture(b->cap_stream, &g));
                cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    ge = nullptr;
                    return bfail(b, DAETI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
                }
            }
            BCK(cudaGraphLaunch(ge, b->stream));
            b->par ^= G & 1;
            b->nstep += G;
            remaining -= G;
        }
    }
    while (remaining > 0) {
        b->par = batch_step(b, StepRef{nullptr, (long long)b->nstep}, b->stream, b->par);
        b->nstep++;
        remaining--;
    }
    BCK(cudaGetLastError());
    return DAETI_OK;
}

int daeti_batch_synchronize(daeti_batch* b) {
    if (!b) return DAETI_EINVAL;
    BCK(cudaStreamSynchronize(b->stream));
    if (b->prepared) {
        int f[4];
        BCK(cudaMemcpy(f, b->s_all.flags, 16, cudaMemcpyDeviceToHost));
        if (f[0] & 1) return bfail(b, DAETI_ENONFINITE, "V became non-finite");
    }
    return DAETI_OK;
}

int daeti_batch_info(daeti_batch* b, int64_t* n_nodes, int* n_tissues, int* l, double* dt) {
    if (!b) return DAETI_EINVAL;
    if (n_nodes) *n_nodes = b->n_total;
    if (n_tissues) *n_tissues = (int)b->tissues.size();
    if (l) *l = b->l;
    if (dt) *dt = b->dt;
    return DAETI_OK;
}

static int batch_read(daeti_batch* b, int tissue, const void* arr, const float* comp, double* out) {
    if (!b || !out) return DAETI_EINVAL;
    if (!b->prepared) return bfail(b, DAETI_ESTATE, "not prepared");
    if (tissue < 0 || tissue >= (int)b->tissues.size()) return bfail(b, DAETI_EINVAL, "tissue index out of range");
    int rc = daeti_batch_synchronize(b);
    if (rc) return rc;
    const BatchTissue& bt = b->tissues[tissue];
    const int64_t nn = bt.n[0] * bt.n[1] * (bt.dim == 3 ? bt.n[2] : 1);
    const int64_t o = b->off[tissue];
    const size_t R = b->s_all.prec == P_F64 ? 8 : 4;
    std::vector<char> raw(nn * R);
    BCK(cudaMemcpy(raw.data(), (const char*)arr + o * R, nn * R, cudaMemcpyDeviceToHost));
    std::vector<float> cc;
    if (comp) {
        cc.resize(nn);
        BCK(cudaMemcpy(cc.data(), comp + o, 4 * nn, cudaMemcpyDeviceToHost));
    }
    for (int64_t i = 0; i < nn; ++i) {
        double v = R == 8 ? ((const double*)raw.data())[i] : (double)((const float*)raw.data())[i];
        if (comp) v -= (double)cc[i];
        out[i] = v;
    }
    return DAETI_OK;
}

int daeti_batch_read_v(daeti_batch* b, int tissue, double* out) {
    if (!b) return DAETI_EINVAL;
    return batch_read(b, tissue, b->s_all.V[b->cur], b->s_all.kahan ? b->s_all.C[b->cur] : nullptr, out);
}

int daeti_batch_read_activation(daeti_batch* b, int tissue, double* out) {
    if (!b) return DAETI_EINVAL;
    return batch_read(b, tissue, b->s_all.act, nullptr, out);
}

}  // extern "C"
