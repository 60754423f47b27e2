// libdaeti C ABI: context, setup, the Strang-splitting scheduler of Eq. 2
// (Section 2) and the read/checkpoint functions.  Host code only; all time
// stepping runs in the kernels of reaction.cu / diffusion.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "assembly.h"
#include "context.h"

using namespace daeti_host;

namespace daeti_host {

int fail(daeti_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

// Copies and fills on the context's stream, completed before returning (the
// legacy default stream does not order against the library's streams).
cudaError_t cpy_(daeti_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

cudaError_t set_(daeti_ctx* c, void* dst, int v, size_t bytes) {
    cudaError_t e = cudaMemsetAsync(dst, v, bytes, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

int dalloc(daeti_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, DAETI_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    return DAETI_OK;
}

size_t rsize(const daeti_ctx* c) { return c->s.prec == P_F64 ? 8 : 4; }

// host double -> device in state precision
int upload_real(daeti_ctx* c, void* dst, const double* src, int64_t count) {
    if (c->s.prec == P_F64) {
        CK(cpy_(c, dst, src, sizeof(double) * count, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> tmp(count);
        for (int64_t i = 0; i < count; ++i) tmp[i] = (float)src[i];
        CK(cpy_(c, dst, tmp.data(), sizeof(float) * count, cudaMemcpyHostToDevice));
    }
    return DAETI_OK;
}

// published initial states
const double TP06_INIT[19] = {-85.23, 0.000126, 3.64, 0.00036, 8.604, 136.89, 0.00172, 0.7444, 0.7045, 0.00621,
                              0.4712, 0.0095, 2.42e-8, 0.999998, 3.373e-5, 0.7888, 0.9755, 0.9953, 0.9073};

// Nodes of element e (structured grids: x fastest, 2^dim nodes; tets: 4).
int elem_nodes(const daeti_ctx* c, int64_t e, int64_t* out) {
    if (c->mesh_kind == 2) {
        for (int a = 0; a < 4; ++a) out[a] = c->tets[e * 4 + a];
        return 4;
    }
    const int64_t nx = c->n[0], ny = c->n[1];
    const int64_t ex = e % (nx - 1), t = e / (nx - 1), ey = t % (ny - 1), ez = t / (ny - 1);
    const int nl = 1 << c->dim;
    for (int a = 0; a < nl; ++a)
        out[a] = (ex + (a & 1)) + nx * ((ey + ((a >> 1) & 1)) + ny * (ez + ((a >> 2) & 1)));
    return nl;
}

// Element values as the means of their nodes' values.
void elem_means(const daeti_ctx* c, const double* nodal, std::vector<double>& out) {
    out.assign(c->n_elem, 0.0);
    int64_t nd[8];
    for (int64_t e = 0; e < c->n_elem; ++e) {
        const int nl = elem_nodes(c, e, nd);
        double s = 0.0;
        for (int a = 0; a < nl; ++a) s += nodal[nd[a]];
        out[e] = s / nl;
    }
}

}  // namespace daeti_host

namespace {

void drop_graphs(daeti_ctx* c) {
    for (int i = 0; i < 8; ++i) {
        if (c->graphs[i]) {
            cudaGraphExecDestroy(c->graphs[i]);
            c->graphs[i] = nullptr;
        }
        if (c->pgraphs[i]) {
            cudaGraphExecDestroy(c->pgraphs[i]);
            c->pgraphs[i] = nullptr;
        }
    }
}

void free_device(daeti_ctx* c) {
    drop_graphs(c);
    free_adjoint(c);
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->s = DevState();
    c->op = DiffOp();
    c->scratch = nullptr;
    c->probe = nullptr;
    c->probe_cap = 0;
    c->prepared = false;
}


int n_states_of(int model) { return model == DAETI_MODEL_MS ? 2 : 19; }

StepRef plain_ref(int64_t n) { return StepRef{nullptr, (long long)n}; }

// ---- launch wrappers (optionally timed with events: 0 reaction, 1 diffusion, 2 other)
// Plain launches: events on both sides, waited for.  Inside the capture of a
// profiling graph: event-record nodes on both sides (cudaEventRecordExternal),
// read after each replay.
void gmark(daeti_ctx* c, cudaStream_t st, int which, bool begin) {
    const int q = c->gnext++;
    while ((int)c->gev.size() <= q) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        c->gev.push_back(e);
    }
    if (begin) {
        if ((int)c->gwhich.size() <= q / 2) c->gwhich.resize(q / 2 + 1);
        c->gwhich[q / 2] = which;
    }
    cudaEventRecordWithFlags(c->gev[q], st, cudaEventRecordExternal);
}

struct Timer {
    daeti_ctx* c;
    cudaStream_t st;
    bool on;
    int which;
    Timer(daeti_ctx* c_, cudaStream_t st_, bool on_, int which_) : c(c_), st(st_), on(on_), which(which_) {
        if (!on) return;
        if (c->gcap) gmark(c, st, which, true);
        else cudaEventRecord(c->ev[0], st);
    }
    ~Timer() {
        if (!on) return;
        if (c->gcap) {
            gmark(c, st, which, false);
            return;
        }
        cudaEventRecord(c->ev[1], st);
        cudaEventSynchronize(c->ev[1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        c->ktime[which] += ms;
        c->klaunch[which] += 1;
    }
};

bool lists_mode(const daeti_ctx* c) { return c->lists && c->sargs.adaptive; }

// quiet: no stimulus window overlaps the step, so the launch is told there are
// no stimuli (it then skips the step time and the window test; J = 0 either way)
void L_react(daeti_ctx* c, StepRef ref, int buf, bool fused, cudaStream_t st, bool timed, bool quiet) {
    Timer t(c, st, timed, 0);
    if (quiet && c->s.n_stims) {
        DevState sv = c->s;
        sv.n_stims = 0;
        launch_reaction(sv, c->margs, c->dt_eff, ref, lists_mode(c), c->par, buf, fused, c->op, c->rtune, st);
    } else {
        launch_reaction(c->s, c->margs, c->dt_eff, ref, lists_mode(c), c->par, buf, fused, c->op, c->rtune, st);
    }
}

void L_diff(daeti_ctx* c, StepRef ref, int src, bool sync, cudaStream_t st, bool timed) {
    Timer t(c, st, timed, 1);
    launch_diffusion(c->s, c->op, src, sync, c->par ^ 1, c->sargs, ref, lists_mode(c), c->diff_block, st,
                     c->rtune.pdl != 0, c->diff_rows);
}

// One Strang step from a synchronisation to the next: step I (l sub-steps,
// the last one fused into the reaction launch unless disabled), step II,
// step III (l sub-steps, synchronisation after the last).  V returns to
// buffer c->cur (2l buffer flips).
void enqueue_step(daeti_ctx* c, StepRef ref, cudaStream_t st, bool timed, bool quiet = false) {
    int buf = c->cur;
    const int first = c->fused ? c->l - 1 : c->l;
    for (int i = 0; i < first; ++i) {
        L_diff(c, ref, buf, false, st, timed);
        buf ^= 1;
    }
    L_react(c, ref, buf, c->fused, st, timed, quiet);
    if (c->fused) buf ^= 1;
    for (int i = 0; i < c->l; ++i) {
        L_diff(c, ref, buf, i == c->l - 1, st, timed);
        buf ^= 1;
    }
    if (lists_mode(c)) c->par ^= 1;
}

// Capture graph_steps steps from the current list parity (quiet: for
// segments in which no stimulus window is open).
// A profiling graph (c->prof == 2) brackets every launch with event-record
// nodes and launches without programmatic dependent launch.
int capture_graph(daeti_ctx* c, cudaGraphExec_t* out, bool quiet) {
    const int G = c->graph_steps;
    const int par0 = c->par;
    const bool profiling = c->prof == 2;
    const int pdl0 = c->rtune.pdl;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    if (profiling) {
        c->gcap = true;
        c->gnext = 0;
        c->rtune.pdl = 0;
    }
    for (int j = 0; j < G; ++j)
        enqueue_step(c, StepRef{c->s.step_ctr, (long long)j}, c->cap_stream, profiling, quiet);
    launch_tick(c->s.step_ctr, G, c->cap_stream);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->gcap = false;
    c->rtune.pdl = pdl0;
    c->par = par0;   // capture only recorded the launches
    if (e != cudaSuccess) return fail(c, DAETI_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(c, DAETI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    return DAETI_OK;
}

// Replay whole graphs while at least `reserve` + graph_steps steps remain.
int replay_graphs(daeti_ctx* c, int64_t& remaining, int64_t reserve, cudaStream_t st) {
    const int G = c->graph_steps;
    if (c->prof == 1 || G <= 0 || remaining - reserve < G) return DAETI_OK;
    const bool profiling = c->prof == 2;
    cudaGraphExec_t* table = profiling ? c->pgraphs : c->graphs;
    launch_set_counter(c->s.step_ctr, c->nstep, st);
    while (remaining - reserve >= G) {
        const bool quiet = !stimulus_in_steps(c->stim_dev.data(), (int)c->stim_dev.size(), c->dt_eff, c->nstep, G);
        const int key = (c->cur * 2 + c->par) * 2 + (quiet ? 1 : 0);
        if (!table[key]) {
            int rc = capture_graph(c, &table[key], quiet);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(table[key], st));
        if (profiling) {
            // the graph's events hold this replay's times until the next replay
            CK(cudaStreamSynchronize(st));
            for (size_t p = 0; p < c->gwhich.size() && 2 * p + 1 < c->gev.size(); ++p) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, c->gev[2 * p], c->gev[2 * p + 1]));
                c->ktime[c->gwhich[p]] += ms;
                c->klaunch[c->gwhich[p]] += 1;
            }
        }
        c->nstep += G;
        remaining -= G;
    }
    return DAETI_OK;
}

}  // namespace

extern "C" {

void daeti_default_options(daeti_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = (int32_t)sizeof(daeti_options);
    o->precision = DAETI_FP32_KAHAN;
    o->scheme = DAETI_SCHEME_DAETI;
    o->l_rounding = DAETI_L_FLOOR;
    o->dt = 0.1;
    o->dt0 = 0.01;
    o->v_threshold = std::numeric_limits<double>::quiet_NaN();
    o->gate_rush_larsen = 1;
    o->bucket_k = 1;
    o->graph_steps = 20;
    o->react_block = 0;
    o->diff_block = 0;
    o->fuse_diffusion = 1;
}

int daeti_create(daeti_ctx** out, const daeti_options* opt) {
    daeti_ctx* c = nullptr;
    if (!out) return DAETI_EINVAL;
    *out = nullptr;
    daeti_options o;
    daeti_default_options(&o);
    if (opt) {
        if (opt->struct_size != (int32_t)sizeof(daeti_options)) return DAETI_EINVAL;
        o = *opt;
    }
    if (!(o.dt > 0) || !(o.dt0 > 0) || o.precision < 0 || o.precision > 2 || o.scheme < 0 || o.scheme > 2 ||
        o.l_rounding < 0 || o.l_rounding > 1 || o.graph_steps < 0 || o.k_rule < 0 || o.k_rule > 1)
        return DAETI_EINVAL;
    if (o.graph_steps % 2) o.graph_steps += 1;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return DAETI_ECUDA;
    c = new daeti_ctx();
    c->opt = o;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return DAETI_ECUDA;
    }
    c->own_stream = true;
    for (int i = 0; i < 4; ++i) cudaEventCreate(&c->ev[i]);
    if (o.react_block > 0) c->rtune.block = o.react_block;
    if (o.diff_block > 0) c->diff_block = o.diff_block;
    c->fused = o.fuse_diffusion != 0;
    c->lists = o.bucket_k != 0;
    c->graph_steps = o.graph_steps;
    *out = c;
    return DAETI_OK;
}

int daeti_destroy(daeti_ctx* c) {
    if (!c) return DAETI_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_device(c);
    for (int i = 0; i < 4; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    for (cudaEvent_t e : c->gev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return DAETI_OK;
}

const char* daeti_last_error(const daeti_ctx* c) { return c ? c->err.c_str() : "null context"; }

int daeti_set_stream(daeti_ctx* c, void* stream) {
    if (!c) return DAETI_EINVAL;
    if (c->own_stream && c->stream) {
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
    }
    c->own_stream = false;
    c->stream = (cudaStream_t)stream;
    return DAETI_OK;
}

int daeti_set_mesh_grid(daeti_ctx* c, int dim, const int64_t n[3], double h) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "mesh cannot change after prepare");
    if ((dim != 2 && dim != 3) || !n || !(h > 0)) return fail(c, DAETI_EINVAL, "bad grid arguments");
    for (int d = 0; d < dim; ++d)
        if (n[d] < 2) return fail(c, DAETI_EINVAL, "grid needs >= 2 nodes per axis");
    c->mesh_kind = 1;
    c->dim = dim;
    c->n[0] = n[0];
    c->n[1] = n[1];
    c->n[2] = dim == 3 ? n[2] : 1;
    c->h = h;
    c->n_nodes = c->n[0] * c->n[1] * c->n[2];
    c->n_elem = (c->n[0] - 1) * (c->n[1] - 1) * (dim == 3 ? c->n[2] - 1 : 1);
    if (c->n_nodes >= (int64_t)1 << 31) return fail(c, DAETI_EINVAL, "more than 2^31 - 1 nodes");
    c->have_cond = false;
    return DAETI_OK;
}

int daeti_set_mesh_tet(daeti_ctx* c, int64_t n_nodes, const double* xyz, int64_t n_tets, const int64_t* tets) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "mesh cannot change after prepare");
    if (n_nodes < 4 || n_tets < 1 || !xyz || !tets) return fail(c, DAETI_EINVAL, "bad tet mesh arguments");
    if (n_nodes >= (int64_t)1 << 31) return fail(c, DAETI_EINVAL, "more than 2^31 - 1 nodes");
    std::vector<unsigned char> used(n_nodes, 0);
    for (int64_t e = 0; e < 4 * n_tets; ++e) {
        if (tets[e] < 0 || tets[e] >= n_nodes) return fail(c, DAETI_EINVAL, "tet node index out of range");
        used[tets[e]] = 1;
    }
    // a node in no tetrahedron has no lumped mass (M_L^-1 K is undefined there)
    for (int64_t i = 0; i < n_nodes; ++i)
        if (!used[i]) return fail(c, DAETI_EINVAL, "node " + std::to_string(i) + " belongs to no tetrahedron");
    c->mesh_kind = 2;
    c->dim = 3;
    c->n_nodes = n_nodes;
    c->n_elem = n_tets;
    c->xyz.assign(xyz, xyz + 3 * n_nodes);
    c->tets.assign(tets, tets + 4 * n_tets);
    c->have_cond = false;
    return DAETI_OK;
}

int daeti_set_conductivity(daeti_ctx* c, int64_t n_elem, const double* d_long, const double* d_trans,
                           const double* fibre) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "conductivity cannot change after prepare");
    if (!c->mesh_kind) return fail(c, DAETI_ESTATE, "set the mesh first");
    if (n_elem != c->n_elem || !d_long) return fail(c, DAETI_EINVAL, "n_elem does not match the mesh");
    for (int64_t e = 0; e < n_elem; ++e) {
        const double a = d_long[e], b = d_trans ? d_trans[e] : d_long[e];
        if (!(a >= 0) || !(b >= 0) || !std::isfinite(a) || !std::isfinite(b))
            return fail(c, DAETI_EINVAL, "conductivities must be finite and >= 0");
    }
    c->dl.assign(d_long, d_long + n_elem);
    c->dtr.assign(d_trans ? d_trans : d_long, (d_trans ? d_trans : d_long) + n_elem);
    c->fib_null = fibre == nullptr;
    if (fibre) c->fib.assign(fibre, fibre + 3 * n_elem);
    else c->fib.clear();
    c->have_cond = true;
    return DAETI_OK;
}

int daeti_set_conductivity_nodal(daeti_ctx* c, int64_t n_nodes, const double* d_long, const double* d_trans,
                                 const double* fibre) {
    if (!c) return DAETI_EINVAL;
    if (!c->mesh_kind) return fail(c, DAETI_ESTATE, "set the mesh first");
    if (n_nodes != c->n_nodes || !d_long) return fail(c, DAETI_EINVAL, "n_nodes does not match the mesh");
    std::vector<double> el, et;
    elem_means(c, d_long, el);
    elem_means(c, d_trans ? d_trans : d_long, et);
    return daeti_set_conductivity(c, c->n_elem, el.data(), et.data(), fibre);
}

int daeti_update_conductivity_nodal(daeti_ctx* c, int64_t n_nodes, const double* d_long, const double* d_trans,
                                    const double* fibre) {
    if (!c) return DAETI_EINVAL;
    if (!c->mesh_kind) return fail(c, DAETI_ESTATE, "set the mesh first");
    if (n_nodes != c->n_nodes || !d_long) return fail(c, DAETI_EINVAL, "n_nodes does not match the mesh");
    std::vector<double> el, et;
    elem_means(c, d_long, el);
    elem_means(c, d_trans ? d_trans : d_long, et);
    return daeti_update_conductivity(c, c->n_elem, el.data(), et.data(), fibre);
}

int daeti_set_cell_model(daeti_ctx* c, int model, const double* params, int n_params) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "cell model cannot change after prepare");
    if (model != DAETI_MODEL_MS && model != DAETI_MODEL_TP06) return fail(c, DAETI_EINVAL, "unknown cell model");
    if (n_params < 0 || (n_params > 0 && !params)) return fail(c, DAETI_EINVAL, "bad parameters");
    c->model = model;
    c->params.assign(params, params + n_params);
    if (model == DAETI_MODEL_MS && n_params != 0 && n_params != 5)
        return fail(c, DAETI_EINVAL, "Mitchell-Schaeffer takes 5 parameters");
    if (model == DAETI_MODEL_TP06 && n_params > 1) return fail(c, DAETI_EINVAL, "TP06 takes 1 parameter");
    if (model == DAETI_MODEL_TP06 && n_params == 1 && (params[0] < 0 || params[0] > 2))
        return fail(c, DAETI_EINVAL, "TP06 celltype must be 0, 1 or 2");
    if (model == DAETI_MODEL_MS && n_params == 5)
        for (int i = 0; i < 4; ++i)
            if (!(params[i] > 0)) return fail(c, DAETI_EINVAL, "time constants must be > 0");
    return DAETI_OK;
}

int daeti_set_cell_types(daeti_ctx* c, int64_t n, const uint8_t* type) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "cell types cannot change after prepare");
    if (!c->mesh_kind) return fail(c, DAETI_ESTATE, "set the mesh first");
    if (n != c->n_nodes || !type) return fail(c, DAETI_EINVAL, "one cell type per node");
    for (int64_t i = 0; i < n; ++i)
        if (type[i] > 2) return fail(c, DAETI_EINVAL, "TP06 cell types are 0, 1 or 2");
    c->ctypes.assign(type, type + n);
    return DAETI_OK;
}

int daeti_add_stimulus(daeti_ctx* c, const int64_t* nodes, int64_t n_nodes, double t_start, double duration,
                       double amplitude, double period, int count) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "stimuli cannot change after prepare");
    if (!c->mesh_kind) return fail(c, DAETI_ESTATE, "set the mesh first");
    if ((int)c->stims.size() >= DAETI_MAX_STIM) return fail(c, DAETI_EINVAL, "at most 32 stimuli");
    if (n_nodes < 0 || (n_nodes > 0 && !nodes) || !(duration >= 0) || count < 1 || !std::isfinite(amplitude) ||
        !std::isfinite(t_start) || (count > 1 && !(period > 0)))
        return fail(c, DAETI_EINVAL, "bad stimulus arguments");
    for (int64_t i = 0; i < n_nodes; ++i)
        if (nodes[i] < 0 || nodes[i] >= c->n_nodes) return fail(c, DAETI_EINVAL, "stimulus node out of range");
    StimHost sh;
    sh.nodes.assign(nodes, nodes + n_nodes);
    sh.t0 = t_start;
    sh.dur = duration;
    sh.amp = amplitude;
    sh.period = count > 1 ? period : 0.0;
    sh.count = count;
    c->stims.push_back(sh);
    return DAETI_OK;
}

// Device buffers that are freed when the scope ends (every return path).
struct TempDev {
    std::vector<void*> p;
    void* get(size_t bytes) {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) return nullptr;
        p.push_back(q);
        return q;
    }
    ~TempDev() {
        for (void* q : p) cudaFree(q);
    }
};

// lambda_max of M_L^-1 K (FP64 Lanczos on the GPU, estimator.cu).
static int estimate_lambda_max(daeti_ctx* c, const EstOp& est, const double* d_m, double* lam_out) {
    const int64_t n = est.n;
    const int max_it = DAETI_LANCZOS_MAX_IT;
    TempDev t;
    double* v[3];
    for (int q = 0; q < 3; ++q)
        if (!(v[q] = (double*)t.get(sizeof(double) * n))) return fail(c, DAETI_ENOMEM, "Lanczos vectors");
    double* hist = (double*)t.get(sizeof(double) * 4 * (max_it + 1));
    if (!hist) return fail(c, DAETI_ENOMEM, "Lanczos coefficients");
    std::vector<double> hh(4 * (size_t)max_it);
    int iters = 0;
    CK(lanczos_lambda_max(est, d_m, v, hist, hh.data(), max_it, c->stream, lam_out, &iters));
    return DAETI_OK;
}

// Assemble K and M_L for the current conductivity; FP64 dt_s (Eq. 3) and
// lambda_max on the GPU; host copy of the lumped mass.
static int assemble_and_estimate(daeti_ctx* c, GridTable& tab, bool& table, CsrK& K) {
    const int64_t N = c->n_nodes;
    const double* fib = c->fib_null ? nullptr : c->fib.data();
    std::string err;
    table = false;
    // (a grid whose operator already has one row per node keeps that layout)
    if (c->mesh_kind == 1 && !c->op.per_node)
        table = build_grid_table(c->dim, c->n, c->h, c->dl.data(), c->dtr.data(), fib, tab);
    if (!table) {
        bool ok = c->mesh_kind == 1
                      ? assemble_grid_csr(c->dim, c->n, c->h, c->dl.data(), c->dtr.data(), fib, K, err)
                      : assemble_tet_csr(N, c->xyz.data(), c->n_elem, c->tets.data(), c->dl.data(), c->dtr.data(),
                                         fib, K, err);
        if (!ok) return fail(c, DAETI_EINVAL, err);
    }
    c->mass.assign(N, 0.0);
    if (table) {
        for (int64_t i = 0; i < N; ++i) {
            const int64_t x = i % c->n[0], y = (i / c->n[0]) % c->n[1], z = i / (c->n[0] * c->n[1]);
            const int cx = x == 0 ? 0 : (x == c->n[0] - 1 ? 2 : 1), cy = y == 0 ? 0 : (y == c->n[1] - 1 ? 2 : 1);
            c->mass[i] = tab.m[(z * 3 + cy) * 3 + cx];
        }
    } else {
        c->mass = K.m;
    }
    if (c->mesh_kind == 1) {
        double I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        box_stiffness(c->dim, c->h, I3, c->kref);
    }
    EstOp est;
    est.n = N;
    std::vector<void*> tmp;
    auto tmalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
        tmp.push_back(p);
        return p;
    };
    auto free_tmp = [&]() {
        for (void* p : tmp) cudaFree(p);
        tmp.clear();
    };
    Sell32 sell;
    double* d_m = (double*)tmalloc(N * 8);
    if (!d_m) return fail(c, DAETI_ENOMEM, "estimator buffers");
    cpy_(c, d_m, c->mass.data(), N * 8, cudaMemcpyHostToDevice);
    if (table) {
        est.kind = 0;
        est.dim = c->dim;
        est.nx = tab.nx;
        est.ny = tab.ny;
        est.nz = tab.nz;
        double* kt = (double*)tmalloc(tab.K.size() * 8);
        double* mt = (double*)tmalloc(tab.m.size() * 8);
        if (!kt || !mt) {
            free_tmp();
            return fail(c, DAETI_ENOMEM, "estimator buffers");
        }
        cpy_(c, kt, tab.K.data(), tab.K.size() * 8, cudaMemcpyHostToDevice);
        cpy_(c, mt, tab.m.data(), tab.m.size() * 8, cudaMemcpyHostToDevice);
        est.ktab = kt;
        est.mtab = mt;
        est.m = d_m;
    } else {
        csr_to_sell32(K, nullptr, sell);
        est.kind = 1;
        est.n_chunks = sell.n_chunks;
        int64_t* cp = (int64_t*)tmalloc(sell.chunk_ptr.size() * 8);
        int* cw = (int*)tmalloc(sell.chunk_w.size() * 4);
        int* col = (int*)tmalloc(sell.col.size() * 4);
        double* kv = (double*)tmalloc(sell.val.size() * 8);
        double* kd = (double*)tmalloc(N * 8);
        if (!cp || !cw || !col || !kv || !kd) {
            free_tmp();
            return fail(c, DAETI_ENOMEM, "estimator buffers");
        }
        cpy_(c, cp, sell.chunk_ptr.data(), sell.chunk_ptr.size() * 8, cudaMemcpyHostToDevice);
        cpy_(c, cw, sell.chunk_w.data(), sell.chunk_w.size() * 4, cudaMemcpyHostToDevice);
        cpy_(c, col, sell.col.data(), sell.col.size() * 4, cudaMemcpyHostToDevice);
        cpy_(c, kv, sell.val.data(), sell.val.size() * 8, cudaMemcpyHostToDevice);
        cpy_(c, kd, sell.diag.data(), N * 8, cudaMemcpyHostToDevice);
        est.chunk_ptr = cp;
        est.chunk_w = cw;
        est.col = col;
        est.kval = kv;
        est.kdiag = kd;
        est.m = d_m;
    }
    {
        unsigned long long* bits = (unsigned long long*)tmalloc(8);
        if (!bits) {
            free_tmp();
            return fail(c, DAETI_ENOMEM, "estimator buffers");
        }
        const double big = 1e300;
        unsigned long long hb;
        std::memcpy(&hb, &big, 8);
        cpy_(c, bits, &hb, 8, cudaMemcpyHostToDevice);
        launch_gershgorin(est, bits, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            free_tmp();
            return fail(c, DAETI_ECUDA, std::string("gershgorin: ") + cudaGetErrorString(e));
        }
        cpy_(c, &hb, bits, 8, cudaMemcpyDeviceToHost);
        double mn;
        std::memcpy(&mn, &hb, 8);
        c->dt_s = 0.9 * mn;
    }
    int rc = estimate_lambda_max(c, est, d_m, &c->lam);
    free_tmp();
    return rc;
}

// Time-stepping operator a_ij = dt_ad k_ij / m_i in the state precision;
// allocates on the first call, overwrites in place afterwards.
static int upload_operator(daeti_ctx* c, const GridTable& tab, bool table, const CsrK& K) {
    const int64_t N = c->n_nodes;
    const size_t R = rsize(c);
    int rc = 0;
    void* p = nullptr;
    const bool fresh = c->op.coef == nullptr && c->op.val == nullptr;
    if (table) {
        if (!fresh && (c->op.kind != 0 || c->op.per_node)) return fail(c, DAETI_EINVAL, "operator layout changed");
        c->op.kind = 0;
        c->op.dim = c->dim;
        c->op.nx = tab.nx;
        c->op.ny = tab.ny;
        c->op.nz = tab.nz;
        // rows of DAETI_ROW entries (27 offsets, zero pad) for 16-byte loads
        std::vector<double> A(tab.m.size() * DAETI_ROW, 0.0);
        const int self = 13;   // the centre entry (2D rows use entries 9..17)
        for (size_t cls = 0; cls < tab.m.size(); ++cls)
            for (int j = 0; j < 27; ++j)
                if (j != self) A[cls * DAETI_ROW + j] = c->dt_ad * tab.K[cls * 27 + j] / tab.m[cls];
        if (fresh && (rc = dalloc(c, &c->op.coef, R * A.size()))) return rc;
        if ((rc = upload_real(c, c->op.coef, A.data(), (int64_t)A.size()))) return rc;
        if (tab.dim == 3 && R == 4) {
            // entry pairs (row of a node, row of the node one y above it) for
            // the 3D y-run diffusion kernel, every pair of y classes; the
            // same doubles as the table, so the same floats
            std::vector<double> P((size_t)tab.nz * 27 * 2 * DAETI_ROW, 0.0);
            for (int z = 0; z < tab.nz; ++z)
                for (int ca = 0; ca < 3; ++ca)
                    for (int cb = 0; cb < 3; ++cb)
                        for (int cx = 0; cx < 3; ++cx) {
                            const size_t ra = ((size_t)z * 3 + ca) * 3 + cx, rb = ((size_t)z * 3 + cb) * 3 + cx;
                            double* row = P.data() + ((((size_t)z * 3 + ca) * 3 + cb) * 3 + cx) * 2 * DAETI_ROW;
                            for (int j = 0; j < DAETI_ROW; ++j) {
                                row[2 * j] = A[ra * DAETI_ROW + j];
                                row[2 * j + 1] = A[rb * DAETI_ROW + j];
                            }
                        }
            if (!c->op.pcoef && (rc = dalloc(c, &c->op.pcoef, R * P.size()))) return rc;
            if ((rc = upload_real(c, c->op.pcoef, P.data(), (int64_t)P.size()))) return rc;
        }
        // per-node table row (z * 3 + y class) * 3 + x class, when it fits 16 bits
        if (fresh && (int64_t)tab.nz * 9 <= 65535) {
            std::vector<uint16_t> cls(N);
            const int64_t nx = tab.nx, ny = tab.ny;
            for (int64_t i = 0; i < N; ++i) {
                const int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
                const int cx = x == 0 ? 0 : (x == nx - 1 ? 2 : 1);
                const int cy = y == 0 ? 0 : (y == ny - 1 ? 2 : 1);
                cls[i] = (uint16_t)((z * 3 + cy) * 3 + cx);
            }
            if ((rc = dalloc(c, &p, 2 * (size_t)N))) return rc;
            c->op.cls = (uint16_t*)p;
            CK(cpy_(c, p, cls.data(), 2 * (size_t)N, cudaMemcpyHostToDevice));
        }
    } else if (c->mesh_kind == 1) {
        // structured grid with D varying within layers: one stencil row per
        // node from the CSR rows (entry (dz+1)*9 + (dy+1)*3 + dx+1 for the
        // neighbour at offset (dx, dy, dz); columns ascend, so the terms are
        // added in the CSR order)
        if (!fresh && c->op.kind != 0) return fail(c, DAETI_EINVAL, "operator layout changed");
        const int64_t nx = c->n[0], ny = c->n[1];
        // every row's reach is checked before anything is uploaded, so a
        // rejected operator leaves the current one untouched
        for (int64_t i = 0; i < N; ++i) {
            const int64_t xi = i % nx, yi = (i / nx) % ny, zi = i / (nx * ny);
            for (int64_t q = K.rowptr[i]; q < K.rowptr[i + 1]; ++q) {
                const int64_t j = K.col[q];
                const int64_t dx = j % nx - xi, dy = (j / nx) % ny - yi, dz = j / (nx * ny) - zi;
                if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1)
                    return fail(c, DAETI_EINVAL, "grid operator reaches beyond the 27-point stencil");
            }
        }
        // a grid prepared with per-layer D gets per-node rows on its first
        // update with D varying within a layer (a new coefficient array: the
        // adjoint's captured sweep is dropped)
        const bool grow = !fresh && !c->op.per_node;
        if (grow) free_adjoint(c);
        c->op.kind = 0;
        c->op.per_node = 1;
        c->op.dim = c->dim;
        c->op.nx = (int)nx;
        c->op.ny = (int)ny;
        c->op.nz = c->dim == 3 ? (int)c->n[2] : 1;
        if ((fresh || grow) && (rc = dalloc(c, &c->op.coef, R * (size_t)N * DAETI_ROW))) return rc;
        // built and uploaded in blocks of rows (bounded host memory on large grids)
        const int64_t B = 65536;
        std::vector<double> A;
        for (int64_t i0 = 0; i0 < N; i0 += B) {
            const int64_t nb = std::min(B, N - i0);
            A.assign((size_t)nb * DAETI_ROW, 0.0);
            for (int64_t i = i0; i < i0 + nb; ++i) {
                const double s = K.m[i] > 0 ? c->dt_ad / K.m[i] : 0.0;
                const int64_t xi = i % nx, yi = (i / nx) % ny, zi = i / (nx * ny);
                for (int64_t q = K.rowptr[i]; q < K.rowptr[i + 1]; ++q) {
                    const int64_t j = K.col[q];
                    if (j == i) continue;
                    const int64_t dx = j % nx - xi, dy = (j / nx) % ny - yi, dz = j / (nx * ny) - zi;
                    A[(size_t)(i - i0) * DAETI_ROW + (size_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1))] = K.val[q] * s;
                }
            }
            if ((rc = upload_real(c, (char*)c->op.coef + R * (size_t)i0 * DAETI_ROW, A.data(), (int64_t)A.size())))
                return rc;
        }
    } else {
        if (!fresh && c->op.kind != 1) return fail(c, DAETI_EINVAL, "operator layout changed");
        std::vector<double> scale(N);
        for (int64_t i = 0; i < N; ++i) scale[i] = K.m[i] > 0 ? c->dt_ad / K.m[i] : 0.0;
        Sell32 sa;
        csr_to_sell32(K, scale.data(), sa);
        c->op.kind = 1;
        c->op.n_chunks = sa.n_chunks;
        if (fresh) {
            c->op.nnz_padded = (int64_t)sa.col.size();
            if ((rc = dalloc(c, &p, sa.chunk_ptr.size() * 8))) return rc;
            c->op.chunk_ptr = (int64_t*)p;
            CK(cpy_(c, p, sa.chunk_ptr.data(), sa.chunk_ptr.size() * 8, cudaMemcpyHostToDevice));
            if ((rc = dalloc(c, &p, sa.chunk_w.size() * 4))) return rc;
            c->op.chunk_w = (int*)p;
            CK(cpy_(c, p, sa.chunk_w.data(), sa.chunk_w.size() * 4, cudaMemcpyHostToDevice));
            if ((rc = dalloc(c, &p, sa.col.size() * 4))) return rc;
            c->op.col = (int*)p;
            CK(cpy_(c, p, sa.col.data(), sa.col.size() * 4, cudaMemcpyHostToDevice));
            if ((rc = dalloc(c, &c->op.val, R * sa.val.size()))) return rc;
        } else if ((int64_t)sa.col.size() != c->op.nnz_padded) {
            return fail(c, DAETI_EINVAL, "operator pattern changed");
        }
        if ((rc = upload_real(c, c->op.val, sa.val.data(), (int64_t)sa.val.size()))) return rc;
    }
    return DAETI_OK;
}

int daeti_prepare(daeti_ctx* c) {
    if (!c) return DAETI_EINVAL;
    if (c->prepared) return fail(c, DAETI_ESTATE, "already prepared");
    if (!c->mesh_kind || !c->have_cond || !c->model)
        return fail(c, DAETI_ESTATE, "prepare needs mesh, conductivity and cell model");
    const int64_t N = c->n_nodes;
    if (!c->ctypes.empty() && (c->model != DAETI_MODEL_TP06 || (int64_t)c->ctypes.size() != N))
        return fail(c, DAETI_EINVAL, "per-node cell types need the TP06 model and one type per node");
    c->s = DevState();
    c->op = DiffOp();
    c->s.prec = c->opt.precision == DAETI_FP64 ? P_F64 : P_F32;
    c->s.kahan = c->opt.precision == DAETI_FP32_KAHAN;
    c->s.n = N;
    c->s.n_states = n_states_of(c->model);

    // ---- assembly and FP64 stable-step estimate
    GridTable tab;
    bool table = false;
    CsrK K;
    int rc = assemble_and_estimate(c, tab, table, K);
    if (rc) return rc;

    // ---- scheme: effective dt, l, k_max (Section 2, Section 3)
    double dt = c->opt.dt;
    const bool no_diff = !(c->dt_s < 1e299);   // all-zero conductivity
    if (c->opt.scheme == DAETI_SCHEME_DAETI) {
        c->l = 1;
        if (!no_diff && dt / 2.0 > c->dt_s) {
            const double x = dt / (2.0 * c->dt_s);
            c->l = c->opt.l_rounding == DAETI_L_FLOOR ? (int)std::floor(x) : (int)std::ceil(x);
        }
        c->kmax = std::max(1, (int)std::floor(dt / c->opt.dt0 + 1e-9));
        c->sargs.adaptive = 1;
    } else if (c->opt.scheme == DAETI_SCHEME_OSTAR) {
        if (!no_diff && c->dt_s < dt) dt = dt / std::ceil(dt / c->dt_s - 1e-12);
        c->l = 1;
        c->kmax = std::max(1, (int)std::floor(dt / c->opt.dt0 + 1e-9));
        c->sargs.adaptive = 1;
    } else {
        c->l = 1;
        c->kmax = 1;
        c->sargs.adaptive = 0;
    }
    if (c->kmax >= DAETI_MAX_K) return fail(c, DAETI_EINVAL, "k_max = floor(dt/dt0) must be < 16");
    c->dt_eff = dt;
    c->dt_ad = dt / (2.0 * c->l);
    if (c->dt_ad * c->lam >= 2.0)
        return fail(c, DAETI_EUNSTABLE, "dt_ad * lambda_max >= 2: explicit diffusion would diverge");

    // ---- device state
    const size_t R = rsize(c);
    void* p = nullptr;
    // V buffers of a structured grid carry a zeroed ghost margin of the stencil
    // reach on both sides, so the stencil needs no per-neighbour boundary tests
    const int64_t pad = c->mesh_kind == 1 ? 1 + c->n[0] + (c->dim == 3 ? c->n[0] * c->n[1] : 0) : 0;
    for (int b = 0; b < 2; ++b) {
        if ((rc = dalloc(c, &p, R * (N + 2 * pad)))) return rc;
        CK(set_(c, p, 0, R * (N + 2 * pad)));
        c->s.V[b] = (char*)p + R * pad;
    }
    c->s.vpad = pad;
    if (c->s.kahan) {
        if ((rc = dalloc(c, &p, 4 * N))) return rc;
        c->s.C[0] = (float*)p;
        if ((rc = dalloc(c, &p, 4 * N))) return rc;
        c->s.C[1] = (float*)p;
    }
    if ((rc = dalloc(c, &c->s.S, R * state_elems(N, c->s.n_states - 1)))) return rc;
    if ((rc = dalloc(c, &c->s.vsync, R * N)) || (rc = dalloc(c, &c->s.act, R * N))) return rc;
    if ((rc = dalloc(c, &p, N))) return rc;
    c->s.kk = (uint8_t*)p;
    if (!c->ctypes.empty()) {
        if ((rc = dalloc(c, &p, N))) return rc;
        CK(cpy_(c, p, c->ctypes.data(), N, cudaMemcpyHostToDevice));
        c->s.ctype = (const uint8_t*)p;
    }
    if (c->opt.k_rule == DAETI_K_REACTION && c->sargs.adaptive) {
        if ((rc = dalloc(c, &c->s.rrate, R * N))) return rc;
    }
    if ((rc = dalloc(c, &p, 4 * 2 * DAETI_MAX_K))) return rc;
    c->s.counts = (int*)p;
    if ((rc = dalloc(c, &p, sizeof(int) * (size_t)(c->kmax + 1) * N))) return rc;
    c->s.lists = (int*)p;
    if ((rc = dalloc(c, &p, 8))) return rc;
    c->s.step_ctr = (long long*)p;
    if ((rc = dalloc(c, &p, 16))) return rc;
    c->s.flags = (int*)p;
    if ((rc = dalloc(c, &p, 8))) return rc;
    c->s.substeps = (unsigned long long*)p;
    if ((rc = dalloc(c, &c->scratch, 8 * N))) return rc;
    if (!c->stims.empty()) {
        std::vector<unsigned> mask(N, 0u);
        std::vector<StimDev> sd(c->stims.size());
        for (size_t k = 0; k < c->stims.size(); ++k) {
            for (int64_t v : c->stims[k].nodes) mask[v] |= 1u << k;
            sd[k].t0 = c->stims[k].t0;
            sd[k].dur = c->stims[k].dur;
            sd[k].amp = c->stims[k].amp;
            sd[k].period = c->stims[k].period;
            sd[k].reps = c->stims[k].count;
            sd[k].pad = 0;
        }
        if ((rc = dalloc(c, &p, 4 * N))) return rc;
        c->s.stim_mask = (unsigned*)p;
        CK(cpy_(c, p, mask.data(), 4 * N, cudaMemcpyHostToDevice));
        if ((rc = dalloc(c, &p, sizeof(StimDev) * sd.size()))) return rc;
        c->s.stims = (StimDev*)p;
        c->stim_dev = sd;
        CK(cpy_(c, p, sd.data(), sizeof(StimDev) * sd.size(), cudaMemcpyHostToDevice));
        c->s.n_stims = (int)sd.size();
    }

    if ((rc = upload_operator(c, tab, table, K))) return rc;

    // ---- model and synchronisation arguments
    c->margs = ModelArgs();
    c->margs.model = c->model == DAETI_MODEL_MS ? M_MS : M_TP06;
    if (c->model == DAETI_MODEL_MS && c->params.size() == 5)
        for (int i = 0; i < 5; ++i) c->margs.ms[i] = c->params[i];
    if (c->model == DAETI_MODEL_TP06 && c->params.size() == 1) c->margs.celltype = (int)c->params[0];
    c->margs.gate_rl = c->opt.gate_rush_larsen ? 1 : 0;
    c->sargs.dt = c->dt_eff;
    c->sargs.vscale = c->model == DAETI_MODEL_MS ? 100.0 : 1.0;
    c->sargs.vth = std::isnan(c->opt.v_threshold) ? (c->model == DAETI_MODEL_MS ? 0.5 : -40.0) : c->opt.v_threshold;
    c->sargs.kmax = c->kmax;
    c->rtune.kmax = c->kmax;
    c->prepared = true;
    return daeti_init_state(c, nullptr);
}

int daeti_update_conductivity(daeti_ctx* c, int64_t n_elem, const double* d_long, const double* d_trans,
                              const double* fibre) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (n_elem != c->n_elem || !d_long) return fail(c, DAETI_EINVAL, "n_elem does not match the mesh");
    for (int64_t e = 0; e < n_elem; ++e) {
        const double a = d_long[e], b = d_trans ? d_trans[e] : d_long[e];
        if (!(a >= 0) || !(b >= 0) || !std::isfinite(a) || !std::isfinite(b))
            return fail(c, DAETI_EINVAL, "conductivities must be finite and >= 0");
    }
    int rc = daeti_synchronize(c);
    if (rc) return rc;
    // the previous description and estimates come back if the new field is
    // rejected (the device operator is only replaced once it is accepted)
    std::vector<double> old_dl, old_dtr, old_fib;
    old_dl.swap(c->dl);
    old_dtr.swap(c->dtr);
    old_fib.swap(c->fib);
    const bool old_fib_null = c->fib_null;
    const double old_dt_s = c->dt_s, old_lam = c->lam;
    auto restore = [&]() {
        c->dl.swap(old_dl);
        c->dtr.swap(old_dtr);
        c->fib.swap(old_fib);
        c->fib_null = old_fib_null;
        c->dt_s = old_dt_s;
        c->lam = old_lam;
    };
    c->dl.assign(d_long, d_long + n_elem);
    c->dtr.assign(d_trans ? d_trans : d_long, (d_trans ? d_trans : d_long) + n_elem);
    c->fib_null = fibre == nullptr;
    if (fibre) c->fib.assign(fibre, fibre + 3 * n_elem);
    else c->fib.clear();
    GridTable tab;
    bool table = false;
    CsrK K;
    if ((rc = assemble_and_estimate(c, tab, table, K))) {
        restore();
        return rc;
    }
    // the schedule (dt, l) stays as prepared; it must remain stable
    if (c->dt_ad * c->lam >= 2.0) {
        const double lam_new = c->lam;
        restore();
        return fail(c, DAETI_EUNSTABLE, "new conductivity: dt_ad * lambda_max = " + std::to_string(c->dt_ad * lam_new) +
                                            " >= 2 with the prepared l");
    }
    drop_graphs(c);
    return upload_operator(c, tab, table, K);
}

int daeti_update_cell_params(daeti_ctx* c, const double* params, int n_params) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (!params) return fail(c, DAETI_EINVAL, "null parameters");
    if (c->model == DAETI_MODEL_MS) {
        if (n_params != 5) return fail(c, DAETI_EINVAL, "Mitchell-Schaeffer takes 5 parameters");
        for (int i = 0; i < 4; ++i)
            if (!(params[i] > 0) || !std::isfinite(params[i])) return fail(c, DAETI_EINVAL, "time constants must be > 0");
        if (!std::isfinite(params[4])) return fail(c, DAETI_EINVAL, "v_gate must be finite");
    } else {
        if (n_params != 1 || !(params[0] == 0.0 || params[0] == 1.0 || params[0] == 2.0))
            return fail(c, DAETI_EINVAL, "TP06 takes 1 parameter: celltype 0, 1 or 2");
        if (!c->ctypes.empty()) return fail(c, DAETI_EINVAL, "the cell types are given per node");
    }
    int rc = daeti_synchronize(c);
    if (rc) return rc;
    c->params.assign(params, params + n_params);
    if (c->model == DAETI_MODEL_MS)
        for (int i = 0; i < 5; ++i) c->margs.ms[i] = params[i];
    else
        c->margs.celltype = (int)params[0];
    drop_graphs(c);            // launch arguments hold the model's rates
    drop_adjoint_graph(c);
    return DAETI_OK;
}

int daeti_get_stability(daeti_ctx* c, double* dt_s, double* lambda_max, int* l, int* k_max, double* dt_eff) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (dt_s) *dt_s = c->dt_s;
    if (lambda_max) *lambda_max = c->lam;
    if (l) *l = c->l;
    if (k_max) *k_max = c->kmax;
    if (dt_eff) *dt_eff = c->dt_eff;
    return DAETI_OK;
}

int daeti_get_sizes(daeti_ctx* c, int64_t* n_nodes, int* n_states) {
    if (!c) return DAETI_EINVAL;
    if (!c->mesh_kind) return fail(c, DAETI_ESTATE, "no mesh");
    if (n_nodes) *n_nodes = c->n_nodes;
    if (n_states) *n_states = c->model ? n_states_of(c->model) : 0;
    return DAETI_OK;
}

int daeti_init_state(daeti_ctx* c, const double* state) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    const int64_t N = c->n_nodes;
    const int ns = c->s.n_states;
    if (ns > 32) return fail(c, DAETI_EINVAL, "too many states");
    CK(cudaStreamSynchronize(c->stream));
    InitDefaults def{};
    for (int k = 0; k < ns; ++k) def.v[k] = c->model == DAETI_MODEL_MS ? (k == 0 ? 0.0 : 1.0) : TP06_INIT[k];
    const double* src = nullptr;
    if (state) {
        // one copy of the caller's array to a device staging buffer; the
        // finiteness check, the conversion and the chunked layout run on the GPU
        const size_t bytes = 8 * (size_t)ns * N;
        int rc;
        if (!c->stage && (rc = dalloc(c, &c->stage, bytes))) return rc;
        CK(cudaMemcpyAsync(c->stage, state, bytes, cudaMemcpyHostToDevice, c->stream));
        int* flag = (int*)c->scratch;
        CK(cudaMemsetAsync(flag, 0, 4, c->stream));
        launch_check_finite((const double*)c->stage, (int64_t)ns * N, flag, c->stream);
        int bad = 0;
        CK(cpy_(c, &bad, flag, 4, cudaMemcpyDeviceToHost));
        if (bad) return fail(c, DAETI_EINVAL, "state must be finite");
        src = (const double*)c->stage;
    }
    launch_init_state(src, def, N, ns, c->s.prec, c->s.V[0], c->s.vsync, c->s.S, c->s.act,
                      c->s.kahan ? c->s.C[0] : nullptr, c->s.kahan ? c->s.C[1] : nullptr, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(c->s.kk, 1, N, c->stream));
    if (c->s.rrate) CK(cudaMemsetAsync(c->s.rrate, 0, rsize(c) * N, c->stream));   // first step: rate 0
    CK(cudaMemsetAsync(c->s.counts, 0, 4 * 2 * DAETI_MAX_K, c->stream));
    launch_rebuild_lists(c->s, 0, c->stream);   // every node in the k = 1 list
    CK(cudaMemsetAsync(c->s.flags, 0, 16, c->stream));
    CK(cudaMemsetAsync(c->s.step_ctr, 0, 8, c->stream));
    CK(cudaMemsetAsync(c->s.substeps, 0, 8, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    c->nstep = 0;
    c->cur = 0;
    c->par = 0;
    return DAETI_OK;
}

int daeti_advance(daeti_ctx* c, double t_end) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (!std::isfinite(t_end)) return fail(c, DAETI_EINVAL, "t_end must be finite");
    const double steps_f = t_end / c->dt_eff;
    const int64_t target = (int64_t)std::llround(steps_f);
    if (std::fabs((double)target * c->dt_eff - t_end) > 1e-9 * std::max(1.0, std::fabs(t_end)))
        return fail(c, DAETI_EINVAL, "t_end is not a whole number of steps");
    if (target < c->nstep) return fail(c, DAETI_EINVAL, "t_end is before the current time");
    int64_t remaining = target - c->nstep;
    if (remaining == 0) return DAETI_OK;
    cudaStream_t st = c->stream;
    const bool timed = c->prof != 0;   // plain steps outside whole graphs are timed in both modes
    int rc;
    while (remaining > 0) {
        if ((rc = replay_graphs(c, remaining, 0, st))) return rc;
        if (remaining > 0) {
            const bool quiet = !stimulus_in_steps(c->stim_dev.data(), (int)c->stim_dev.size(), c->dt_eff, c->nstep, 1);
            enqueue_step(c, plain_ref(c->nstep), st, timed, quiet);
            c->nstep++;
            remaining--;
        }
    }
    CK(cudaGetLastError());
    return DAETI_OK;
}

int daeti_synchronize(daeti_ctx* c) {
    if (!c) return DAETI_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    if (c->prepared) {
        int f[4];
        CK(cpy_(c, f, c->s.flags, 16, cudaMemcpyDeviceToHost));
        if (f[0] & 1) return fail(c, DAETI_ENONFINITE, "V became non-finite");
    }
    return DAETI_OK;
}

int daeti_get_time(daeti_ctx* c, double* t, int64_t* n_steps) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (t) *t = (double)c->nstep * c->dt_eff;
    if (n_steps) *n_steps = c->nstep;
    return DAETI_OK;
}

static int read_array(daeti_ctx* c, const void* src, const float* comp, void* out, int dtype, int on_device) {
    if (!out || (dtype != DAETI_DTYPE_F64 && dtype != DAETI_DTYPE_F32)) return fail(c, DAETI_EINVAL, "bad output");
    const int64_t N = c->n_nodes;
    const size_t ob = dtype == DAETI_DTYPE_F64 ? 8 : 4;
    if (on_device) {
        launch_convert(src, c->s.prec, comp, out, dtype == DAETI_DTYPE_F32, N, c->stream);
        CK(cudaGetLastError());
        return DAETI_OK;
    }
    launch_convert(src, c->s.prec, comp, c->scratch, dtype == DAETI_DTYPE_F32, N, c->stream);
    CK(cudaMemcpyAsync(out, c->scratch, ob * N, cudaMemcpyDeviceToHost, c->stream));
    return daeti_synchronize(c);
}

int daeti_read_v_nodes(daeti_ctx* c, const int64_t* nodes, int64_t n_probe, double* out) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (n_probe < 0 || (n_probe > 0 && (!nodes || !out))) return fail(c, DAETI_EINVAL, "bad probe arguments");
    if (n_probe == 0) return DAETI_OK;
    for (int64_t j = 0; j < n_probe; ++j)
        if (nodes[j] < 0 || nodes[j] >= c->n_nodes) return fail(c, DAETI_EINVAL, "probe node out of range");
    if (n_probe > c->probe_cap) {
        void* p = nullptr;
        int rc = dalloc(c, &p, 16 * (size_t)n_probe);
        if (rc) return rc;
        c->probe = p;
        c->probe_cap = n_probe;
    }
    int64_t* dn = (int64_t*)c->probe;
    double* dv = (double*)((char*)c->probe + 8 * (size_t)c->probe_cap);
    CK(cudaMemcpyAsync(dn, nodes, 8 * (size_t)n_probe, cudaMemcpyHostToDevice, c->stream));
    launch_gather_v(c->s.V[c->cur], c->s.prec, c->s.kahan ? c->s.C[c->cur] : nullptr, dn, dv, n_probe, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dv, 8 * (size_t)n_probe, cudaMemcpyDeviceToHost, c->stream));
    return daeti_synchronize(c);
}

int daeti_read_v(daeti_ctx* c, void* out, int dtype, int on_device) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    return read_array(c, c->s.V[c->cur], c->s.kahan ? c->s.C[c->cur] : nullptr, out, dtype, on_device);
}

int daeti_read_activation(daeti_ctx* c, void* out, int dtype, int on_device) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    return read_array(c, c->s.act, nullptr, out, dtype, on_device);
}

int daeti_read_state(daeti_ctx* c, double* out) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (!out) return fail(c, DAETI_EINVAL, "null output");
    const int64_t N = c->n_nodes;
    int rc = daeti_read_v(c, out, DAETI_DTYPE_F64, 0);
    if (rc) return rc;
    for (int k = 1; k < c->s.n_states; ++k) {
        launch_gather_state(c->s.S, c->s.prec, c->s.n_states - 1, k - 1, (double*)c->scratch, N, c->stream);
        CK(cudaMemcpyAsync(out + (size_t)k * N, c->scratch, 8 * N, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return DAETI_OK;
}

// checkpoint layout: header (8 int64) | V | C | S | vsync | act | kk | counts
static int64_t ckpt_bytes(const daeti_ctx* c) {
    const int64_t N = c->n_nodes;
    const int64_t R = (int64_t)rsize(c);
    int64_t b = 64 + R * N;
    if (c->s.kahan) b += 4 * N;
    b += R * state_elems(N, c->s.n_states - 1) + 2 * R * N + N + 4 * 2 * DAETI_MAX_K;
    return b;
}

int daeti_state_bytes(daeti_ctx* c, int64_t* bytes) {
    if (!c || !bytes) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    *bytes = ckpt_bytes(c);
    return DAETI_OK;
}

int daeti_save_state(daeti_ctx* c, void* buf, int64_t buf_bytes) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (!buf || buf_bytes < ckpt_bytes(c)) return fail(c, DAETI_EINVAL, "checkpoint buffer too small");
    CK(cudaStreamSynchronize(c->stream));
    const int64_t N = c->n_nodes, R = (int64_t)rsize(c);
    char* p = (char*)buf;
    int64_t hdr[8] = {0x444145544931LL, N, c->s.n_states, c->s.prec, c->s.kahan, c->nstep, c->par, 0};
    std::memcpy(p, hdr, 64);
    p += 64;
    CK(cpy_(c, p, c->s.V[c->cur], R * N, cudaMemcpyDeviceToHost));
    p += R * N;
    if (c->s.kahan) {
        CK(cpy_(c, p, c->s.C[c->cur], 4 * N, cudaMemcpyDeviceToHost));
        p += 4 * N;
    }
    CK(cpy_(c, p, c->s.S, R * state_elems(N, c->s.n_states - 1), cudaMemcpyDeviceToHost));
    p += R * state_elems(N, c->s.n_states - 1);
    CK(cpy_(c, p, c->s.vsync, R * N, cudaMemcpyDeviceToHost));
    p += R * N;
    CK(cpy_(c, p, c->s.act, R * N, cudaMemcpyDeviceToHost));
    p += R * N;
    CK(cpy_(c, p, c->s.kk, N, cudaMemcpyDeviceToHost));
    p += N;
    CK(cpy_(c, p, c->s.counts, 4 * 2 * DAETI_MAX_K, cudaMemcpyDeviceToHost));
    return DAETI_OK;
}

int daeti_load_state(daeti_ctx* c, const void* buf, int64_t buf_bytes) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (!buf || buf_bytes < ckpt_bytes(c)) return fail(c, DAETI_EINVAL, "checkpoint buffer too small");
    const int64_t N = c->n_nodes, R = (int64_t)rsize(c);
    const char* p = (const char*)buf;
    int64_t hdr[8];
    std::memcpy(hdr, p, 64);
    if (hdr[0] != 0x444145544931LL || hdr[1] != N || hdr[2] != c->s.n_states || hdr[3] != c->s.prec ||
        hdr[4] != (int64_t)c->s.kahan)
        return fail(c, DAETI_EINVAL, "checkpoint does not match this context");
    CK(cudaStreamSynchronize(c->stream));
    p += 64;
    c->cur = 0;
    CK(cpy_(c, c->s.V[0], p, R * N, cudaMemcpyHostToDevice));
    p += R * N;
    if (c->s.kahan) {
        CK(cpy_(c, c->s.C[0], p, 4 * N, cudaMemcpyHostToDevice));
        p += 4 * N;
    }
    CK(cpy_(c, c->s.S, p, R * state_elems(N, c->s.n_states - 1), cudaMemcpyHostToDevice));
    p += R * state_elems(N, c->s.n_states - 1);
    CK(cpy_(c, c->s.vsync, p, R * N, cudaMemcpyHostToDevice));
    p += R * N;
    CK(cpy_(c, c->s.act, p, R * N, cudaMemcpyHostToDevice));
    p += R * N;
    CK(cpy_(c, c->s.kk, p, N, cudaMemcpyHostToDevice));
    p += N;
    CK(set_(c, c->s.flags, 0, 16));
    CK(set_(c, c->s.substeps, 0, 8));
    c->nstep = hdr[5];
    c->par = (int)hdr[6];
    // the per-k lists follow from k
    CK(set_(c, c->s.counts, 0, 4 * 2 * DAETI_MAX_K));
    launch_rebuild_lists(c->s, c->par, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    return DAETI_OK;
}

int daeti_get_substeps(daeti_ctx* c, int64_t* total) {
    if (!c || !total) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    unsigned long long v = 0;
    CK(cpy_(c, &v, c->s.substeps, 8, cudaMemcpyDeviceToHost));
    *total = (int64_t)v;
    return DAETI_OK;
}

int daeti_set_profiling(daeti_ctx* c, int enable) {
    if (!c) return DAETI_EINVAL;
    if (enable < 0 || enable > 2) return fail(c, DAETI_EINVAL, "profiling mode is 0, 1 or 2");
    int rc = daeti_synchronize(c);
    if (rc) return rc;
    c->prof = enable;
    for (int i = 0; i < 3; ++i) {
        c->ktime[i] = 0.0;
        c->klaunch[i] = 0;
    }
    return DAETI_OK;
}

int daeti_time_launches(daeti_ctx* c, int which, int count, double* ms_per_launch) {
    if (!c) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    if (which < 0 || which > 2 || count < 1 || count > 1000 || !ms_per_launch)
        return fail(c, DAETI_EINVAL, "which must be 0, 1 or 2 and count in 1..1000");
    int rc = daeti_synchronize(c);
    if (rc) return rc;
    const bool quiet = !stimulus_in_steps(c->stim_dev.data(), (int)c->stim_dev.size(), c->dt_eff, c->nstep, 1);
    const StepRef ref = plain_ref(c->nstep);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < count; ++q) {
        if (which == 0) L_react(c, ref, c->cur, c->fused, c->cap_stream, false, quiet);
        else L_diff(c, ref, c->cur, which == 2, c->cap_stream, false);
    }
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return fail(c, DAETI_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, DAETI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    float ms = 0.f;
    e = cudaGraphLaunch(ge, c->stream);   // warm-up replay
    if (e == cudaSuccess) e = cudaEventRecord(c->ev[2], c->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev[3], c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(c->ev[3]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return fail(c, DAETI_ECUDA, std::string("timing replay: ") + cudaGetErrorString(e));
    *ms_per_launch = (double)ms / count;
    return DAETI_OK;
}

int daeti_get_kernel_time(daeti_ctx* c, int which, double* total_ms, int64_t* launches) {
    if (!c || which < 0 || which > 2) return DAETI_EINVAL;
    if (total_ms) *total_ms = c->ktime[which];
    if (launches) *launches = c->klaunch[which];
    return DAETI_OK;
}

int daeti_kernel_work(daeti_ctx* c, int which, double* bytes, double* flops) {
    if (!c || which < 0 || which > 2) return DAETI_EINVAL;
    if (!c->prepared) return fail(c, DAETI_ESTATE, "not prepared");
    const double N = (double)c->n_nodes, R = (double)rsize(c);
    const double comp = c->s.kahan ? 8.0 : 0.0;   // Kahan term read + written
    const double sync = 2.0 * R + 1.0 + R + (lists_mode(c) ? 4.0 : 0.0);   // vsync r/w, k w, act r, list w
    double b = 0.0, f = 0.0;
    if (which == 0) {
        // every state read and written once per step A, plus the node's list entry;
        // flops: arithmetic operations per node sub-step of the cell model, counted
        // from cells.cuh (add/sub/mul/fma and each exp, log, reciprocal, rsqrt as one)
        b = N * (2.0 * R * c->s.n_states + comp + (lists_mode(c) ? 4.0 : 1.0));
        f = c->model == DAETI_MODEL_TP06 ? 450.0 : 20.0;
        if (c->fused) {
            // plus the fused diffusion sub-step: V and the Kahan term of the source buffer
            b += N * (R + (c->s.kahan ? 4.0 : 0.0));
            if (c->op.kind == 1) b += (double)c->op.nnz_padded * (R + 4.0);
            if (c->op.per_node) b += N * (c->dim == 3 ? 26.0 : 8.0) * R;
        }
    } else if (which == 1) {
        // one sub-step launch: V and the Kahan term read and written once,
        // neighbours from cache; the synchronising launch adds its epilogue
        const double npts = c->op.kind == 0 ? (c->dim == 3 ? 26.0 : 8.0) : 15.0;
        b = N * (2.0 * R + comp);
        if (c->op.kind == 1) b += (double)c->op.nnz_padded * (R + 4.0);
        if (c->op.per_node) b += N * npts * R;   // the node's stencil row
        f = N * 2.0 * npts;
    } else {
        b = N * sync;
    }
    if (bytes) *bytes = b;
    if (flops) *flops = f;
    return DAETI_OK;
}

int daeti_get_tuning(daeti_ctx* c, daeti_tuning* t) {
    if (!c || !t) return DAETI_EINVAL;
    t->struct_size = (int32_t)sizeof(daeti_tuning);
    t->react_block = c->rtune.block;
    t->react_min_blocks = c->rtune.min_blocks;
    t->diff_block = c->diff_block;
    t->fuse_diffusion = c->fused ? 1 : 0;
    t->bucket_k = c->lists ? 1 : 0;
    t->graph_steps = c->graph_steps;
    t->pdl = c->rtune.pdl;
    t->diff_rows = c->diff_rows;
    return DAETI_OK;
}

int daeti_set_tuning(daeti_ctx* c, const daeti_tuning* t) {
    if (!c || !t || t->struct_size != (int32_t)sizeof(daeti_tuning)) return DAETI_EINVAL;
    if (t->react_block <= 0 || t->react_block > 128 || t->react_block % 32 || t->diff_block < 0 ||
        t->diff_block > 256 || t->diff_block % 32 || t->graph_steps < 0 ||
        (t->react_min_blocks != 6 && t->react_min_blocks != 8 && t->react_min_blocks != 10) || (t->pdl != 0 && t->pdl != 1) ||
        (t->diff_rows != 0 && t->diff_rows != 2 && t->diff_rows != 4))
        return fail(c, DAETI_EINVAL, "bad tuning values");
    int rc = daeti_synchronize(c);
    if (rc) return rc;
    drop_graphs(c);
    c->rtune.block = t->react_block;
    c->rtune.min_blocks = t->react_min_blocks;
    c->rtune.pdl = t->pdl;
    c->diff_block = t->diff_block;
    c->diff_rows = t->diff_rows;
    c->fused = t->fuse_diffusion != 0;
    const bool new_lists = t->bucket_k != 0;
    if (new_lists != c->lists && c->prepared) {
        c->lists = new_lists;
        // re-derive the lists of the next step A from k
        CK(set_(c, c->s.counts, 0, 4 * 2 * DAETI_MAX_K));
        launch_rebuild_lists(c->s, c->par, c->stream);
        CK(cudaStreamSynchronize(c->stream));
    }
    c->lists = new_lists;
    c->graph_steps = t->graph_steps + (t->graph_steps % 2);
    return DAETI_OK;
}

}  // extern "C"
