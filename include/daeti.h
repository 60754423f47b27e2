/*
 * daeti.h — C ABI of libdaeti, a GB300 (sm_103a) solver for the cardiac
 * monodomain equation by dual adaptive explicit time integration.
 *
 * Method (Mountris & Pueyo, arXiv:2011.04747):
 *   Eq. 1    dV/dt = -I_ion(V)/C + div(D grad V),  n . D grad V = 0 on the boundary.
 *   Eq. 2    Strang operator splitting: step I  (diffusion, dt/2),
 *            step II (reaction, dt), step III (diffusion, dt/2); steps III and I of
 *            consecutive steps merge into one "step B" (Section 2).
 *   Step A   (Section 2) forward Euler (Rush-Larsen gates for TP06) with
 *            dt_ar = dt/k per node, k = k0 + floor(|dV/dt|), k0 = 5 if dV/dt > 0
 *            else 1, clamped to [1, k_max], k_max = floor(dt/dt0).
 *   Step B   (Section 2) forward Euler with dt_ad = dt/(2l) on M_L dV/dt = -K V,
 *            l = floor(dt/(2 dt_s)) if dt/2 > dt_s else 1.
 *   Eq. 3    dt_s = 0.9 min_i m_ii / (k_ii + sum_{j!=i} |k_ij|)  (Gershgorin).
 *
 * Conventions common to every entry point
 *   - Every function returns an int status: DAETI_OK (0) or one of the
 *     DAETI_E* codes below; daeti_last_error() gives a message for the last
 *     failure on that context.  No function aborts the process.
 *   - Input arrays are host memory owned by the caller and are copied during
 *     the call; the caller may free them on return.
 *   - The library owns every device allocation it makes (cudaMalloc in
 *     daeti_prepare); daeti_destroy frees them.
 *   - Work is enqueued on the stream given by daeti_set_stream (default: a
 *     stream created by the library).  daeti_advance is asynchronous;
 *     daeti_synchronize and the host-side read functions wait for it.
 *   - Node numbering of structured grids: x + nx*(y + ny*z); element
 *     numbering: ex + (nx-1)*(ey + (ny-1)*ez).  Units: ms, cm, cm^2/ms and
 *     the cell model's own voltage unit (mV for TP06, dimensionless for
 *     Mitchell-Schaeffer).
 *   - Call order: create -> set_mesh_* -> set_conductivity -> set_cell_model
 *     -> add_stimulus* -> prepare -> [init_state] -> advance / read_* ... ->
 *     destroy.  Out-of-order calls return DAETI_ESTATE.
 */
#ifndef DAETI_H
#define DAETI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DAETI_OK 0
#define DAETI_EINVAL 1        /* bad argument (NULL, size, negative D, t_end not a multiple of dt, ...) */
#define DAETI_ENOMEM 2        /* device or host allocation failed */
#define DAETI_ECUDA 3         /* a CUDA runtime call failed (message names it) */
#define DAETI_ESTATE 4        /* call made in the wrong order */
#define DAETI_EUNSTABLE 5     /* dt_ad * lambda_max >= 2 (explicit diffusion would diverge) */
#define DAETI_ENONFINITE 6    /* V became NaN/Inf during advance */
/* 7 is unused (no call waits on the device with a time limit) */
#define DAETI_EUNSUPPORTED 8  /* valid request the library does not implement */

/* arithmetic of the time stepping */
#define DAETI_FP64 0          /* every state, operator and update in double */
#define DAETI_FP32_KAHAN 1    /* float state/operators, compensated (Kahan) V updates */
#define DAETI_FP32 2          /* float, plain V updates */

/* splitting variants of Section 3 */
#define DAETI_SCHEME_DAETI 0  /* adaptive k (step A) and adaptive l (step B) */
#define DAETI_SCHEME_OSTAR 1  /* adaptive k, l = 1, dt reduced to dt/ceil(dt/dt_s) if dt_s < dt */
#define DAETI_SCHEME_OST 2    /* k = l = 1 at the given dt */

#define DAETI_L_FLOOR 0       /* l = floor(dt / (2 dt_s)), as printed in Section 2 */
#define DAETI_L_CEIL 1        /* l = ceil(dt / (2 dt_s)) */

/* the dV/dt of Section 2's k rule ("dV/dt at the previous iteration") */
#define DAETI_K_TOTAL 0       /* (V(t_n) - V(t_{n-1})) / dt of the split solution at the synchronisations */
#define DAETI_K_REACTION 1    /* the reaction's dV/dt at the last sub-step of the previous step A */

/* cell models */
#define DAETI_MODEL_MS 1      /* Mitchell-Schaeffer, params {tau_in, tau_out, tau_open, tau_close, v_gate} */
#define DAETI_MODEL_TP06 2    /* ten Tusscher-Panfilov 2006, params {celltype: 0 endo, 1 epi, 2 mid} */

/* dtype codes for the read functions */
#define DAETI_DTYPE_F64 0
#define DAETI_DTYPE_F32 1

typedef struct daeti_options {
    int32_t struct_size;       /* sizeof(daeti_options); checked by daeti_create */
    int32_t precision;         /* DAETI_FP64 | DAETI_FP32_KAHAN | DAETI_FP32 */
    int32_t scheme;            /* DAETI_SCHEME_* */
    int32_t l_rounding;        /* DAETI_L_FLOOR | DAETI_L_CEIL */
    double dt;                 /* splitting step (ms), > 0 */
    double dt0;                /* smallest reaction sub-step (ms): k_max = floor(dt/dt0) */
    double v_threshold;        /* activation threshold; NaN = model default (MS 0.5, TP06 -40 mV) */
    int32_t gate_rush_larsen;  /* TP06 gates: 1 Rush-Larsen, 0 forward Euler */
    int32_t bucket_k;          /* 1: group nodes by k before step A (warp-uniform sub-step counts) */
    int32_t graph_steps;       /* steps per captured CUDA graph (even, 0 = plain launches) */
    int32_t react_block;       /* threads per block of the reaction kernel (0 = default) */
    int32_t diff_block;        /* threads per block of the diffusion kernel (0 = default) */
    int32_t fuse_diffusion;    /* 1: last diffusion sub-step of step I inside the reaction launch */
    int32_t k_rule;            /* DAETI_K_TOTAL | DAETI_K_REACTION (single tissues; the batch and the
                                  adjoint take DAETI_K_TOTAL) */
} daeti_options;

typedef struct daeti_ctx daeti_ctx;

/* Fill *opt with defaults: FP32_KAHAN, DAETI, FLOOR, dt = 0.1, dt0 = 0.01,
 * v_threshold = NaN, Rush-Larsen gates, bucketing on, 20 steps per graph,
 * default block sizes, fused diffusion on, k rule DAETI_K_TOTAL. */
void daeti_default_options(daeti_options* opt);

/* Create a context.  opt may be NULL (defaults).  *out receives the handle.
 * Errors: EINVAL (bad struct_size or option values), ECUDA (no device). */
int daeti_create(daeti_ctx** out, const daeti_options* opt);

/* Free every host and device resource of ctx (NULL is accepted). */
int daeti_destroy(daeti_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  Owned by ctx. */
const char* daeti_last_error(const daeti_ctx* ctx);

/* Use cuda_stream (a cudaStream_t, may be NULL for the legacy default stream)
 * for all later work.  The stream stays owned by the caller. */
int daeti_set_stream(daeti_ctx* ctx, void* cuda_stream);

/* Structured grid (Section 3.1/3.2 "4-node regular elements"; 8-node hexes in
 * 3D): dim = 2 or 3, n[0..dim-1] >= 2 nodes per axis (n[2] ignored in 2D),
 * spacing h > 0 (cm). */
int daeti_set_mesh_grid(daeti_ctx* ctx, int dim, const int64_t n[3], double h);

/* Tetrahedral mesh (Section 3.3): xyz = 3*n_nodes doubles (cm), tets =
 * 4*n_tets node indices in [0, n_nodes).  EINVAL for an index out of range
 * or a node in no tetrahedron (it would have no lumped mass); degenerate
 * tets -> EINVAL at prepare. */
int daeti_set_mesh_tet(daeti_ctx* ctx, int64_t n_nodes, const double* xyz,
                       int64_t n_tets, const int64_t* tets);

/* Per-element conductivity D_e = d_trans I + (d_long - d_trans) f f^T
 * (Section 3.1: longitudinal d0, transverse rho*d0, fibre direction f).
 * n_elem must equal the mesh's element count; d_long, d_trans >= 0 (0 makes
 * a non-conducting element); fibre = 3*n_elem doubles (normalised here), or
 * NULL for isotropic d_long. */
int daeti_set_conductivity(daeti_ctx* ctx, int64_t n_elem, const double* d_long,
                           const double* d_trans, const double* fibre);

/* The same from per-node values: each element takes the mean of its nodes'
 * d_long and d_trans (n_nodes doubles each; d_trans may be NULL for
 * d_long); fibre as above, per element.  Errors as daeti_set_conductivity
 * (EINVAL if n_nodes differs from the mesh's node count). */
int daeti_set_conductivity_nodal(daeti_ctx* ctx, int64_t n_nodes, const double* d_long,
                                 const double* d_trans, const double* fibre);

/* Cell model for every node (DAETI_MODEL_*) with n_params parameters
 * (params may be NULL for the published defaults). */
int daeti_set_cell_model(daeti_ctx* ctx, int model, const double* params, int n_params);

/* TP06 cell type of each node (transmural heterogeneity): type[i] in
 * {0 endocardial, 1 epicardial, 2 mid-myocardial}, n = the mesh's node count,
 * copied at call; it replaces the single type of daeti_set_cell_model's
 * parameter.  Before prepare; prepare fails with EINVAL unless the cell model
 * is TP06 and n still equals the node count.  Errors: EINVAL (n, a null
 * array or a type out of range), ESTATE (after prepare or before the mesh). */
int daeti_set_cell_types(daeti_ctx* ctx, int64_t n, const uint8_t* type);

/* Stimulus (Section 3: current injected at a node set): amplitude is added to
 * dV/dt (model units per ms) at every reaction sub-step whose start time t
 * satisfies t0 + p*period <= t < t0 + p*period + duration, p < count
 * (1e-9 ms guard on both edges).  At most 32 stimuli. */
int daeti_add_stimulus(daeti_ctx* ctx, const int64_t* nodes, int64_t n_nodes,
                       double t_start, double duration, double amplitude,
                       double period, int count);

/* Assemble K and the lumped mass M_L, allocate device memory, compute dt_s
 * (Eq. 3, FP64 on the GPU), lambda_max(M_L^-1 K) by FP64 Lanczos iteration,
 * l, k_max and the effective dt of the scheme; set the published initial
 * state.  Errors: ESTATE (missing mesh/conductivity/model), EUNSTABLE,
 * ENOMEM, ECUDA. */
int daeti_prepare(daeti_ctx* ctx);

/* Replace the conductivity after prepare (same mesh) keeping the prepared
 * schedule (dt, l, k_max): reassembles K, recomputes dt_s and lambda_max,
 * and returns DAETI_EUNSTABLE if dt_ad * lambda_max >= 2.  On a structured
 * grid prepared with D constant on each layer, the first update with D
 * varying within a layer moves the operator to one stencil row per node
 * (and drops a captured adjoint sweep); that layout is then kept.  The state
 * is kept.  Used for parameter studies and gradient checks. */
int daeti_update_conductivity(daeti_ctx* ctx, int64_t n_elem, const double* d_long,
                              const double* d_trans, const double* fibre);
/* The same from per-node values (element = mean of its nodes). */
int daeti_update_conductivity_nodal(daeti_ctx* ctx, int64_t n_nodes, const double* d_long,
                                    const double* d_trans, const double* fibre);

/* Replace the cell model's parameters after prepare (same model, same count
 * as daeti_set_cell_model: Mitchell-Schaeffer {tau_in, tau_out, tau_open,
 * tau_close, v_gate}, TP06 {celltype} unless types are given per node).  The
 * state and the schedule are kept; captured graphs (also the adjoint's) are
 * dropped, since they hold the model's rates.  Used with
 * daeti_update_conductivity to re-evaluate a misfit and its gradient without
 * a new prepare.  Errors: EINVAL, ESTATE. */
int daeti_update_cell_params(daeti_ctx* ctx, const double* params, int n_params);

/* Stability data computed by prepare (any pointer may be NULL). */
int daeti_get_stability(daeti_ctx* ctx, double* dt_s, double* lambda_max, int* l,
                        int* k_max, double* dt_eff);

/* Node and state counts after prepare. */
int daeti_get_sizes(daeti_ctx* ctx, int64_t* n_nodes, int* n_states);

/* Set the state (host, double, state-major: state[s*n_nodes + i]; row 0 = V)
 * or the model's published initial state when state == NULL; resets t = 0,
 * activation times to -1 and k to 1. */
int daeti_init_state(daeti_ctx* ctx, const double* state);

/* Advance from the current time to t_end (ms; must be a whole number of
 * steps ahead).  Enqueues work and returns without waiting. */
int daeti_advance(daeti_ctx* ctx, double t_end);

/* Wait for enqueued work; returns ENONFINITE if V became NaN/Inf. */
int daeti_synchronize(daeti_ctx* ctx);

/* Current simulated time (ms) and number of completed steps. */
int daeti_get_time(daeti_ctx* ctx, double* t, int64_t* n_steps);

/* Copy V (n_nodes values) into out as dtype (DAETI_DTYPE_*); on_device = 1
 * means out is device memory (enqueued on the stream), 0 host (waits). */
int daeti_read_v(daeti_ctx* ctx, void* out, int dtype, int on_device);

/* V at n_probe given nodes (probe traces, e.g. every step at a few sites):
 * out[j] = V(nodes[j]) as double, into host memory (waits).  nodes is
 * caller-owned host memory of node indices in [0, n_nodes); EINVAL for an
 * index out of range or n_probe < 0. */
int daeti_read_v_nodes(daeti_ctx* ctx, const int64_t* nodes, int64_t n_probe, double* out);

/* Activation times (ms, first upward crossing of v_threshold, -1 if none). */
int daeti_read_activation(daeti_ctx* ctx, void* out, int dtype, int on_device);

/* Full state into host memory (double, state-major, n_states*n_nodes). */
int daeti_read_state(daeti_ctx* ctx, double* out);

/* Checkpoint: byte size of a saved state (*bytes), and save/restore of the
 * complete time-stepping state (state, Kahan terms, V at the last sync, k,
 * activation times, step counter) to/from caller host memory. */
int daeti_state_bytes(daeti_ctx* ctx, int64_t* bytes);
int daeti_save_state(daeti_ctx* ctx, void* buf, int64_t buf_bytes);
int daeti_load_state(daeti_ctx* ctx, const void* buf, int64_t buf_bytes);

/* Total node reaction sub-steps (sum of k over nodes and steps) since the
 * last init_state/load_state; waits for enqueued work. */
int daeti_get_substeps(daeti_ctx* ctx, int64_t* total);

/* Launch shapes (set by the caller or an autotuner; results do not depend on
 * them).  react_block: threads per reaction block (32..128, multiple of 32);
 * react_min_blocks: 6, 8 or 10 resident reaction blocks per SM the register
 * budget must allow (TP06 in float); diff_block: threads per block of the
 * one-thread-per-node diffusion kernel (32..256, multiple of 32; default
 * 256); 0: on structured grids, 2D shared-memory tiles, or in 3D (float
 * precisions, per-layer D) runs of diff_rows nodes along y per thread that
 * share their rows' loads and go in pairs through packed FP32 operations
 * (other meshes, FP64, per-node D and the synchronising launch of the
 * reaction-rate k rule take 256);
 * fuse_diffusion: run the last diffusion sub-step of step I inside the
 * reaction launch; bucket_k: group nodes by k before step A; graph_steps:
 * steps per captured CUDA graph (rounded up to even, 0 = plain launches);
 * pdl: 1 = launch the per-step kernels with
 * programmatic dependent launch, so each one's blocks are resident when its
 * predecessor ends (default), 0 = plain launches; diff_rows: nodes per
 * thread along y of that 3D kernel, 2 or 4 (0 = 2; other values EINVAL).
 * set waits for enqueued work and drops captured graphs. */
typedef struct daeti_tuning {
    int32_t struct_size;       /* sizeof(daeti_tuning) */
    int32_t react_block;
    int32_t react_min_blocks;
    int32_t diff_block;
    int32_t fuse_diffusion;
    int32_t bucket_k;
    int32_t graph_steps;
    int32_t pdl;
    int32_t diff_rows;
} daeti_tuning;
int daeti_get_tuning(daeti_ctx* ctx, daeti_tuning* tuning);
int daeti_set_tuning(daeti_ctx* ctx, const daeti_tuning* tuning);

/* Discrete adjoint (Mitchell-Schaeffer cells, structured grid, isotropic
 * per-element D).  From the current state, runs n_steps steps and returns
 *   *loss = sum_j sum_s (v_{sensors[s]}(t_j) - data[j*n_sensors + s])^2
 * with samples t_j after steps sample_every, 2*sample_every, ... (n_samples =
 * n_steps / sample_every rows of data), and its gradient for the schedule the
 * run chose (k per node and step, gate branch per sub-step, held fixed):
 * grad_d[e] = dL/dD_e (n_elem doubles) and *grad_tau_close = dL/dtau_close.
 * States are recomputed from n_slots device checkpoints (binomial schedule);
 * one slot holds the start, n_slots >= 1.  Sensors must be distinct.  The
 * context's state and time are unchanged on return.
 * flags: DAETI_ADJ_RECORD (forward and loss only, recording the schedule),
 * DAETI_ADJ_REPLAY (forward and loss only, with the recorded schedule; same
 * sensors/samples/slots as the recording), DAETI_ADJ_NO_GRADIENT (forward and
 * loss only), DAETI_ADJ_NODAL_GRADIENT (grad_d holds n_nodes values,
 * dL/dD_i for per-node D whose element values are the means of their nodes:
 * the sum over the elements of node i of dL/dD_e / nodes per element).
 * Errors: EUNSUPPORTED (other models/meshes, anisotropy, the k rule
 * DAETI_K_REACTION), ESTATE (replay without a recording). */
#define DAETI_ADJ_RECORD 1
#define DAETI_ADJ_REPLAY 2
#define DAETI_ADJ_NO_GRADIENT 4
#define DAETI_ADJ_NODAL_GRADIENT 8
int daeti_adjoint(daeti_ctx* ctx, const int64_t* sensors, int n_sensors, int sample_every,
                  const double* data, int64_t n_steps, int n_slots, int flags, double* loss,
                  double* grad_d, double* grad_tau_close);

/* Batch of independent tissues advanced together (one launch per phase of
 * the split step over all tissues, CUDA graphs over runs of steps).  Each
 * tissue is described by a daeti_ctx that received a structured grid,
 * conductivity (constant on each z layer), a cell model and stimuli but need
 * not be prepared; daeti_batch_add copies that description (the context may
 * be destroyed afterwards).  Restrictions: tissues of one cell model share its
 * parameters, all tissues get the same l, at most 32 distinct stimuli.
 * Results per tissue equal advancing that tissue alone with the same
 * options.  tissue indices follow the order of daeti_batch_add. */
typedef struct daeti_batch daeti_batch;
int daeti_batch_create(daeti_batch** out, const daeti_options* opt);
int daeti_batch_destroy(daeti_batch* batch);
const char* daeti_batch_last_error(const daeti_batch* batch);
int daeti_batch_set_stream(daeti_batch* batch, void* cuda_stream);
int daeti_batch_add(daeti_batch* batch, const daeti_ctx* tissue);
int daeti_batch_prepare(daeti_batch* batch);
int daeti_batch_advance(daeti_batch* batch, double t_end);
int daeti_batch_synchronize(daeti_batch* batch);
int daeti_batch_info(daeti_batch* batch, int64_t* n_nodes, int* n_tissues, int* l, double* dt);
int daeti_batch_read_v(daeti_batch* batch, int tissue, double* out);
int daeti_batch_read_activation(daeti_batch* batch, int tissue, double* out);

/* Per-kernel timing.  enable = 1: CUDA events around every launch of the
 * plain-launch path (graphs are not used; each timed interval includes the
 * host launch cost).  enable = 2: runs of graph_steps steps replay captured
 * graphs in which every launch is bracketed by event-record nodes and
 * launched without programmatic dependent launch; the intervals are read
 * after each replay (steps outside whole graphs are timed as with 1).
 * 0 = off.  which: 0 reaction, 1 diffusion (plain sub-steps and fused step
 * B), 2 other.  Returns total milliseconds and launch count since profiling
 * was last set.  Errors: EINVAL (mode). */
int daeti_set_profiling(daeti_ctx* ctx, int enable);
int daeti_get_kernel_time(daeti_ctx* ctx, int which, double* total_ms, int64_t* launches);

/* Duration of one launch of a kernel in graph context at the current state:
 * captures `count` (1..1000) back-to-back launches of the launch the next
 * step would make (which = 0: the reaction launch, with the fused diffusion
 * sub-step if enabled; 1: a diffusion sub-step; 2: the synchronising
 * diffusion sub-step), replays the graph once untimed and once between two
 * CUDA events on the context's stream, and returns the elapsed time / count
 * in *ms_per_launch.  The launches change the state (cells integrated, V
 * diffused, bucket lists appended past their step): save the state before
 * and load it after (daeti_save_state / daeti_load_state).  Waits for the
 * replays.  Errors: EINVAL, ESTATE, ECUDA. */
int daeti_time_launches(daeti_ctx* ctx, int which, int count, double* ms_per_launch);

/* Algorithmic bytes of one launch of kernel `which` at the current problem
 * and its arithmetic operations: for which = 1 (diffusion) per launch, for
 * which = 0 (reaction) per node sub-step (multiply by daeti_get_substeps per
 * launch); add/sub/mul/fma and each exp, log, reciprocal, rsqrt count one.
 * which = 2: the bytes the synchronisation adds to the diffusion launch that
 * ends step III (V at the last synchronisation read and written, k written,
 * activation time read, list entry written with k lists), so that launch
 * moves the bytes of which = 1 plus these; no operations. */
int daeti_kernel_work(daeti_ctx* ctx, int which, double* bytes, double* flops);

/* ---------------------------------------------------------------------------
 * Allocation-free stable-step estimate.  The paper has no counterpart: this is
 * a deployment convenience, not part of the method.
 *
 * For callers that cannot call cudaMalloc: hosts that own all device memory
 * through their own pool or budget, plugins that must not allocate after
 * start-up, and code that must avoid the implicit synchronisation of
 * cudaMalloc / cudaFree.  Computes, for a structured grid whose conductivity
 * is constant on each element layer, the same two numbers that
 * daeti_prepare + daeti_get_stability report: the FP64 Gershgorin stable step
 * dt_s and lambda_max of M_L^-1 K (FP64 Lanczos), with the same table builder
 * and estimator routines.  It calls no cudaMalloc, cudaFree or other
 * allocating library routine: its work vectors live in one fixed __device__
 * array of about 17.8 MB that every GPU which loads libdaeti holds until the
 * process exits.
 *   - Limits: at most DAETI_NOALLOC_MAX_NODES nodes and
 *     DAETI_NOALLOC_MAX_LAYERS node layers in z; larger grids return
 *     DAETI_EINVAL with a message.  Conductivity varying inside an element
 *     layer returns DAETI_EUNSUPPORTED.
 *   - Arguments: as daeti_set_mesh_grid and daeti_set_conductivity (host
 *     arrays, copied during the call); stream = cudaStream_t to run on (NULL =
 *     legacy default stream); results in *dt_s and *lambda_max (host);
 *     errbuf/errbuf_len: optional caller buffer for an error message.
 *   - The first call on each device (with that device current) looks up the
 *     array's device address (cudaGetSymbolAddress).  Every call synchronises
 *     `stream` and copies its results into host memory before it returns, so
 *     it must not be made on a stream under capture: such a call returns
 *     DAETI_EINVAL before any work.
 *   - Every call shares the one array and leaves its contents behind; calls
 *     whose work overlaps on the GPU (from several host threads with
 *     different streams) race on it.  Host-side calls are serialised. */
#define DAETI_NOALLOC_MAX_NODES 524288
#define DAETI_NOALLOC_MAX_LAYERS 512
int daeti_grid_stability_noalloc(int dim, const int64_t n[3], double h, int64_t n_elem,
                                 const double* d_long, const double* d_trans,
                                 const double* fibre, void* stream, double* dt_s,
                                 double* lambda_max, char* errbuf, int errbuf_len);

#ifdef __cplusplus
}
#endif

#endif /* DAETI_H */
