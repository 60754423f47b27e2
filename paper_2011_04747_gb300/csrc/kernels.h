// Host-visible launch interface of the libdaeti kernels (no device code).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace daeti {

enum Prec { P_F64 = 0, P_F32 = 1 };
enum Model { M_MS = 1, M_TP06 = 2 };

// Device buffers of the time-stepping state (typed by the context's precision).
struct DevState {
    int prec = P_F32;        // arithmetic of state and operators
    bool kahan = false;      // compensated V updates (float only)
    int64_t n = 0;           // nodes
    int n_states = 0;        // including V
    void* V[2] = {nullptr, nullptr};      // ping-pong V
    int64_t vpad = 0;                     // finite ghost elements before and after each V buffer (stencil reach)
    float* C[2] = {nullptr, nullptr};     // Kahan compensation (nullable)
    void* S = nullptr;                    // other states, in chunks of 32 nodes (state_index)
    void* vsync = nullptr;                // V at the last synchronisation
    uint8_t* kk = nullptr;                // sub-step count of the next step A
    void* act = nullptr;                  // activation times
    int* lists = nullptr;                 // per-k node lists of the next step A: list k at lists + k*n
    int* counts = nullptr;                // [2][DAETI_MAX_K] bucket lengths (k >= 1) by step parity; [par][0]
                                          // = bucketing mode: 1 lists, -K every node expected at k = K
    const uint8_t* ctype = nullptr;       // TP06 cell type per node (nullable: ModelArgs::celltype everywhere)
    void* rrate = nullptr;                // k rule from the reaction rate: dV/dt of each node's last
                                          // sub-step, written by step A, read by the next synchronisation
    unsigned* stim_mask = nullptr;        // per-node stimulus membership bits (nullable)
    StimDev* stims = nullptr;             // stimulus table
    int n_stims = 0;
    long long* step_ctr = nullptr;        // device step counter used by graph replays
    unsigned long long* substeps = nullptr;   // running total of node reaction sub-steps (bucketing)
    int* flags = nullptr;                 // [0] non-finite, [1] unused, [2 + par] k not uniform (mode -K)
};

struct ModelArgs {
    int model = M_TP06;
    double ms[5] = {0.3, 6.0, 120.0, 150.0, 0.13};   // tau_in, tau_out, tau_open, tau_close, v_gate
    int celltype = 0;
    int gate_rl = 1;
};

// Stencil table rows are DAETI_ROW entries: the 27 offsets (dz+1)*9 +
// (dy+1)*3 + (dx+1) (2D uses 9..17), the centre 13 being 0, and one zero pad,
// so that a row is read with 16-byte loads.
#define DAETI_ROW 28

// Diffusion operator in one of two layouts.
struct DiffOp {
    int kind = 0;            // 0 structured stencil table, 1 SELL-32
    int dim = 3;
    int nx = 1, ny = 1, nz = 1;
    void* coef = nullptr;    // table: [nz*9][28] off-diagonal dt_ad K_ij / m_i (centre entry and pad 0)
    uint16_t* cls = nullptr; // table row of each node (nullable)
    // 3D table in float: entry pairs of the rows of nodes (x, y, z) and
    // (x, y + 1, z), [nz][3 y class of the first][3 y class of the second]
    // [3 x class][28][2] (nullable)
    void* pcoef = nullptr;
    int per_node = 0;        // 1: coef holds one row per node (row i for node i), cls unused
    // SELL-32 (rows in chunks of 32, column-major inside a chunk)
    int64_t n_chunks = 0;
    int64_t* chunk_ptr = nullptr;   // start of chunk c in val/col
    int* chunk_w = nullptr;         // width (entries per row) of chunk c
    int* col = nullptr;
    void* val = nullptr;            // off-diagonal dt_ad K_ij / m_i
    int64_t nnz_padded = 0;
};

// True if some stimulus window [t0 + p T, t0 + p T + dur) (the kernels test
// sub-step start times with a 1e-9 ms guard; widened by 1e-6 ms here) meets
// the sub-step times of steps n0 .. n0 + G - 1, i.e. [n0 dt, (n0 + G) dt).
// A launch for steps where this is false may be told there are no stimuli.
inline bool stimulus_in_steps(const StimDev* st, int n, double dt, int64_t n0, int64_t G) {
    const double a = (double)n0 * dt - 1e-6, b = (double)(n0 + G) * dt + 1e-6;
    for (int q = 0; q < n; ++q) {
        const StimDev& s = st[q];
        if (s.reps <= 0) continue;
        const int reps = s.period > 0.0 ? s.reps : 1;
        // repetitions p with t0 + p T < b and t0 + p T + dur > a
        double p0 = 0.0, p1 = (double)(reps - 1);
        if (reps > 1) {
            p0 = std::max(p0, std::ceil((a - s.t0 - s.dur) / s.period) - 1.0);
            p1 = std::min(p1, std::floor((b - s.t0) / s.period) + 1.0);
        }
        for (double p = p0; p <= p1; p += 1.0)
            if (s.t0 + p * s.period < b && s.t0 + p * s.period + s.dur > a) return true;
    }
    return false;
}

// Cell states other than V are stored in chunks of 32 nodes: state s (of ns)
// of node i sits at ((i / 32) * ns + s) * 32 + i % 32.  A thread's states are
// then fixed offsets from one base address, and a warp of consecutive nodes
// reads 128 contiguous bytes per state.  With ns = 1 this is the plain array.
inline int64_t state_chunks(int64_t n) { return (n + 31) / 32; }
inline int64_t state_elems(int64_t n, int ns) { return state_chunks(n) * 32 * ns; }
inline int64_t state_index(int64_t i, int s, int ns) { return ((i >> 5) * ns + s) * 32 + (i & 31); }

// Largest |index offset| of a stencil neighbour on a structured grid (0 for SELL-32).
inline int64_t stencil_reach(const DiffOp& op) {
    if (op.kind != 0) return 0;
    return 1 + (int64_t)op.nx + (op.dim == 3 ? (int64_t)op.nx * op.ny : 0);
}

struct SyncArgs {
    double dt = 0.1;
    double vscale = 1.0;
    double vth = -40.0;
    int kmax = 10;
    int adaptive = 1;
};

// Launch shape of the reaction kernel.
struct ReactTuning {
    int block = 128;        // threads per block (<= 128)
    int min_blocks = 8;     // float TP06: resident 128-thread blocks per SM the registers must allow (6, 8 or 10)
    int kmax = 10;
    int pdl = 1;            // launch the per-step kernels with programmatic dependent launch
};

// Launchers.  `step` identifies the step whose work is launched.
// Step A.  fused = false: on V[src] in place.  fused = true: first one
// diffusion sub-step V[src] -> node value, then step A, result in V[1-src].
// With `lists`, nodes come from the per-k lists of parity `par` (lengths
// counts[par]); counts[1-par] is cleared for the next synchronisation, which
// builds lists unless this step had one k at every node (then it only checks
// that the next step has it too: counts[1-par][0] = -k).
void launch_reaction(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par, int src,
                     bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st);
// One diffusion sub-step from V[src] to V[1-src]; with `sync`, the
// synchronisation epilogue runs on the result (lists of parity `par`).
// pdl: launch with programmatic dependent launch (the kernels wait for their
// predecessor before touching memory either way).
// block: 32..256 one thread per node; 0 on structured grids: 2D shared-memory
// tiles, or in 3D (float, ghost-padded V, per-class table) runs of `rows`
// nodes along y per thread (2 or 4; 0 = 2), else one thread per node.
void launch_diffusion(const DevState& s, const DiffOp& op, int src, bool sync, int par, const SyncArgs& sa,
                      StepRef step, bool lists, int block, cudaStream_t st, bool pdl = false, int rows = 0);
void launch_rebuild_lists(const DevState& s, int par, cudaStream_t st);
void launch_tick(long long* ctr, long long inc, cudaStream_t st);
void launch_set_counter(long long* ctr, long long value, cudaStream_t st);

// FP64 stable-step estimator (Eq. 3) and power iteration on M_L^-1 K.
struct EstOp {
    int kind = 0;                    // 0 table, 1 SELL
    int dim = 3, nx = 1, ny = 1, nz = 1;
    const double* ktab = nullptr;    // table: [nz*9][27] K entries (with diagonal)
    const double* mtab = nullptr;    // table: [nz*9] lumped mass
    int64_t n_chunks = 0;
    const int64_t* chunk_ptr = nullptr;
    const int* chunk_w = nullptr;
    const int* col = nullptr;
    const double* kval = nullptr;    // SELL off-diagonal K
    const double* kdiag = nullptr;   // K diagonal per row
    const double* m = nullptr;       // lumped mass per row
    int64_t n = 0;
};
void launch_gershgorin(const EstOp& op, unsigned long long* out_bits, cudaStream_t st);
void launch_apply_minvk(const EstOp& op, const double* x, double* y, cudaStream_t st);
void launch_mdots(int64_t n, const double* m, const double* x, const double* y, double* out2,
                  cudaStream_t st);
// Largest eigenvalue of M_L^-1 K by Lanczos in the M_L inner product (FP64):
// a start vector fixed by the node numbering, at most max_it iterations,
// stopping when the largest Ritz value changes by <= 1e-13 relative between
// host checks (every 32 iterations) or the Krylov space becomes invariant.
// Work memory is the caller's: v[0..2] n doubles each (device), hist
// 4 (max_it + 1) doubles (device), hh 4 max_it doubles (host).  *iters =
// the order of the final tridiagonal matrix.
cudaError_t lanczos_lambda_max(const EstOp& est, const double* m, double* const v[3], double* hist, double* hh,
                               int max_it, cudaStream_t st, double* lam, int* iters);
// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal
// a[0], a[stride], ... (k entries) and squared off-diagonal b2[0], b2[stride],
// ... (k - 1 entries), by Sturm-sequence bisection.
double tridiag_max_eig(const double* a, const double* b2, int stride, int k);
constexpr int DAETI_LANCZOS_MAX_IT = 2000;
void launch_node_mass(const EstOp& op, double* m_out, cudaStream_t st);

// Conversions between the state precision and the caller's dtype.
void launch_convert(const void* src, int src_prec, const float* comp, void* dst, int dst_f32,
                    int64_t n, cudaStream_t st);
// V at the given nodes (minus the Kahan term), as double.
void launch_gather_v(const void* src, int src_prec, const float* comp, const int64_t* nodes, double* dst, int64_t m,
                     cudaStream_t st);
// State s of every node from the chunked state array, as double.
void launch_gather_state(const void* src, int src_prec, int ns, int s, double* dst, int64_t n, cudaStream_t st);
// Initial state in the device layout: state k of node i from src[k n + i] (ns
// x n doubles on the device; null: def.v[k] at every node) to V and vsync
// (k = 0) and to the chunked cell states (k > 0, lanes of the last chunk past
// n set to 0), in precision prec; act = -1, the compensation terms c0, c1
// (nullable) 0.
struct InitDefaults {
    double v[32];
};
void launch_init_state(const double* src, const InitDefaults& def, int64_t n, int ns, int prec, void* V, void* vsync,
                       void* S, void* act, float* c0, float* c1, cudaStream_t st);
// *flag |= 1 when one of the n values is not finite.
void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t st);
}  // namespace daeti
