// Private definition of the libdaeti context and host helpers shared by the
// C-ABI translation units (api.cu, adjoint.cu).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/daeti.h"
#include "kernels.h"

using namespace daeti;

struct StimHost {
    std::vector<int64_t> nodes;
    double t0, dur, amp, period;
    int count;
};

struct daeti_ctx {
    daeti_options opt;
    std::string err;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    bool own_stream = false;
    // inputs
    int mesh_kind = 0;   // 1 grid, 2 tets
    int dim = 0;
    int64_t n[3] = {1, 1, 1};
    double h = 0.0;
    int64_t n_nodes = 0, n_elem = 0;
    std::vector<double> xyz;
    std::vector<int64_t> tets;
    bool have_cond = false;
    std::vector<double> dl, dtr, fib;
    bool fib_null = true;
    int model = 0;
    std::vector<double> params;
    std::vector<StimHost> stims;
    // prepared
    bool prepared = false;
    DevState s;
    DiffOp op;
    ModelArgs margs;
    SyncArgs sargs;
    double dt_eff = 0.1, dt_s = 0.0, lam = 0.0, dt_ad = 0.0;
    int l = 1, kmax = 1;
    int64_t nstep = 0;
    int cur = 0;
    int par = 0;
    void* scratch = nullptr;   // n doubles for conversions
    std::vector<uint8_t> ctypes;  // TP06 cell type per node (empty: the model parameter everywhere)
    void* stage = nullptr;     // n_states x n doubles: a caller's initial state (allocated on first use)
    void* probe = nullptr;     // probe node indices then values (daeti_read_v_nodes)
    int64_t probe_cap = 0;     // probes the buffer holds
    std::vector<double> mass;  // lumped mass per node (host, FP64)
    double kref[64];           // unit-D element stiffness of a grid element (adjoint)
    struct AdjointBuffers* adj = nullptr;   // adjoint work buffers (adjoint.cu)
    int64_t adj_fwd_steps = 0;              // forward steps run by the last adjoint call
    std::vector<void*> allocs;
    // launch shapes
    ReactTuning rtune;
    int diff_block = 256;       // 0: shared-memory tiles on structured grids
    int diff_rows = 0;          // nodes per thread along y of the 3D structured kernel (0 = 2, 2 or 4)
    bool fused = true;          // last sub-step of step I inside the reaction launch
    bool lists = true;
    int graph_steps = 20;
    std::vector<StimDev> stim_dev;   // host copy of the device stimulus table
    // graphs of graph_steps steps, keyed by (start V buffer, list parity,
    // stimulus-free segment)
    cudaGraphExec_t graphs[8] = {};
    // profiling: 1 = events around plain launches; 2 = event-record nodes
    // around every launch inside captured graphs (graph_steps > 0)
    int prof = 0;
    bool gcap = false;                  // capturing a profiling graph
    int gnext = 0;                      // next event of the capture
    std::vector<cudaEvent_t> gev;       // begin/end event of each launch of a profiling graph
    std::vector<int> gwhich;            // kernel class of each begin/end pair
    cudaGraphExec_t pgraphs[8] = {};    // profiling graphs, keyed like graphs
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double ktime[3] = {0, 0, 0};
    int64_t klaunch[3] = {0, 0, 0};
};

namespace daeti_host {

int fail(daeti_ctx* c, int code, const std::string& msg);
cudaError_t cpy_(daeti_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind);
cudaError_t set_(daeti_ctx* c, void* dst, int v, size_t bytes);
int dalloc(daeti_ctx* c, void** p, size_t bytes);
size_t rsize(const daeti_ctx* c);
int upload_real(daeti_ctx* c, void* dst, const double* src, int64_t count);
void free_adjoint(daeti_ctx* c);
void drop_adjoint_graph(daeti_ctx* c);   // the captured gradient sweep (kernel arguments changed)
// Nodes of element e (returns their count); element means of a nodal field.
int elem_nodes(const daeti_ctx* c, int64_t e, int64_t* out);
void elem_means(const daeti_ctx* c, const double* nodal, std::vector<double>& out);
extern const double TP06_INIT[19];   // published TP06 initial state (state order of cells.cuh)

}  // namespace daeti_host

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return daeti_host::fail(c, e_ == cudaErrorMemoryAllocation ? DAETI_ENOMEM : DAETI_ECUDA, \
                                    std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)
