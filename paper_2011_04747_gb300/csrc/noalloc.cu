// Allocation-free stable-step estimate for structured grids.
//
// Some callers cannot call cudaMalloc: code that runs inside a host that
// owns all device memory through its own pool or budget, plugins loaded into
// an application that forbids device allocation after start-up, and code
// paths that must not trigger the implicit synchronisation a cudaMalloc or
// cudaFree can cause.  daeti_grid_stability_noalloc gives them the FP64
// stable-step estimate (the Gershgorin bound and the Lanczos lambda_max that
// daeti_prepare computes, through the same table builder and estimator
// routines) without any device allocation: its work vectors live in one
// file-scope __device__ array of fixed size that every GPU which loads the
// library holds until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/daeti.h"
#include "assembly.h"
#include "kernels.h"

using namespace daeti;

namespace {

constexpr int64_t kMaxNodes = DAETI_NOALLOC_MAX_NODES;
constexpr int kMaxLayers = DAETI_NOALLOC_MAX_LAYERS;      // node layers in z (1 in 2D)
constexpr int64_t kMaxClasses = (int64_t)kMaxLayers * 9;
// scratch layout (doubles): K table | mass table | node mass | 3 Lanczos
// vectors | Lanczos coefficients | Gershgorin bits
constexpr int kMaxIt = DAETI_LANCZOS_MAX_IT;
constexpr int64_t kOffK = 0;
constexpr int64_t kOffMt = kOffK + kMaxClasses * 27;
constexpr int64_t kOffM = kOffMt + kMaxClasses;
constexpr int64_t kOffV = kOffM + kMaxNodes;
constexpr int64_t kOffHist = kOffV + 3 * kMaxNodes;
constexpr int64_t kOffBits = kOffHist + 4 * (kMaxIt + 1);
constexpr int64_t kScratchDoubles = kOffBits + 2;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Host-side staging (file scope: no heap, guarded by g_mu).
double h_layer_k[kMaxLayers * 64];
double h_table[kMaxClasses * 27];
double h_mass[kMaxClasses];
double h_coef[4 * kMaxIt];

std::mutex g_mu;
double* g_scratch_addr[128] = {nullptr};

void set_err(char* buf, int len, const char* msg) {
    if (buf && len > 0) std::snprintf(buf, (size_t)len, "%s", msg);
}

// Device address of the scratch array for the current device (set up once per device).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int daeti_grid_stability_noalloc(int dim, const int64_t n[3], double h, int64_t n_elem,
                                            const double* d_long, const double* d_trans, const double* fibre,
                                            void* stream, double* dt_s, double* lambda_max, char* errbuf,
                                            int errbuf_len) {
    set_err(errbuf, errbuf_len, "");
    if ((dim != 2 && dim != 3) || !n || !(h > 0) || !d_long || !dt_s || !lambda_max) {
        set_err(errbuf, errbuf_len, "bad arguments");
        return DAETI_EINVAL;
    }
    const int64_t nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
    if (nx < 2 || ny < 2 || nz < 1 || (dim == 3 && nz < 2)) {
        set_err(errbuf, errbuf_len, "grid needs >= 2 nodes per axis");
        return DAETI_EINVAL;
    }
    const int64_t n_nodes = nx * ny * nz;
    if (n_nodes > kMaxNodes || nz > kMaxLayers) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "grid of %lld nodes / %lld layers exceeds the fixed scratch (%lld nodes, %d layers)",
                      (long long)n_nodes, (long long)nz, (long long)kMaxNodes, kMaxLayers);
        set_err(errbuf, errbuf_len, msg);
        return DAETI_EINVAL;
    }
    const int64_t ex_n = nx - 1, ey_n = ny - 1, ez_n = dim == 3 ? nz - 1 : 1;
    if (n_elem != ex_n * ey_n * ez_n) {
        set_err(errbuf, errbuf_len, "n_elem does not match the grid");
        return DAETI_EINVAL;
    }
    // the call synchronises the stream and reads its results on the host,
    // neither of which a capturing stream allows
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t qe = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (qe != cudaSuccess) cudaGetLastError();
    if (qe != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        set_err(errbuf, errbuf_len, "stream is capturing (or its capture status is unavailable)");
        return DAETI_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);

    for (int64_t e = 0; e < n_elem; ++e) {
        const double a = d_long[e], b = d_trans ? d_trans[e] : d_long[e];
        if (!(a >= 0) || !(b >= 0) || !std::isfinite(a) || !std::isfinite(b)) {
            set_err(errbuf, errbuf_len, "conductivities must be finite and >= 0");
            return DAETI_EINVAL;
        }
    }
    // stencil table per node class (z layer, y class, x class) and lumped
    // mass, by the builder daeti_prepare uses; D must be constant within each
    // element layer
    if (!grid_layer_stiffness(dim, n, h, d_long, d_trans, fibre, h_layer_k)) {
        set_err(errbuf, errbuf_len, "conductivity varies within an element layer (not supported here)");
        return DAETI_EUNSUPPORTED;
    }
    const int64_t ncls = nz * 9;
    grid_class_table(dim, n, h, h_layer_k, h_table, h_mass);

    double* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_err(errbuf, errbuf_len, cudaGetErrorString(e));
        return DAETI_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* ktab = base + kOffK;
    double* mtab = base + kOffMt;
    double* m = base + kOffM;
    double* const v[3] = {base + kOffV, base + kOffV + kMaxNodes, base + kOffV + 2 * kMaxNodes};
    double* hist = base + kOffHist;
    unsigned long long* bits = (unsigned long long*)(base + kOffBits);
    EstOp est;
    est.kind = 0;
    est.dim = dim;
    est.nx = (int)nx;
    est.ny = (int)ny;
    est.nz = (int)nz;
    est.n = n_nodes;
    est.ktab = ktab;
    est.mtab = mtab;
    est.m = m;

#define NA_CK(call)                                                       \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) {                                          \
            set_err(errbuf, errbuf_len, cudaGetErrorString(e_));          \
            return DAETI_ECUDA;                                           \
        }                                                                 \
    } while (0)

    NA_CK(cudaMemcpyAsync(ktab, h_table, sizeof(double) * ncls * 27, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(mtab, h_mass, sizeof(double) * ncls, cudaMemcpyHostToDevice, st));
    const double big = 1e300;
    unsigned long long hb;
    std::memcpy(&hb, &big, 8);
    NA_CK(cudaMemcpyAsync(bits, &hb, 8, cudaMemcpyHostToDevice, st));
    NA_CK(cudaStreamSynchronize(st));   // host staging buffers may be reused after this
    launch_gershgorin(est, bits, st);
    launch_node_mass(est, m, st);
    NA_CK(cudaMemcpyAsync(&hb, bits, 8, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    double mn;
    std::memcpy(&mn, &hb, 8);
    *dt_s = 0.9 * mn;

    // lambda_max(M_L^-1 K) by the Lanczos routine daeti_prepare uses
    double lam = 0.0;
    int iters = 0;
    NA_CK(lanczos_lambda_max(est, m, v, hist, h_coef, kMaxIt, st, &lam, &iters));
    NA_CK(cudaStreamSynchronize(st));
    NA_CK(cudaGetLastError());
    *lambda_max = lam;
    return DAETI_OK;
#undef NA_CK
}
