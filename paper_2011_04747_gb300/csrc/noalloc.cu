// Allocation-free stable-step estimate for structured grids.
//
// Some callers cannot call cudaMalloc: code that runs inside a host that
// owns all device memory through its own pool or budget, plugins loaded into
// an application that forbids device allocation after start-up, and code
// paths that must not trigger the implicit synchronisation a cudaMalloc or
// cudaFree can cause.  daeti_grid_stability_noalloc gives them the FP64
// stable-step estimate (the Gershgorin bound and the power-iteration
// lambda_max that daeti_prepare computes) without any device allocation: its
// work vectors live in one file-scope __device__ array of fixed size that
// every GPU which loads the library holds until the process exits.
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
// scratch layout (doubles): K table | mass table | node mass | x | y | dots[2] | Gershgorin bits
constexpr int64_t kOffK = 0;
constexpr int64_t kOffMt = kOffK + kMaxClasses * 27;
constexpr int64_t kOffM = kOffMt + kMaxClasses;
constexpr int64_t kOffX = kOffM + kMaxNodes;
constexpr int64_t kOffY = kOffX + kMaxNodes;
constexpr int64_t kOffDots = kOffY + kMaxNodes;
constexpr int64_t kOffBits = kOffDots + 2;
constexpr int64_t kScratchDoubles = kOffBits + 2;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Host-side staging for the stencil tables (file scope: no heap, guarded by g_mu).
double h_layer_k[kMaxLayers][64];
double h_table[kMaxClasses * 27];
double h_mass[kMaxClasses];

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

// x_i of the power iteration's start vector: the i-th draw of the same 64-bit
// LCG the context path uses (advanced to position i by squaring its affine map).
__global__ void start_vector_kernel(int64_t n, int nx, int ny, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long A = 6364136223846793005ull, C = 1442695040888963407ull;
    unsigned long long ra = 1ull, rc = 0ull;        // accumulated map s -> ra s + rc
    unsigned long long pa = A, pc = C;              // map raised to the current power of two
    unsigned long long m = (unsigned long long)i + 1ull;
    while (m) {
        if (m & 1ull) {
            rc = pa * rc + pc;
            ra = pa * ra;
        }
        pc = pa * pc + pc;
        pa = pa * pa;
        m >>= 1;
    }
    const unsigned long long st = ra * 0x9E3779B97F4A7C15ull + rc;
    const double u = (double)(st >> 11) * (1.0 / 9007199254740992.0);
    const int64_t xx = i % nx, yy = (i / nx) % ny, zz = i / ((int64_t)nx * ny);
    const double sgn = ((xx + yy + zz) & 1) ? -1.0 : 1.0;
    x[i] = sgn * (1.0 + 0.1 * u);
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
    const int nl = 1 << dim;
    std::lock_guard<std::mutex> lock(g_mu);

    // element stiffness per layer; D must be constant within each element layer
    const int64_t per_layer = ex_n * ey_n;
    for (int64_t ez = 0; ez < ez_n; ++ez) {
        double D0[9];
        const int64_t e0 = ez * per_layer;
        conductivity_tensor(d_long[e0], d_trans ? d_trans[e0] : d_long[e0], fibre ? fibre + 3 * e0 : nullptr, dim, D0);
        for (int64_t e = e0; e < e0 + per_layer; ++e) {
            double D[9];
            const double a = d_long[e], b = d_trans ? d_trans[e] : d_long[e];
            if (!(a >= 0) || !(b >= 0) || !std::isfinite(a) || !std::isfinite(b)) {
                set_err(errbuf, errbuf_len, "conductivities must be finite and >= 0");
                return DAETI_EINVAL;
            }
            conductivity_tensor(a, b, fibre ? fibre + 3 * e : nullptr, dim, D);
            for (int r = 0; r < 9; ++r)
                if (D[r] != D0[r]) {
                    set_err(errbuf, errbuf_len, "conductivity varies within an element layer (not supported here)");
                    return DAETI_EUNSUPPORTED;
                }
        }
        box_stiffness(dim, h, D0, h_layer_k[ez]);
    }
    // stencil table per node class (z layer, y class, x class) and lumped mass
    const int64_t ncls = nz * 9;
    std::memset(h_table, 0, sizeof(double) * ncls * 27);
    std::memset(h_mass, 0, sizeof(double) * ncls);
    const double emass = std::pow(h, dim) / nl;
    for (int64_t z = 0; z < nz; ++z)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                const int64_t cls = (z * 3 + cy) * 3 + cx;
                for (int oz = (dim == 3 ? -1 : 0); oz <= 0; ++oz) {
                    const int64_t ez = z + oz;
                    if (dim == 3 && (ez < 0 || ez >= ez_n)) continue;
                    const int64_t layer = dim == 3 ? ez : 0;
                    for (int oy = -1; oy <= 0; ++oy) {
                        if ((oy == -1 && cy == 0) || (oy == 0 && cy == 2)) continue;
                        for (int ox = -1; ox <= 0; ++ox) {
                            if ((ox == -1 && cx == 0) || (ox == 0 && cx == 2)) continue;
                            const int a = (-ox) | ((-oy) << 1) | ((dim == 3 ? -oz : 0) << 2);
                            for (int b = 0; b < nl; ++b) {
                                const int dx = ox + (b & 1), dy = oy + ((b >> 1) & 1);
                                const int dz = dim == 3 ? oz + ((b >> 2) & 1) : 0;
                                h_table[cls * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] += h_layer_k[layer][a * nl + b];
                            }
                            h_mass[cls] += emass;
                        }
                    }
                }
            }

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
    double* x = base + kOffX;
    double* y = base + kOffY;
    double* dots = base + kOffDots;
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

    // power iteration for lambda_max(M_L^-1 K), as in daeti_prepare
    start_vector_kernel<<<(unsigned)((n_nodes + 255) / 256), 256, 0, st>>>(n_nodes, (int)nx, (int)ny, x);
    double hd[2];
    NA_CK(cudaMemsetAsync(dots, 0, sizeof(double) * 2, st));
    launch_mdots(n_nodes, m, x, x, dots, st);
    NA_CK(cudaMemcpyAsync(hd, dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    launch_scale(n_nodes, x, 1.0 / std::sqrt(hd[1]), x, st);
    double lam = 0.0, prev = 0.0;
    for (int it = 0; it < 500; ++it) {
        launch_apply_minvk(est, x, y, st);
        NA_CK(cudaMemsetAsync(dots, 0, sizeof(double) * 2, st));
        launch_mdots(n_nodes, m, x, y, dots, st);
        NA_CK(cudaMemcpyAsync(hd, dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        lam = hd[0];
        if (!(hd[1] > 0)) break;
        launch_scale(n_nodes, y, 1.0 / std::sqrt(hd[1]), x, st);
        if (it > 5 && std::fabs(lam - prev) <= 1e-8 * std::fabs(lam)) break;
        prev = lam;
    }
    NA_CK(cudaStreamSynchronize(st));
    NA_CK(cudaGetLastError());
    *lambda_max = lam;
    return DAETI_OK;
#undef NA_CK
}
