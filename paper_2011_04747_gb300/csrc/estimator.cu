// FP64 stable-step estimator: Eq. 3's Gershgorin bound
//   dt_s = 0.9 min_i m_ii / (k_ii + sum_{j != i} |k_ij|)
// as a grid-wide min-reduction over rows, and the building blocks of a power
// iteration for lambda_max(M_L^-1 K) (apply, M-weighted dot products,
// scaling).  Also the state/dtype conversion used by the read functions and
// the initial state written in the device layout.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace daeti {

__device__ __forceinline__ void class_of(int i, int nx, int ny, int& x, int& y, int& z, int& cls) {
    x = i % nx;
    const int yz = i / nx;
    y = yz % ny;
    z = yz / ny;
    const int cx = x == 0 ? 0 : (x == nx - 1 ? 2 : 1);
    const int cy = y == 0 ? 0 : (y == ny - 1 ? 2 : 1);
    cls = (z * 3 + cy) * 3 + cx;
}

// Non-negative doubles order like their bit patterns, so an integer atomicMin works.
__device__ __forceinline__ void block_min_to(double v, unsigned long long* out) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 1e300;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomicMin(out, (unsigned long long)__double_as_longlong(v));
    }
}

__global__ void gersh_table_kernel(EstOp op, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 1e300;
    if (i < op.n) {
        int x, y, z, cls;
        class_of(i, op.nx, op.ny, x, y, z, cls);
        const double* kr = op.ktab + (size_t)cls * 27;
        const int self = op.dim == 3 ? 13 : 4;
        double s = kr[self];
        for (int j = 0; j < 27; ++j)
            if (j != self) s += fabs(kr[j]);
        if (s > 0.0) v = op.mtab[cls] / s;
    }
    block_min_to(v, out);
}

__global__ void gersh_sell_kernel(EstOp op, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 1e300;
    if (i < op.n) {
        const int chunk = i >> 5, lane = i & 31;
        const int64_t off = op.chunk_ptr[chunk] + lane;
        double s = op.kdiag[i];
        for (int j = 0; j < op.chunk_w[chunk]; ++j) s += fabs(op.kval[off + 32 * (int64_t)j]);
        if (s > 0.0) v = op.m[i] / s;
    }
    block_min_to(v, out);
}

void launch_gershgorin(const EstOp& op, unsigned long long* out_bits, cudaStream_t st) {
    const int block = 256;
    const int grid = (int)((op.n + block - 1) / block);
    if (op.kind == 0)
        gersh_table_kernel<<<grid, block, 0, st>>>(op, out_bits);
    else
        gersh_sell_kernel<<<grid, block, 0, st>>>(op, out_bits);
}

// y = M_L^-1 K x in FP64.
__global__ void apply_table_kernel(EstOp op, const double* __restrict__ x, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= op.n) return;
    int cx_, cy_, z, cls;
    class_of(i, op.nx, op.ny, cx_, cy_, z, cls);
    const int cx = cx_ == 0 ? 0 : (cx_ == op.nx - 1 ? 2 : 1);
    const int cy = cy_ == 0 ? 0 : (cy_ == op.ny - 1 ? 2 : 1);
    const double* kr = op.ktab + (size_t)cls * 27;
    const int nxy = op.nx * op.ny;
    double acc = 0.0;
    const int zlo = op.dim == 3 ? -1 : 0, zhi = op.dim == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const bool ok = (dx >= 0 || cx > 0) && (dx <= 0 || cx < 2) && (dy >= 0 || cy > 0) &&
                                (dy <= 0 || cy < 2) && (dz >= 0 || z > 0) && (dz <= 0 || z < op.nz - 1);
                if (!ok) continue;
                const int j = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                acc += kr[j] * x[i + dx + dy * op.nx + dz * nxy];
            }
    y[i] = acc / op.mtab[cls];
}

__global__ void apply_sell_kernel(EstOp op, const double* __restrict__ x, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= op.n) return;
    const int chunk = i >> 5, lane = i & 31;
    const int64_t off = op.chunk_ptr[chunk] + lane;
    double acc = op.kdiag[i] * x[i];
    for (int j = 0; j < op.chunk_w[chunk]; ++j) {
        const int64_t e = off + 32 * (int64_t)j;
        acc += op.kval[e] * x[op.col[e]];
    }
    y[i] = acc / op.m[i];
}

void launch_apply_minvk(const EstOp& op, const double* x, double* y, cudaStream_t st) {
    const int block = 256;
    const int grid = (int)((op.n + block - 1) / block);
    if (op.kind == 0)
        apply_table_kernel<<<grid, block, 0, st>>>(op, x, y);
    else
        apply_sell_kernel<<<grid, block, 0, st>>>(op, x, y);
}

// out2[0] += sum m x y, out2[1] += sum m y y
__global__ void mdots_kernel(int64_t n, const double* __restrict__ m, const double* __restrict__ x,
                             const double* __restrict__ y, double* out2) {
    __shared__ double sh[2][32];
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a += m[i] * x[i] * y[i];
        b += m[i] * y[i] * y[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < (int)(blockDim.x >> 5) ? sh[0][lane] : 0.0;
        b = lane < (int)(blockDim.x >> 5) ? sh[1][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            atomicAdd(&out2[0], a);
            atomicAdd(&out2[1], b);
        }
    }
}

void launch_mdots(int64_t n, const double* m, const double* x, const double* y, double* out2, cudaStream_t st) {
    int grid = (int)((n + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    mdots_kernel<<<grid, 256, 0, st>>>(n, m, x, y, out2);
}

// ------------------------------------------------------------ Lanczos estimate
// lambda_max of M_L^-1 K, which is self-adjoint in the M_L inner product
// <u, v> = sum_i m_i u_i v_i: Lanczos in that inner product builds the
// tridiagonal T_j (diagonal alpha, off-diagonal beta) whose largest
// eigenvalue approaches lambda_max from below.  Plain power iteration
// converges as (lambda_2/lambda_1)^(2j), which on structured grids (top
// eigenvalues a relative O(h^2) apart) leaves a relative error of 1e-4..1e-3
// after 500 iterations; the largest Ritz value converges to rounding within a
// few hundred iterations on the same grids.

// Start vector: x_i from the i-th draw u_i in [0, 1) of the 64-bit linear
// congruential generator s <- A s + C (s_0 = 0x9E3779B97F4A7C15; u = the top
// 53 bits of s_{i+1} / 2^53), reached by raising the affine map to the power
// i + 1 (square and multiply).  Structured grids: the checkerboard
// (-1)^(x+y+z) (1 + 0.1 u), close to the highest-frequency mode; otherwise
// u - 0.5.
__global__ void start_vector_kernel(int64_t n, int kind, int nx, int ny, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long A = 6364136223846793005ull, C = 1442695040888963407ull;
    unsigned long long ra = 1ull, rc = 0ull;   // accumulated map s -> ra s + rc
    unsigned long long pa = A, pc = C;         // the map raised to the current power of two
    unsigned long long e = (unsigned long long)i + 1ull;
    while (e) {
        if (e & 1ull) {
            rc = pa * rc + pc;
            ra = pa * ra;
        }
        pc = pa * pc + pc;
        pa = pa * pa;
        e >>= 1;
    }
    const unsigned long long s = ra * 0x9E3779B97F4A7C15ull + rc;
    const double u = (double)(s >> 11) * (1.0 / 9007199254740992.0);
    if (kind == 0) {
        const int64_t xx = i % nx, yy = (i / nx) % ny, zz = i / ((int64_t)nx * ny);
        x[i] = (((xx + yy + zz) & 1) ? -1.0 : 1.0) * (1.0 + 0.1 * u);
    } else {
        x[i] = u - 0.5;
    }
}

// x = y / sqrt(*nrm2) with the squared norm read from device memory.
__global__ void scale_by_norm_kernel(int64_t n, const double* __restrict__ y, const double* nrm2, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = y[i] * (1.0 / sqrt(*nrm2));
}

// Three-term recurrence: y -= alpha x + beta xp (alpha = h[0], beta =
// sqrt(hp[2]), 0 for the first vector), then h[2] += <y, y>_M.
__global__ void lanczos_update_kernel(int64_t n, const double* __restrict__ m, const double* __restrict__ x,
                                      const double* __restrict__ xp, double* __restrict__ y, double* h,
                                      const double* hp) {
    __shared__ double sh[32];
    const double alpha = h[0];
    const double beta = hp ? sqrt(hp[2]) : 0.0;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = y[i] - alpha * x[i];
        if (hp) v -= beta * xp[i];
        y[i] = v;
        acc += m[i] * v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = acc;
    __syncthreads();
    if (w == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(&h[2], acc);
    }
}

double tridiag_max_eig(const double* a, const double* b2, int stride, int k) {
    if (k <= 0) return 0.0;
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::sqrt(b2[(i - 1) * stride]) : 0.0) + (i < k - 1 ? std::sqrt(b2[i * stride]) : 0.0);
        const double ai = a[i * stride];
        lo = i ? std::min(lo, ai - r) : ai - r;
        hi = i ? std::max(hi, ai + r) : ai + r;
    }
    // number of eigenvalues below x: negative pivots of T - x I = L D L^T
    auto below = [&](double x) {
        int c = 0;
        double d = 1.0;
        for (int i = 0; i < k; ++i) {
            d = a[i * stride] - x - (i > 0 ? b2[(i - 1) * stride] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++c;
        }
        return c;
    };
    for (int it = 0; it < 2000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (below(mid) == k) hi = mid;
        else lo = mid;
    }
    return hi;
}

cudaError_t lanczos_lambda_max(const EstOp& est, const double* m, double* const v[3], double* hist, double* hh,
                               int max_it, cudaStream_t st, double* lam, int* iters) {
    const int64_t n = est.n;
    *lam = 0.0;
    if (iters) *iters = 0;
    if (n <= 0 || max_it < 1) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(double) * 4 * (size_t)(max_it + 1), st);
    if (e != cudaSuccess) return e;
    const int grid = (int)((n + 255) / 256);
    const int rgrid = std::min(grid, 152 * 8);
    double* xp = v[0];
    double* x = v[1];
    double* y = v[2];
    start_vector_kernel<<<grid, 256, 0, st>>>(n, est.kind == 0 ? 0 : 1, est.nx, est.ny, x);
    launch_mdots(n, m, x, x, hist, st);   // hist[1] = <x, x>_M
    scale_by_norm_kernel<<<grid, 256, 0, st>>>(n, x, hist + 1, x);
    double* h = hist + 4;                   // iteration j: h[4j] alpha_j, h[4j + 2] beta_j^2
    const int B = 32;                       // iterations between host checks
    double theta = 0.0, prev = 0.0;
    bool have_prev = false;
    int j = 0;
    while (j < max_it) {
        const int jb = std::min(max_it, j + B);
        for (; j < jb; ++j) {
            launch_apply_minvk(est, x, y, st);
            launch_mdots(n, m, x, y, h + 4 * j, st);
            lanczos_update_kernel<<<rgrid, 256, 0, st>>>(n, m, x, xp, y, h + 4 * j, j > 0 ? h + 4 * (j - 1) : nullptr);
            scale_by_norm_kernel<<<grid, 256, 0, st>>>(n, y, h + 4 * j + 2, xp);   // next vector, into xp's buffer
            std::swap(xp, x);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(hh, h, sizeof(double) * 4 * (size_t)j, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        // T_k: stop at a breakdown (beta_i ~ 0: the Krylov space is invariant,
        // T_{i+1} holds eigenvalues exactly)
        int k = j;
        bool stop = false;
        double amax = 0.0;
        for (int i = 0; i < j; ++i) {
            amax = std::max(amax, std::fabs(hh[4 * i]));
            const double b2 = hh[4 * i + 2];
            if (!std::isfinite(hh[4 * i])) {
                k = i;
                stop = true;
                break;
            }
            if (!(b2 > 1e-24 * amax * amax) || !std::isfinite(b2)) {
                k = i + 1;
                stop = true;
                break;
            }
        }
        theta = tridiag_max_eig(hh, hh + 2, 4, k);
        if (iters) *iters = k;
        if (stop || (have_prev && std::fabs(theta - prev) <= 1e-13 * std::fabs(theta))) break;
        prev = theta;
        have_prev = true;
    }
    *lam = theta;
    return cudaSuccess;
}

__global__ void node_mass_kernel(EstOp op, double* m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= op.n) return;
    int x, y, z, cls;
    class_of(i, op.nx, op.ny, x, y, z, cls);
    m[i] = op.mtab[cls];
}

void launch_node_mass(const EstOp& op, double* m_out, cudaStream_t st) {
    const int grid = (int)((op.n + 255) / 256);
    if (grid) node_mass_kernel<<<grid, 256, 0, st>>>(op, m_out);
}

// dst = src (- comp), converted to double or float.
template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, const float* __restrict__ comp, D* __restrict__ dst,
                               int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = (double)src[i];
    if (comp) v -= (double)comp[i];
    dst[i] = (D)v;
}

void launch_convert(const void* src, int src_prec, const float* comp, void* dst, int dst_f32, int64_t n,
                    cudaStream_t st) {
    const int grid = (int)((n + 255) / 256);
    if (!grid) return;
    if (src_prec == P_F64) {
        if (dst_f32) convert_kernel<double, float><<<grid, 256, 0, st>>>((const double*)src, comp, (float*)dst, n);
        else convert_kernel<double, double><<<grid, 256, 0, st>>>((const double*)src, comp, (double*)dst, n);
    } else {
        if (dst_f32) convert_kernel<float, float><<<grid, 256, 0, st>>>((const float*)src, comp, (float*)dst, n);
        else convert_kernel<float, double><<<grid, 256, 0, st>>>((const float*)src, comp, (double*)dst, n);
    }
}

// dst[j] = V(nodes[j]) (- comp), as double.
template <typename S>
__global__ void gather_v_kernel(const S* __restrict__ src, const float* __restrict__ comp,
                                const int64_t* __restrict__ nodes, double* __restrict__ dst, int64_t m) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t i = nodes[j];
    double v = (double)src[i];
    if (comp) v -= (double)comp[i];
    dst[j] = v;
}

void launch_gather_v(const void* src, int src_prec, const float* comp, const int64_t* nodes, double* dst, int64_t m,
                     cudaStream_t st) {
    const int grid = (int)((m + 127) / 128);
    if (!grid) return;
    if (src_prec == P_F64) gather_v_kernel<double><<<grid, 128, 0, st>>>((const double*)src, comp, nodes, dst, m);
    else gather_v_kernel<float><<<grid, 128, 0, st>>>((const float*)src, comp, nodes, dst, m);
}

// dst[i] = state s of node i from the chunked state array (state_index), as double.
template <typename S>
__global__ void gather_state_kernel(const S* __restrict__ src, int ns, int s, double* __restrict__ dst, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = (double)src[((i >> 5) * ns + s) * 32 + (i & 31)];
}

void launch_gather_state(const void* src, int src_prec, int ns, int s, double* dst, int64_t n, cudaStream_t st) {
    const int grid = (int)((n + 255) / 256);
    if (!grid) return;
    if (src_prec == P_F64) gather_state_kernel<double><<<grid, 256, 0, st>>>((const double*)src, ns, s, dst, n);
    else gather_state_kernel<float><<<grid, 256, 0, st>>>((const float*)src, ns, s, dst, n);
}

// Initial state (one thread per node, the last chunk's lanes past n included):
// state k of node i from src[k * n + i] (or def.v[k] when src is null).
template <typename R>
__global__ void init_state_kernel(const double* __restrict__ src, InitDefaults def, int64_t n, int ns, R* V, R* vsync,
                                  R* S, R* act, float* c0, float* c1) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nsx = ns - 1;
    if (i >= ((n + 31) & ~(int64_t)31)) return;
    const bool in = i < n;
    for (int k = 1; k < ns; ++k) {
        const double x = in ? (src ? src[(int64_t)k * n + i] : def.v[k]) : 0.0;
        S[((i >> 5) * nsx + (k - 1)) * 32 + (i & 31)] = (R)x;
    }
    if (!in) return;
    const R v = (R)(src ? src[i] : def.v[0]);
    V[i] = v;
    vsync[i] = v;
    act[i] = (R)-1;
    if (c0) c0[i] = 0.f;
    if (c1) c1[i] = 0.f;
}

__global__ void check_finite_kernel(const double* __restrict__ x, int64_t n, int* flag) {
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

void launch_init_state(const double* src, const InitDefaults& def, int64_t n, int ns, int prec, void* V, void* vsync,
                       void* S, void* act, float* c0, float* c1, cudaStream_t st) {
    const int64_t lanes = (n + 31) & ~(int64_t)31;
    const int grid = (int)((lanes + 255) / 256);
    if (!grid) return;
    if (prec == P_F64)
        init_state_kernel<double><<<grid, 256, 0, st>>>(src, def, n, ns, (double*)V, (double*)vsync, (double*)S,
                                                        (double*)act, c0, c1);
    else
        init_state_kernel<float><<<grid, 256, 0, st>>>(src, def, n, ns, (float*)V, (float*)vsync, (float*)S,
                                                       (float*)act, c0, c1);
}

void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t st) {
    if (n <= 0) return;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * 152);
    check_finite_kernel<<<grid, 256, 0, st>>>(x, n, flag);
}

}  // namespace daeti
