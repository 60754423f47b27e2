// Steps I/III (step B) of Section 2: explicit Euler sub-steps of length
// dt_ad = dt/(2l) on M_L dV/dt = -K V, i.e. V <- V - dt_ad M_L^-1 K V.
// Rows of K sum to zero, so (K V)_i = sum_{j != i} k_ij (V_j - V_i); the
// kernels apply that form with the pre-scaled off-diagonal coefficients
// a_ij = dt_ad k_ij / m_i, which keeps the float differences exact for
// neighbouring nodes.  Two layouts:
//   * structured grids: a 9-point (2D) / 27-point (3D) stencil whose
//     coefficients depend only on the node's z layer and its x/y boundary
//     class (table [nz][3][3][27]); used when D varies at most with z;
//   * any mesh: SELL-32 sparse rows (chunks of 32 rows, column-major).
// The launch that ends a diffusion half at t_n also runs the synchronisation
// epilogue (activation time, k of the next step A, k histogram).
#include "common.cuh"
#include "kernels.h"

namespace daeti {

template <typename R>
struct StencilArgs {
    int n, nx, ny, nz;
    const R* vin;
    R* vout;
    const float* cin;
    float* cout;
    const R* coef;
};

template <typename R, int DIM, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(256) stencil_kernel(StencilArgs<R> a, SyncParams<R> sp) {
    __shared__ int hist[DAETI_MAX_K];
    if (SYNC) {
        if (threadIdx.x < DAETI_MAX_K) hist[threadIdx.x] = 0;
        __syncthreads();
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.n;
    int k = 0;
    if (valid) {
        const int x = i % a.nx;
        const int yz = i / a.nx;
        const int y = yz % a.ny;
        const int z = yz / a.ny;
        const int cx = x == 0 ? 0 : (x == a.nx - 1 ? 2 : 1);
        const int cy = y == 0 ? 0 : (y == a.ny - 1 ? 2 : 1);
        const R* c = a.coef + ((size_t)(z * 3 + cy) * 3 + cx) * 27;
        const R vi = a.vin[i];
        const int nxy = a.nx * a.ny;
        R acc = (R)0;
#pragma unroll
        for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0 && dz == 0) continue;
                    const bool ok = (dx >= 0 || cx > 0) && (dx <= 0 || cx < 2) && (dy >= 0 || cy > 0) &&
                                    (dy <= 0 || cy < 2) &&
                                    (DIM == 2 || ((dz >= 0 || z > 0) && (dz <= 0 || z < a.nz - 1)));
                    if (ok) {
                        const int j = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                        acc += __ldg(c + j) * (a.vin[i + dx + dy * a.nx + dz * nxy] - vi);
                    }
                }
            }
        }
        R v = vi;
        float cc = KAHAN ? a.cin[i] : 0.f;
        add_comp(v, KAHAN ? &cc : (float*)nullptr, -acc);
        a.vout[i] = v;
        if (KAHAN) a.cout[i] = cc;
        if (SYNC) k = sync_node(sp, i, v);
    }
    if (SYNC) {
        if (sp.counts) {
            warp_count(hist, k, valid);
            __syncthreads();
            if (threadIdx.x < DAETI_MAX_K && hist[threadIdx.x]) atomicAdd(&sp.counts[threadIdx.x], hist[threadIdx.x]);
        }
    }
}

template <typename R>
struct SellArgs {
    int n;
    const R* vin;
    R* vout;
    const float* cin;
    float* cout;
    const int64_t* chunk_ptr;
    const int* chunk_w;
    const int* col;
    const R* val;
};

template <typename R, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(256) sell_kernel(SellArgs<R> a, SyncParams<R> sp) {
    __shared__ int hist[DAETI_MAX_K];
    if (SYNC) {
        if (threadIdx.x < DAETI_MAX_K) hist[threadIdx.x] = 0;
        __syncthreads();
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.n;
    int k = 0;
    if (valid) {
        const int chunk = i >> 5;
        const int lane = i & 31;
        const int64_t off = a.chunk_ptr[chunk] + lane;
        const int w = a.chunk_w[chunk];
        const R vi = a.vin[i];
        R acc = (R)0;
        for (int j = 0; j < w; ++j) {
            const int cj = __ldg(a.col + off + 32 * (int64_t)j);
            const R aj = __ldg(a.val + off + 32 * (int64_t)j);
            acc += aj * (a.vin[cj] - vi);
        }
        R v = vi;
        float cc = KAHAN ? a.cin[i] : 0.f;
        add_comp(v, KAHAN ? &cc : (float*)nullptr, -acc);
        a.vout[i] = v;
        if (KAHAN) a.cout[i] = cc;
        if (SYNC) k = sync_node(sp, i, v);
    }
    if (SYNC) {
        if (sp.counts) {
            warp_count(hist, k, valid);
            __syncthreads();
            if (threadIdx.x < DAETI_MAX_K && hist[threadIdx.x]) atomicAdd(&sp.counts[threadIdx.x], hist[threadIdx.x]);
        }
    }
}

template <typename R, bool KAHAN>
static void diff_typed(const DevState& s, const DiffOp& op, int src, bool sync, int par, const SyncArgs& sa,
                       StepRef step, bool count, int block, cudaStream_t st) {
    SyncParams<R> sp;
    sp.vsync = (R*)s.vsync;
    sp.kk = s.kk;
    sp.act = (R*)s.act;
    sp.counts = count ? s.counts + par * DAETI_MAX_K : nullptr;
    sp.flags = s.flags;
    sp.dt = sa.dt;
    sp.vscale = (R)sa.vscale;
    sp.vth = (R)sa.vth;
    sp.kmax = sa.kmax;
    sp.adaptive = sa.adaptive;
    sp.step = step;
    if (block <= 0) block = 256;
    const int grid = (int)((s.n + block - 1) / block);
    if (grid == 0) return;
    const R* vin = (const R*)s.V[src];
    R* vout = (R*)s.V[1 - src];
    const float* cin = KAHAN ? s.C[src] : nullptr;
    float* cout = KAHAN ? s.C[1 - src] : nullptr;
    if (op.kind == 0) {
        StencilArgs<R> a{(int)s.n, op.nx, op.ny, op.nz, vin, vout, cin, cout, (const R*)op.coef};
        if (op.dim == 2) {
            if (sync) stencil_kernel<R, 2, KAHAN, true><<<grid, block, 0, st>>>(a, sp);
            else stencil_kernel<R, 2, KAHAN, false><<<grid, block, 0, st>>>(a, sp);
        } else {
            if (sync) stencil_kernel<R, 3, KAHAN, true><<<grid, block, 0, st>>>(a, sp);
            else stencil_kernel<R, 3, KAHAN, false><<<grid, block, 0, st>>>(a, sp);
        }
    } else {
        SellArgs<R> a{(int)s.n, vin, vout, cin, cout, op.chunk_ptr, op.chunk_w, op.col, (const R*)op.val};
        if (sync) sell_kernel<R, KAHAN, true><<<grid, block, 0, st>>>(a, sp);
        else sell_kernel<R, KAHAN, false><<<grid, block, 0, st>>>(a, sp);
    }
}

void launch_diffusion(const DevState& s, const DiffOp& op, int src, bool sync, int par, const SyncArgs& sa,
                      StepRef step, bool count, int block, cudaStream_t st) {
    if (s.prec == P_F64)
        diff_typed<double, false>(s, op, src, sync, par, sa, step, count, block, st);
    else if (s.kahan)
        diff_typed<float, true>(s, op, src, sync, par, sa, step, count, block, st);
    else
        diff_typed<float, false>(s, op, src, sync, par, sa, step, count, block, st);
}

// ------------------------------------------------------------ k bucketing
// Nodes are placed in buckets of equal k, largest k first, so that the
// reaction kernel's warps run a uniform sub-step count.  counts[par] holds
// the histogram made at the last synchronisation; the other parity's
// counts and cursors are cleared for the next synchronisation.
__global__ void __launch_bounds__(256) bucket_scatter_kernel(int n, const uint8_t* __restrict__ kk,
                                                             const int* __restrict__ counts, int* cursor,
                                                             int* __restrict__ perm, int* other_counts,
                                                             int* other_cursor, int kmax,
                                                             unsigned long long* substeps) {
    __shared__ int off[DAETI_MAX_K];
    __shared__ int blk[DAETI_MAX_K];
    __shared__ int base[DAETI_MAX_K];
    if (threadIdx.x < DAETI_MAX_K) blk[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = DAETI_MAX_K - 1; k >= 1; --k) {
            off[k] = acc;
            acc += (k <= kmax) ? counts[k] : 0;
        }
        off[0] = acc;
    }
    if (blockIdx.x == 0 && threadIdx.x < DAETI_MAX_K) {
        other_counts[threadIdx.x] = 0;
        other_cursor[threadIdx.x] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 32 && substeps) {
        unsigned long long tot = 0;
        for (int k = 1; k <= kmax && k < DAETI_MAX_K; ++k) tot += (unsigned long long)k * counts[k];
        atomicAdd(substeps, tot);
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int k = valid ? (int)kk[i] : 0;
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    int rank = 0, wbase = 0;
    if (valid) {
        const unsigned peers = __match_any_sync(active, k);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        rank = __popc(peers & ((1u << lane) - 1u));
        if (lane == leader) wbase = atomicAdd(&blk[k], __popc(peers));
        wbase = __shfl_sync(peers, wbase, leader);
    }
    __syncthreads();
    if (threadIdx.x < DAETI_MAX_K) {
        const int c = blk[threadIdx.x];
        base[threadIdx.x] = c ? atomicAdd(&cursor[threadIdx.x], c) : 0;
    }
    __syncthreads();
    if (valid) perm[off[k] + base[k] + wbase + rank] = i;
}

void launch_bucket_scatter(const DevState& s, int par, int kmax, int block, cudaStream_t st) {
    if (block <= 0) block = 256;
    const int grid = (int)((s.n + block - 1) / block);
    if (grid == 0) return;
    bucket_scatter_kernel<<<grid, block, 0, st>>>((int)s.n, s.kk, s.counts + par * DAETI_MAX_K,
                                                  s.cursor + par * DAETI_MAX_K, s.perm,
                                                  s.counts + (1 - par) * DAETI_MAX_K,
                                                  s.cursor + (1 - par) * DAETI_MAX_K, kmax, s.substeps);
}

__global__ void tick_kernel(long long* ctr, long long inc) { *ctr += inc; }
__global__ void set_counter_kernel(long long* ctr, long long v) { *ctr = v; }

void launch_tick(long long* ctr, long long inc, cudaStream_t st) { tick_kernel<<<1, 1, 0, st>>>(ctr, inc); }
void launch_set_counter(long long* ctr, long long value, cudaStream_t st) {
    set_counter_kernel<<<1, 1, 0, st>>>(ctr, value);
}

}  // namespace daeti
