// Steps I/III (step B) of Section 2: explicit Euler sub-steps of length
// dt_ad = dt/(2l) on M_L dV/dt = -K V, i.e. V <- V - dt_ad M_L^-1 K V.
// Rows of K sum to zero, so (K V)_i = sum_{j != i} k_ij (V_j - V_i); the
// kernels apply that form with the pre-scaled off-diagonal coefficients
// a_ij = dt_ad k_ij / m_i, which keeps the float differences exact for
// neighbouring nodes.  Layouts:
//   * structured grids: a 9-point (2D) / 27-point (3D) stencil whose
//     coefficients depend only on the node's z layer and its x/y boundary
//     class (table [nz][3][3][28], the 27 offsets and a pad) when D varies
//     at most with z, else one such row per node (neighbour offsets stay
//     implicit; the entries are SELL's, in the same order);
//   * unstructured meshes: SELL-32 sparse rows (chunks of 32 rows,
//     column-major).
// The launch that ends a diffusion half at t_n also runs the synchronisation
// epilogue (activation time, k of the next step A, and either the per-k node
// lists or, after a step with one k at every node, the check that k is still
// uniform).  The last sub-step of each step I is fused into the reaction
// launch (reaction_impl.cuh).  Launch shapes, all with the same terms in the
// same order (bit-identical results): one thread per node; 2D shared-memory
// tiles; in 3D (float) runs of 2 or 4 nodes along y per thread.
#include "diffops.cuh"
#include "fastdiv.h"

namespace daeti {

// EXT: per-node operator rows and the reaction-rate k rule are possible
// (their tests are compiled out of the plain instance).
template <typename R, int DIM, bool KAHAN, bool SYNC, bool PAD, bool EXT>
__global__ void __launch_bounds__(256) substep_kernel(OpView<R> op, int n, const R* __restrict__ vin, R* vout,
                                                     const float* cin, float* cout, SyncParams<R> sp) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    int k = 1;
    if (valid) {
        R v;
        float cc;
        diffuse_node<R, DIM, KAHAN, PAD, EXT>(op, vin, cin, i, v, cc);
        vout[i] = v;
        if (KAHAN) cout[i] = cc;
        if (SYNC) k = sync_node<R, EXT>(sp, i, v);
    }
    if (SYNC && sp.counts) bucket_nodes(sp.counts, sp.lists, sp.uflag, sp.n, i, k, valid);
}

// 2D structured grids, shared-memory tiles: a block owns a TX x TY tile with
// a one-node halo in shared memory; the 9 neighbours come from there.
constexpr int TX = 32, TY = 8;

template <typename R, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(TX * TY) tiled2d_substep_kernel(OpView<R> op, int n, const R* __restrict__ vin,
                                                                 R* vout, const float* cin, float* cout,
                                                                 SyncParams<R> sp) {
    pdl_wait();
    pdl_trigger();
    constexpr int PX = TX + 2, PY = TY + 2, PLANE = PX * PY;
    __shared__ R buf[PLANE];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = op.nx, ny = op.ny;
    for (int q = threadIdx.x; q < PLANE; q += TX * TY) {
        const int gx = x0 + q % PX - 1, gy = y0 + q / PX - 1;
        const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        buf[q] = in ? vin[gx + nx * gy] : (R)0;
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    const bool col_in = gx < nx && gy < ny;
    int k = 1, i = 0;
    if (col_in) {
        const int cx = gx == 0 ? 0 : (gx == nx - 1 ? 2 : 1);
        const int cy = gy == 0 ? 0 : (gy == ny - 1 ? 2 : 1);
        const int li = (ty + 1) * PX + (tx + 1);
        i = gx + nx * gy;
        const R* crow = op.coef + ((size_t)cy * 3 + cx) * DAETI_ROW;
        auto fetch = [&](int dx, int dy, int) { return buf[li + dx + dy * PX]; };
        R v;
        float cc;
        stencil_update<R, 2, KAHAN>(crow, cx, cy, 0, 1, buf[li], KAHAN ? cin[i] : 0.f, fetch, v, cc);
        vout[i] = v;
        if (KAHAN) cout[i] = cc;
        if (SYNC) k = sync_node<R, false>(sp, i, v);
    }
    if (SYNC && sp.counts) bucket_nodes(sp.counts, sp.lists, sp.uflag, sp.n, i, k, col_in);
}

template <typename R>
static SyncParams<R> make_sync(const DevState& s, const SyncArgs& sa, StepRef step, int par, bool lists) {
    SyncParams<R> sp;
    sp.vsync = (R*)s.vsync;
    sp.kk = s.kk;
    sp.act = (R*)s.act;
    sp.counts = lists ? s.counts + par * DAETI_MAX_K : nullptr;
    sp.lists = s.lists;
    sp.n = (int)s.n;
    sp.flags = s.flags;
    sp.uflag = s.flags + 2 + par;
    sp.dt = sa.dt;
    sp.rate_scale = (R)(sa.vscale / sa.dt);
    sp.rrate = (const R*)s.rrate;
    sp.rrate_scale = (R)sa.vscale;
    sp.vth = (R)sa.vth;
    sp.kmax = sa.kmax;
    sp.adaptive = sa.adaptive;
    sp.step = step;
    return sp;
}

template <typename R, int DIM, bool KAHAN, bool PAD>
static void sub_launch(bool sync, int grid, int block, cudaStream_t st, bool pdl, const OpView<R>& op, int n,
                       const R* vin, R* vout, const float* cin, float* cout, const SyncParams<R>& sp) {
    const bool ext = op.per_node || (sync && sp.rrate);
    if (sync && ext)
        launch_ex(substep_kernel<R, DIM, KAHAN, true, PAD, true>, grid, block, st, pdl, op, n, vin, vout, cin, cout, sp);
    else if (sync)
        launch_ex(substep_kernel<R, DIM, KAHAN, true, PAD, false>, grid, block, st, pdl, op, n, vin, vout, cin, cout,
                  sp);
    else if (ext)
        launch_ex(substep_kernel<R, DIM, KAHAN, false, PAD, true>, grid, block, st, pdl, op, n, vin, vout, cin, cout,
                  sp);
    else
        launch_ex(substep_kernel<R, DIM, KAHAN, false, PAD, false>, grid, block, st, pdl, op, n, vin, vout, cin,
                  cout, sp);
}

// ------------------------------------ 3D runs of nodes along y, packed FP32
// A thread updates the NY nodes (x, y + m, z), m = 0 .. NY - 1, y a multiple
// of NY.  In each plane they share rows: NY + 2 rows of three values instead
// of 3 NY (36 loads for two nodes, 54 for four, against 27 per node), and
// the nodes go in pairs (m, m + 1) through packed f32x2 subtractions and
// fmas.  Both halves of a packed operation round exactly as the scalar
// operation does (round to nearest, no flush), and the terms are added in
// stencil_update's order, so results equal the one-thread-per-node kernel's.
// Coefficients come from the table of entry pairs (op.pcoef): one 16-byte
// load gives the pairs of two entries.

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

template <int NY, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(256, NY == 2 ? 5 : 3)
    yrun_substep_kernel(OpView<float> op, int nthreads, FastDiv dnx, FastDiv dnyr, const float* __restrict__ vin,
                        float* __restrict__ vout, const float* __restrict__ cin, float* __restrict__ cout,
                        SyncParams<float> sp) {
    constexpr int NP = NY / 2;   // node pairs
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < nthreads;
    const int tt = active ? t : 0;
    const int nx = op.nx, ny = op.ny, nyr = (op.ny + NY - 1) / NY;
    const int r = fdiv(tt, dnx), x = tt - r * nx;
    const int z = fdiv(r, dnyr), y = NY * (r - z * nyr);
    const int nxy = nx * ny;
    const int i0 = x + nx * (y + ny * z);
    bool ok[NY];
    int idx[NY];
#pragma unroll
    for (int m = 0; m < NY; ++m) {
        ok[m] = active && y + m < ny;
        idx[m] = i0 + m * nx;
    }
    // rows y - 1 .. y + NY of planes z - 1, z, z + 1; rows past y + 1 are
    // clamped to row ny (only they can leave the grid): inside the ghost
    // margins
    const float* p = vin + i0;
    int roff[NY + 2];
#pragma unroll
    for (int row = 0; row < NY + 2; ++row) roff[row] = (row < 3 ? row - 1 : min(row - 1, ny - y)) * nx;
    float v[3][NY + 2][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int row = 0; row < NY + 2; ++row) {
            const float* q = p + ((dz - 1) * nxy + roff[row]);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) v[dz][row][dx] = q[dx - 1];
        }
    float ci[NY], vs[NY];
#pragma unroll
    for (int m = 0; m < NY; ++m) {
        ci[m] = KAHAN && ok[m] ? __ldg(cin + idx[m]) : 0.f;
        // V at the last synchronisation, loaded with V (activation times
        // only where V crosses the threshold)
        vs[m] = SYNC && ok[m] ? sp.vsync[idx[m]] : 0.f;
    }
    const int cx = bclass(x, nx);
    const float* prow[NP];
    unsigned long long vi[NP], acc[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        const int ca = ok[2 * h] ? bclass(y + 2 * h, ny) : 1;
        const int cb = ok[2 * h + 1] ? bclass(y + 2 * h + 1, ny) : ca;
        prow[h] = op.pcoef + ((((size_t)z * 3 + ca) * 3 + cb) * 3 + cx) * (2 * DAETI_ROW);
        vi[h] = pack2(v[1][2 * h + 1][1], v[1][2 * h + 2][1]);
        acc[h] = pack2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < DAETI_ROW / 2; ++q) {
        float4 c4[NP];
#pragma unroll
        for (int h = 0; h < NP; ++h) c4[h] = __ldg(reinterpret_cast<const float4*>(prow[h]) + q);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int j = 2 * q + e;
            if (j >= 27 || j == 13) continue;
            const int dz = j / 9, dy = (j / 3) % 3, dx = j % 3;
#pragma unroll
            for (int h = 0; h < NP; ++h) {
                const unsigned long long cj = e ? pack2(c4[h].z, c4[h].w) : pack2(c4[h].x, c4[h].y);
                const unsigned long long vj = pack2(v[dz][2 * h + dy][dx], v[dz][2 * h + dy + 1][dx]);
                acc[h] = fma2(cj, sub2(vj, vi[h]), acc[h]);
            }
        }
    }
    int kk[NY];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        float a[2];
        unpack2(acc[h], a[0], a[1]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int m = 2 * h + e;
            float vn = v[1][m + 1][1], cc = ci[m];
            add_comp(vn, KAHAN ? &cc : (float*)nullptr, -a[e]);
            kk[m] = 1;
            if (ok[m]) {
                vout[idx[m]] = vn;
                if (KAHAN) cout[idx[m]] = cc;
                if (SYNC) kk[m] = sync_core<float, false>(sp, idx[m], vn, vs[m], [&] { return sp.act[idx[m]]; });
            }
        }
    }
    if (SYNC && sp.counts) bucket_nodes_n<NY>(sp.counts, sp.lists, sp.uflag, sp.n, idx, kk, ok);
}

template <int NY, bool KAHAN>
static void yrun_launch(bool sync, cudaStream_t st, bool pdl, const OpView<float>& op, const DiffOp& dop,
                        const float* vin, float* vout, const float* cin, float* cout, const SyncParams<float>& sp) {
    const int nyr = (dop.ny + NY - 1) / NY;
    const long long nt = (long long)dop.nx * nyr * dop.nz;
    const int grid = (int)((nt + 255) / 256);
    if (!grid) return;
    const FastDiv dnx = fast_div((unsigned)dop.nx), dnyr = fast_div((unsigned)nyr);
    if (sync)
        launch_ex(yrun_substep_kernel<NY, KAHAN, true>, grid, 256, st, pdl, op, (int)nt, dnx, dnyr, vin, vout, cin,
                  cout, sp);
    else
        launch_ex(yrun_substep_kernel<NY, KAHAN, false>, grid, 256, st, pdl, op, (int)nt, dnx, dnyr, vin, vout, cin,
                  cout, sp);
}

// diff_block = 0 on 2D structured grids: shared-memory tiles.
template <typename R, bool KAHAN>
static void tiled2d_launch(bool sync, cudaStream_t st, bool pdl, const OpView<R>& op, const DiffOp& dop, int n,
                           const R* vin, R* vout, const float* cin, float* cout, const SyncParams<R>& sp) {
    const dim3 grid((dop.nx + TX - 1) / TX, (dop.ny + TY - 1) / TY);
    if (sync) launch_ex(tiled2d_substep_kernel<R, KAHAN, true>, grid, TX * TY, st, pdl, op, n, vin, vout, cin, cout, sp);
    else launch_ex(tiled2d_substep_kernel<R, KAHAN, false>, grid, TX * TY, st, pdl, op, n, vin, vout, cin, cout, sp);
}

template <typename R, bool KAHAN>
static void diff_typed(const DevState& s, const DiffOp& dop, int src, bool sync, int par, const SyncArgs& sa,
                       StepRef step, bool lists, int block, cudaStream_t st, bool pdl, int rows) {
    SyncParams<R> sp = make_sync<R>(s, sa, step, par, lists);
    const bool padded = s.vpad >= stencil_reach(dop);
    const bool table = dop.kind == 0 && !dop.per_node && !(sync && s.rrate);
    if (block == 0 && table) {
        const OpView<R> op = op_view<R>(dop);
        const R* vin = (const R*)s.V[src];
        R* vout = (R*)s.V[1 - src];
        const float* cin = KAHAN ? s.C[src] : nullptr;
        float* cout = KAHAN ? s.C[1 - src] : nullptr;
        if (dop.dim == 2) {
            tiled2d_launch<R, KAHAN>(sync, st, pdl, op, dop, (int)s.n, vin, vout, cin, cout, sp);
            return;
        }
        if constexpr (sizeof(R) == 4) {
            // 3D in float with ghost-padded V: runs of 2 or 4 nodes along y
            if (padded && dop.pcoef) {
                if (rows == 4) yrun_launch<4, KAHAN>(sync, st, pdl, op, dop, vin, vout, cin, cout, sp);
                else yrun_launch<2, KAHAN>(sync, st, pdl, op, dop, vin, vout, cin, cout, sp);
                return;
            }
        }
    }
    if (block <= 0) block = 256;
    const int grid = (int)((s.n + block - 1) / block);
    if (grid == 0) return;
    const OpView<R> op = op_view<R>(dop);
    const R* vin = (const R*)s.V[src];
    R* vout = (R*)s.V[1 - src];
    const float* cin = KAHAN ? s.C[src] : nullptr;
    float* cout = KAHAN ? s.C[1 - src] : nullptr;
    const int n = (int)s.n;
    const bool pad = s.vpad >= stencil_reach(dop);
    if (dop.kind == 1) sub_launch<R, 0, KAHAN, false>(sync, grid, block, st, pdl, op, n, vin, vout, cin, cout, sp);
    else if (dop.dim == 2 && pad) sub_launch<R, 2, KAHAN, true>(sync, grid, block, st, pdl, op, n, vin, vout, cin, cout, sp);
    else if (dop.dim == 2) sub_launch<R, 2, KAHAN, false>(sync, grid, block, st, pdl, op, n, vin, vout, cin, cout, sp);
    else if (pad) sub_launch<R, 3, KAHAN, true>(sync, grid, block, st, pdl, op, n, vin, vout, cin, cout, sp);
    else sub_launch<R, 3, KAHAN, false>(sync, grid, block, st, pdl, op, n, vin, vout, cin, cout, sp);
}

void launch_diffusion(const DevState& s, const DiffOp& op, int src, bool sync, int par, const SyncArgs& sa,
                      StepRef step, bool lists, int block, cudaStream_t st, bool pdl, int rows) {
    if (s.prec == P_F64)
        diff_typed<double, false>(s, op, src, sync, par, sa, step, lists, block, st, pdl, rows);
    else if (s.kahan)
        diff_typed<float, true>(s, op, src, sync, par, sa, step, lists, block, st, pdl, rows);
    else
        diff_typed<float, false>(s, op, src, sync, par, sa, step, lists, block, st, pdl, rows);
}

// ---------------------------------------------------------- per-k node lists
// Rebuild the lists of the next step A from kk (after init or a checkpoint load).
__global__ void __launch_bounds__(256) rebuild_lists_kernel(int n, const uint8_t* __restrict__ kk, int* counts,
                                                            int* lists) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    block_append(counts, lists, n, i, valid ? (int)kk[i] : 1, valid);
    if (i == 0) counts[0] = 1;   // the lists of this parity are built
}

void launch_rebuild_lists(const DevState& s, int par, cudaStream_t st) {
    const int grid = (int)((s.n + 255) / 256);
    if (grid) rebuild_lists_kernel<<<grid, 256, 0, st>>>((int)s.n, s.kk, s.counts + par * DAETI_MAX_K, s.lists);
}

__global__ void tick_kernel(long long* ctr, long long inc) {
    pdl_wait();
    *ctr += inc;
}
__global__ void set_counter_kernel(long long* ctr, long long v) {
    pdl_wait();
    *ctr = v;
}

void launch_tick(long long* ctr, long long inc, cudaStream_t st) { tick_kernel<<<1, 1, 0, st>>>(ctr, inc); }
void launch_set_counter(long long* ctr, long long value, cudaStream_t st) {
    set_counter_kernel<<<1, 1, 0, st>>>(ctr, value);
}

}  // namespace daeti
