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
// uniform).  The
// last sub-step of each step I is fused into the reaction launch
// (reaction.cu).
#include <algorithm>

#include "diffops.cuh"

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

// ------------------------------------------------- 3D register z-march
// 3D structured grids with ghost-padded V buffers and the per-class table,
// one thread per (x, y) column over a run of z planes and no barriers (but
// the synchronisation's bucketing): a thread keeps the 3 x 3 neighbourhoods
// of planes z - 1, z, z + 1 and z + 2 in registers and loads only the 9
// values of one new plane per node (instead of 26 neighbours), two planes
// ahead; the loop is unrolled by four so the planes change roles instead of
// being copied.  Same
// stencil_update, same term order: results equal the one-thread-per-node
// kernel's.
constexpr int RZX = 32, RZY = 8;

// One plane of a column: the 3 x 3 neighbourhood of V and, for planes the
// thread computes, the node's Kahan term, V at the last synchronisation and
// activation time (loaded with the plane, ahead of their use).
template <typename R>
struct ZPlane {
    R v[9];
    float c;
    R vs, ac;
};

template <typename R, bool KAHAN, bool SYNC>
struct ZColumn {
    const OpView<R>& op;
    const R* base;        // V of this column at plane 0 (a column of the grid; column 0 off the grid)
    long long nxy;
    int nx, cx, cy, i0;   // i0: node index of the column at plane 0
    bool col_in;
    int z0, z1;
    R* __restrict__ vout;
    const float* __restrict__ cin;
    float* __restrict__ cout;
    const SyncParams<R>& sp;

    __device__ __forceinline__ void load(ZPlane<R>& P, int p) const {
        const R* q = base + nxy * p;
        P.v[0] = q[-nx - 1];
        P.v[1] = q[-nx];
        P.v[2] = q[-nx + 1];
        P.v[3] = q[-1];
        P.v[4] = q[0];
        P.v[5] = q[1];
        P.v[6] = q[nx - 1];
        P.v[7] = q[nx];
        P.v[8] = q[nx + 1];
        if (p >= z0 && p < z1) {
            const int i = i0 + (int)(nxy * p);
            if (KAHAN) P.c = __ldg(cin + i);
            if (SYNC) {
                P.vs = sp.vsync[i];
                P.ac = sp.act[i];
            }
        }
    }
    // node at plane z from planes z - 1 (A), z (B) and z + 1 (C, loaded a
    // step earlier); the load of plane z + 2 into D is issued first, so two
    // planes of loads are in flight while the node is computed.  mode: the
    // bucketing mode of this synchronisation (counts[0]); in the uniform-k
    // mode (< 0) a node whose k differs only sets `differs`, voted on once
    // per block at the end, instead of a block barrier per plane
    __device__ __forceinline__ void step(const ZPlane<R>& A, const ZPlane<R>& B, const ZPlane<R>& C, ZPlane<R>& D,
                                         int z, int mode, int& differs) const {
        if (z + 2 <= z1) load(D, z + 2);
        int k = 1;
        const int i = i0 + (int)(nxy * z);
        if (col_in) {
            const R* crow = op.coef + ((size_t)(z * 3 + cy) * 3 + cx) * DAETI_ROW;
            auto fetch = [&](int dx, int dy, int dz) {
                const int j = (dy + 1) * 3 + (dx + 1);
                return dz < 0 ? A.v[j] : (dz == 0 ? B.v[j] : C.v[j]);
            };
            R v;
            float cc;
            stencil_update<R, 3, KAHAN, true>(crow, 1, 1, 1, 3, B.v[4], KAHAN ? B.c : 0.f, fetch, v, cc);
            vout[i] = v;
            if (KAHAN) cout[i] = cc;
            if (SYNC) k = sync_node_loaded<R, false>(sp, i, v, B.vs, B.ac);
        }
        if (SYNC && sp.counts) {
            if (mode < 0) differs |= col_in && k != -mode;
            else block_append(sp.counts, sp.lists, sp.n, i, k, col_in);
        }
    }
};

template <typename R, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(RZX * RZY, sizeof(R) == 4 ? 3 : 2) zreg_substep_kernel(OpView<R> op, int n, int zrun,
                                                                const R* __restrict__ vin, R* __restrict__ vout,
                                                                const float* __restrict__ cin,
                                                                float* __restrict__ cout, SyncParams<R> sp) {
    pdl_wait();
    pdl_trigger();
    const int gx = blockIdx.x * RZX + threadIdx.x % RZX, gy = blockIdx.y * RZY + threadIdx.x / RZX;
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int z0 = blockIdx.z * zrun, z1 = min(nz, z0 + zrun);
    const bool col_in = gx < nx && gy < ny;
    // offsets reach one plane, row and node beyond the column, inside the
    // ghost margins; columns off the grid read column 0 and store nothing
    const int col = col_in ? gx + nx * gy : 0;
    const ZColumn<R, KAHAN, SYNC> zc{op, vin + col, (long long)nx * ny, nx,
                                     gx == 0 ? 0 : (gx == nx - 1 ? 2 : 1), gy == 0 ? 0 : (gy == ny - 1 ? 2 : 1),
                                     col, col_in, z0, z1, vout, cin, cout, sp};
    const int mode = SYNC && sp.counts ? sp.counts[0] : 1;
    int differs = 0;
    ZPlane<R> P0, P1, P2, P3;
    zc.load(P0, z0 - 1);
    zc.load(P1, z0);
    zc.load(P2, z0 + 1);
    int z = z0;
    for (; z + 4 <= z1; z += 4) {
        zc.step(P0, P1, P2, P3, z, mode, differs);
        zc.step(P1, P2, P3, P0, z + 1, mode, differs);
        zc.step(P2, P3, P0, P1, z + 2, mode, differs);
        zc.step(P3, P0, P1, P2, z + 3, mode, differs);
    }
    if (z < z1) zc.step(P0, P1, P2, P3, z, mode, differs);
    if (z + 1 < z1) zc.step(P1, P2, P3, P0, z + 1, mode, differs);
    if (z + 2 < z1) zc.step(P2, P3, P0, P1, z + 2, mode, differs);
    if (SYNC && sp.counts && mode < 0) {
        if (__syncthreads_or(differs) && threadIdx.x == 0) atomicOr(sp.uflag, 1);
    }
}

// Resident blocks per SM of a kernel at `threads` threads, and the SM count
// (queried once per kernel instance; 4 and 152 if a query fails).
template <typename K>
static int resident_blocks(K kern, int threads) {
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        cached = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, 0) == cudaSuccess && nb > 0 ? nb : 4;
    }
    return cached;
}
static int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cached = cudaGetDevice(&dev) == cudaSuccess &&
                         cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0
                     ? v
                     : 152;
    }
    return cached;
}

// diff_block = 0 on structured grids: 2D shared-memory tiles, or the 3D
// register z-march with its z range split into runs (zrun_req planes, or
// chosen so that the blocks cover the GPU's resident slots in few waves).
template <typename R, bool KAHAN>
static void tiled_launch(bool sync, cudaStream_t st, bool pdl, const OpView<R>& op, const DiffOp& dop, int n,
                         const R* vin, R* vout, const float* cin, float* cout, const SyncParams<R>& sp,
                         int zrun_req) {
    if (dop.dim == 2) {
        const dim3 grid((dop.nx + TX - 1) / TX, (dop.ny + TY - 1) / TY);
        if (sync) launch_ex(tiled2d_substep_kernel<R, KAHAN, true>, grid, TX * TY, st, pdl, op, n, vin, vout, cin, cout, sp);
        else launch_ex(tiled2d_substep_kernel<R, KAHAN, false>, grid, TX * TY, st, pdl, op, n, vin, vout, cin, cout, sp);
        return;
    }
    const long cols = (long)((dop.nx + RZX - 1) / RZX) * ((dop.ny + RZY - 1) / RZY);
    const int nb = sync ? resident_blocks(zreg_substep_kernel<R, KAHAN, true>, RZX * RZY)
                        : resident_blocks(zreg_substep_kernel<R, KAHAN, false>, RZX * RZY);
    const long slots = (long)sm_count() * nb;
    int best = 1;
    double best_cost = 1e300;
    for (int ns = 1; ns <= dop.nz; ++ns) {   // waves x (planes per run + prologue)
        const int zr = (dop.nz + ns - 1) / ns;
        const long blocks = cols * ((dop.nz + zr - 1) / zr);
        const double cost = (double)((blocks + slots - 1) / slots) * (zr + 1.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = ns;
        }
    }
    const int zrun = zrun_req > 0 ? std::min(zrun_req, dop.nz) : (dop.nz + best - 1) / best;
    const dim3 grid((dop.nx + RZX - 1) / RZX, (dop.ny + RZY - 1) / RZY, (dop.nz + zrun - 1) / zrun);
    if (sync)
        launch_ex(zreg_substep_kernel<R, KAHAN, true>, grid, RZX * RZY, st, pdl, op, n, zrun, vin, vout, cin, cout, sp);
    else
        launch_ex(zreg_substep_kernel<R, KAHAN, false>, grid, RZX * RZY, st, pdl, op, n, zrun, vin, vout, cin, cout, sp);
}

template <typename R, bool KAHAN>
static void diff_typed(const DevState& s, const DiffOp& dop, int src, bool sync, int par, const SyncArgs& sa,
                       StepRef step, bool lists, int block, cudaStream_t st, bool pdl, int zrun) {
    SyncParams<R> sp = make_sync<R>(s, sa, step, par, lists);
    const bool padded = s.vpad >= stencil_reach(dop);
    if (dop.kind == 0 && block == 0 && !dop.per_node && !(sync && s.rrate) && (dop.dim == 2 || padded)) {
        // structured grid: 2D shared-memory tiles, or the 3D register
        // z-march (which reads the ghost margins of padded V buffers)
        const OpView<R> op = op_view<R>(dop);
        const R* vin = (const R*)s.V[src];
        R* vout = (R*)s.V[1 - src];
        const float* cin = KAHAN ? s.C[src] : nullptr;
        float* cout = KAHAN ? s.C[1 - src] : nullptr;
        tiled_launch<R, KAHAN>(sync, st, pdl, op, dop, (int)s.n, vin, vout, cin, cout, sp, zrun);
        return;
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
                      StepRef step, bool lists, int block, cudaStream_t st, bool pdl, int zrun) {
    if (s.prec == P_F64)
        diff_typed<double, false>(s, op, src, sync, par, sa, step, lists, block, st, pdl, zrun);
    else if (s.kahan)
        diff_typed<float, true>(s, op, src, sync, par, sa, step, lists, block, st, pdl, zrun);
    else
        diff_typed<float, false>(s, op, src, sync, par, sa, step, lists, block, st, pdl, zrun);
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
