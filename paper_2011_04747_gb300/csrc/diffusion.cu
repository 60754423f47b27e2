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

// Structured grids: a block owns a TX x TY tile in x-y and marches through a
// run of z planes, keeping three planes of V (tile plus a one-node halo) in
// shared memory; the 27 (9) neighbours then come from shared memory and every
// V value is read from global memory about once per plane it feeds.
constexpr int TX = 32, TY = 8;

template <typename R, int DIM, bool KAHAN, bool SYNC>
__global__ void __launch_bounds__(TX * TY) tiled_substep_kernel(OpView<R> op, int n, int zrun,
                                                               const R* __restrict__ vin, R* vout,
                                                               const float* cin, float* cout, SyncParams<R> sp) {
    pdl_wait();
    pdl_trigger();
    constexpr int PX = TX + 2, PY = TY + 2, PLANE = PX * PY;
    constexpr int NP = DIM == 3 ? 3 : 1;
    __shared__ R buf[NP][PLANE];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int z_begin = DIM == 3 ? blockIdx.z * zrun : 0;
    const int z_end = DIM == 3 ? min(nz, z_begin + zrun) : 1;
    const int nxy = nx * ny;

    auto load_plane = [&](int z) {
        R* dst = buf[DIM == 3 ? (z % 3) : 0];
        for (int q = threadIdx.x; q < PLANE; q += TX * TY) {
            const int lx = q % PX, ly = q / PX;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny && z >= 0 && z < nz;
            dst[q] = in ? vin[gx + nx * gy + nxy * z] : (R)0;
        }
    };
    if (DIM == 3) {
        if (z_begin - 1 >= 0) load_plane(z_begin - 1);
        load_plane(z_begin);
    }
    const int gx = x0 + tx, gy = y0 + ty;
    const bool col_in = gx < nx && gy < ny;
    const int cx = gx == 0 ? 0 : (gx == nx - 1 ? 2 : 1);
    const int cy = gy == 0 ? 0 : (gy == ny - 1 ? 2 : 1);
    const int li = (ty + 1) * PX + (tx + 1);
    for (int z = z_begin; z < z_end; ++z) {
        if (DIM == 3) {
            if (z + 1 < nz) load_plane(z + 1);
        } else {
            load_plane(0);
        }
        __syncthreads();
        int k = 1;
        int i = 0;
        if (col_in) {
            i = gx + nx * gy + nxy * z;
            const R* crow = op.coef + ((size_t)(z * 3 + cy) * 3 + cx) * DAETI_ROW;
            auto fetch = [&](int dx, int dy, int dz) {
                return buf[DIM == 3 ? ((z + dz + 3) % 3) : 0][li + dx + dy * PX];
            };
            R v;
            float cc;
            stencil_update<R, DIM, KAHAN>(crow, cx, cy, z, nz, buf[DIM == 3 ? (z % 3) : 0][li],
                                          KAHAN ? cin[i] : 0.f, fetch, v, cc);
            vout[i] = v;
            if (KAHAN) cout[i] = cc;
            if (SYNC) k = sync_node<R, false>(sp, i, v);
        }
        if (SYNC && sp.counts) bucket_nodes(sp.counts, sp.lists, sp.uflag, sp.n, i, k, col_in);
        __syncthreads();   // the plane z - 1 buffer is refilled next
    }
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

template <typename R, int DIM, bool KAHAN>
static void tiled_launch(bool sync, cudaStream_t st, bool pdl, const OpView<R>& op, const DiffOp& dop, int n,
                         const R* vin, R* vout, const float* cin, float* cout, const SyncParams<R>& sp) {
    const int gx = (dop.nx + TX - 1) / TX, gy = (dop.ny + TY - 1) / TY;
    int zrun = 1, gz = 1;
    if (DIM == 3) {
        // enough blocks to fill the GPU (about 8 per SM), long z runs otherwise
        const long tiles = (long)gx * gy;
        zrun = (int)std::max<long>(1, std::min<long>(dop.nz, (tiles * dop.nz + 1215) / 1216));
        gz = (dop.nz + zrun - 1) / zrun;
    }
    const dim3 grid(gx, gy, gz);
    if (sync)
        launch_ex(tiled_substep_kernel<R, DIM, KAHAN, true>, grid, TX * TY, st, pdl, op, n, zrun, vin, vout, cin, cout,
                  sp);
    else
        launch_ex(tiled_substep_kernel<R, DIM, KAHAN, false>, grid, TX * TY, st, pdl, op, n, zrun, vin, vout, cin,
                  cout, sp);
}

template <typename R, bool KAHAN>
static void diff_typed(const DevState& s, const DiffOp& dop, int src, bool sync, int par, const SyncArgs& sa,
                       StepRef step, bool lists, int block, cudaStream_t st, bool pdl) {
    SyncParams<R> sp = make_sync<R>(s, sa, step, par, lists);
    if (dop.kind == 0 && block == 0 && !dop.per_node && !(sync && s.rrate)) {
        // structured grid, shared-memory tiles
        const OpView<R> op = op_view<R>(dop);
        const R* vin = (const R*)s.V[src];
        R* vout = (R*)s.V[1 - src];
        const float* cin = KAHAN ? s.C[src] : nullptr;
        float* cout = KAHAN ? s.C[1 - src] : nullptr;
        if (dop.dim == 2) tiled_launch<R, 2, KAHAN>(sync, st, pdl, op, dop, (int)s.n, vin, vout, cin, cout, sp);
        else tiled_launch<R, 3, KAHAN>(sync, st, pdl, op, dop, (int)s.n, vin, vout, cin, cout, sp);
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
                      StepRef step, bool lists, int block, cudaStream_t st, bool pdl) {
    if (s.prec == P_F64)
        diff_typed<double, false>(s, op, src, sync, par, sa, step, lists, block, st, pdl);
    else if (s.kahan)
        diff_typed<float, true>(s, op, src, sync, par, sa, step, lists, block, st, pdl);
    else
        diff_typed<float, false>(s, op, src, sync, par, sa, step, lists, block, st, pdl);
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
