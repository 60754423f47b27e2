// Per-node explicit diffusion sub-step on the two operator layouts, shared
// by the diffusion kernels and the reaction kernel that fuses the last
// sub-step of step I (so every path gives bit-identical results).
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace daeti {

// Boundary class of a coordinate: 0 low face, 1 interior, 2 high face.
__device__ __forceinline__ int bclass(int x, int n) { return x == 0 ? 0 : (x == n - 1 ? 2 : 1); }

template <typename R>
__device__ __forceinline__ void ld16(const R* p, R* out);
template <>
__device__ __forceinline__ void ld16<float>(const float* p, float* out) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
}
template <>
__device__ __forceinline__ void ld16<double>(const double* p, double* out) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    out[0] = v.x;
    out[1] = v.y;
}

// One explicit sub-step at a node whose neighbour at offset (dx,dy,dz) is
// fetch(dx,dy,dz).  Shared by the plain and the fused kernels so both give
// the same results: the terms are added in the order of the table entries.
// Offsets outside the grid have coefficient 0 in the table; PAD (V buffers
// with a finite ghost margin wider than the stencil reach) reads them anyway
// and adds 0 * (finite), which leaves the sum unchanged, instead of testing
// the boundary class per neighbour.
template <typename R, int DIM, bool KAHAN, bool PAD = false, class Fetch>
__device__ __forceinline__ void stencil_update(const R* __restrict__ crow, int cx, int cy, int z, int nz, R vi,
                                               float ci, const Fetch& fetch, R& vout, float& cout) {
    constexpr int NV = 16 / (int)sizeof(R);           // entries per 16-byte load
    constexpr int J0 = DIM == 3 ? 0 : 9;              // entries used: [J0, J1)
    constexpr int J1 = DIM == 3 ? 27 : 18;
    R acc = (R)0;
#pragma unroll
    for (int q = J0 / NV; q * NV < J1; ++q) {
        R cs[NV];
        ld16<R>(crow + q * NV, cs);
#pragma unroll
        for (int r = 0; r < NV; ++r) {
            const int j = q * NV + r;
            if (j < J0 || j >= J1 || j == 13) continue;
            const int dz = j / 9 - 1, dy = (j / 3) % 3 - 1, dx = j % 3 - 1;
            const bool ok = PAD || ((dx >= 0 || cx > 0) && (dx <= 0 || cx < 2) && (dy >= 0 || cy > 0) &&
                                    (dy <= 0 || cy < 2) &&
                                    (DIM == 2 || ((dz >= 0 || z > 0) && (dz <= 0 || z < nz - 1))));
            if (ok) acc = fma(cs[r], fetch(dx, dy, dz) - vi, acc);
        }
    }
    R v = vi;
    float cc = ci;
    add_comp(v, KAHAN ? &cc : (float*)nullptr, -acc);
    vout = v;
    cout = cc;
}

// SELL-32 row i: V_i - sum_j a_ij (V_j - V_i) with compensation.
template <typename R, bool KAHAN>
__device__ __forceinline__ void sell_update(const int64_t* __restrict__ chunk_ptr, const int* __restrict__ chunk_w,
                                            const int* __restrict__ col, const R* __restrict__ val,
                                            const R* __restrict__ vin, int i, R vi, float ci, R& vout, float& cout) {
    const int chunk = i >> 5;
    const int lane = i & 31;
    const int64_t off = chunk_ptr[chunk] + lane;
    const int w = chunk_w[chunk];
    R acc = (R)0;
    // batches of 8 entries: all column and value loads of a batch are issued
    // before its gathers, so a warp keeps up to 16 streaming loads in flight.
    // Past the row's width an entry is (column i, value 0), like SELL's own
    // padding, and adds an exact 0; the terms are added in entry order.
    for (int j = 0; j < w; j += 8) {
        int cj[8];
        R aj[8], vj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool in = j + u < w;
            cj[u] = in ? __ldg(col + off + 32 * (int64_t)(j + u)) : i;
            aj[u] = in ? __ldg(val + off + 32 * (int64_t)(j + u)) : (R)0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) vj[u] = vin[cj[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fma(aj[u], vj[u] - vi, acc);
    }
    R v = vi;
    float cc = ci;
    add_comp(v, KAHAN ? &cc : (float*)nullptr, -acc);
    vout = v;
    cout = cc;
}

// Operator view passed to kernels.
template <typename R>
struct OpView {
    int kind;             // 0 stencil table, 1 SELL-32
    int nx, ny, nz;
    const R* coef;
    const uint16_t* cls;  // table row of each node (nullable)
    const R* pcoef;       // 3D float table of entry pairs (y-paired kernel; nullable)
    int per_node;         // one coefficient row per node
    const int64_t* chunk_ptr;
    const int* chunk_w;
    const int* col;
    const R* val;
};

// One sub-step at node i from vin (and cin), any layout (PAD: see stencil_update).
// EXT: the operator may hold one row per node (op.per_node); without it the
// per-node test is compiled out and only the per-class table is read.
template <typename R, int DIM, bool KAHAN, bool PAD, bool EXT>
__device__ __forceinline__ void diffuse_node(const OpView<R>& op, const R* __restrict__ vin, const float* cin, int i,
                                             R& vout, float& cout) {
    const R vi = vin[i];
    const float ci = KAHAN ? cin[i] : 0.f;
    if (DIM == 0) {
        sell_update<R, KAHAN>(op.chunk_ptr, op.chunk_w, op.col, op.val, vin, i, vi, ci, vout, cout);
    } else {
        const int nxy = op.nx * op.ny;
        const int nx = op.nx;
        auto fetch = [&](int dx, int dy, int dz) { return vin[i + dx + dy * nx + dz * nxy]; };
        const bool pn = EXT && op.per_node;
        if (PAD && (pn || op.cls)) {
            // no boundary tests: the table row is all the stencil needs
            const R* crow = op.coef + (size_t)(pn ? i : op.cls[i]) * DAETI_ROW;
            stencil_update<R, (DIM == 0 ? 3 : DIM), KAHAN, PAD>(crow, 1, 1, 1, 3, vi, ci, fetch, vout, cout);
        } else {
            const int x = i % op.nx;
            const int yz = i / op.nx;
            const int y = yz % op.ny;
            const int z = yz / op.ny;
            const int cx = bclass(x, op.nx), cy = bclass(y, op.ny);
            const R* crow = op.coef + (pn ? (size_t)i : (size_t)(z * 3 + cy) * 3 + cx) * DAETI_ROW;
            stencil_update<R, (DIM == 0 ? 3 : DIM), KAHAN, PAD>(crow, cx, cy, z, op.nz, vi, ci, fetch, vout, cout);
        }
    }
}

template <typename R>
inline OpView<R> op_view(const DiffOp& op) {
    OpView<R> v;
    v.kind = op.kind;
    v.nx = op.nx;
    v.ny = op.ny;
    v.nz = op.nz;
    v.coef = (const R*)op.coef;
    v.cls = op.cls;
    v.pcoef = (const R*)op.pcoef;
    v.per_node = op.per_node;
    v.chunk_ptr = op.chunk_ptr;
    v.chunk_w = op.chunk_w;
    v.col = op.col;
    v.val = (const R*)op.val;
    return v;
}

}  // namespace daeti
