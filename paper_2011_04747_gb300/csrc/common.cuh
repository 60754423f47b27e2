// Device-side shared definitions of libdaeti: parameter blocks, precision
// helpers, the synchronisation epilogue run at t_n = n*dt (activation time,
// next k, V(t_n) bookkeeping) and warp-aggregated bucket counting.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#define DAETI_MAX_STIM 32
#define DAETI_MAX_K 16

namespace daeti {

// Step index n of a launch: graph replays read a device counter and add
// their offset inside the graph; plain launches pass the absolute index.
struct StepRef {
    const long long* base;
    long long off;
};

__device__ __forceinline__ long long step_index(const StepRef& s) {
    return (s.base ? *s.base : 0LL) + s.off;
}

// One stimulus (Section 3: 1-2 ms current at a node set; S1-S2 protocols).
struct StimDev {
    double t0, dur, amp, period;
    int reps;
    int pad;
};

// True if the stimulus is on at sub-step start time t (1e-9 ms guard).
__device__ __forceinline__ bool stim_on(const StimDev& s, double t) {
    for (int p = 0; p < s.reps; ++p) {
        double a = s.t0 + p * s.period;
        if (t >= a - 1e-9 && t < a + s.dur - 1e-9) return true;
    }
    return false;
}

// True if the stimulus is on at some instant of [t0, t1).
__device__ __forceinline__ bool stim_overlaps(const StimDev& s, double t0, double t1) {
    for (int p = 0; p < s.reps; ++p) {
        double a = s.t0 + p * s.period - 1e-9;
        double b = s.t0 + p * s.period + s.dur - 1e-9;
        if (a < t1 && b > t0) return true;
    }
    return false;
}

// ------------------------------------------------- dependent launch overlap
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while its predecessor in
// the stream drains, so its blocks are resident when the predecessor ends.
// pdl_wait() blocks until the predecessor grid has completed and its writes
// are visible (a no-op after a normal launch); every kernel that can be
// launched that way calls it before its first global memory access.
// pdl_trigger() allows the successor to be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, bool pdl,
                             Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- precision
template <typename R> struct Fm;
template <> struct Fm<float> {
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float lg(float x) { return __logf(x); }
    // a / b as a times the SFU reciprocal (rcp.approx.ftz of the PTX ISA,
    // relative error ~2^-23; 0 for |b| beyond the normal range)
    static __device__ __forceinline__ float dv(float a, float b) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
        return a * r;
    }
    static __device__ __forceinline__ float rsq(float x) {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float em1(float x) { return expm1f(x); }
    // 2^x and log2(x) by the SFU instructions of the PTX ISA (ex2.approx,
    // lg2.approx; relative error ~2^-22), so that exp(a v + b) = 2^(a' v + b')
    // costs one FFMA with a' = a log2(e), b' = b log2(e) folded at compile time.
    static __device__ __forceinline__ float ex2(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float lg2(float x) {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
};
template <> struct Fm<double> {
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double em1(double x) { return expm1(x); }
    static __device__ __forceinline__ double ex2(double x) { return exp2(x); }
    static __device__ __forceinline__ double lg2(double x) { return log2(x); }
};

#define DAETI_LOG2E 1.4426950408889634
#define DAETI_LN2 0.6931471805599453
// exp(a v + b) for compile-time constants a, b (R and M in scope).
#define EXL(v, a, b) M::ex2(fma((v), (R)((a) * DAETI_LOG2E), (R)((b) * DAETI_LOG2E)))

// v += d with optional Kahan compensation c (true value ~= v - c).
template <typename R>
__device__ __forceinline__ void add_comp(R& v, float* c, R d) {
    if (c) {
        R y = d - (R)(*c);
        R t = v + y;
        *c = (float)((t - v) - y);
        v = t;
    } else {
        v += d;
    }
}

// ------------------------------------------------------------ sync epilogue
// Parameters of the synchronisation at t_{n+1} = (n+1) dt, run on V(t_{n+1})
// right after the first diffusion half that ends there.
template <typename R>
struct SyncParams {
    R* vsync;          // V at the previous synchronisation, updated in place
    uint8_t* kk;       // sub-step count of the next step A
    R* act;            // activation times (-1 = not yet)
    int* counts;       // per-k list lengths of the next step A (nullable: no lists)
    int* lists;        // list of k starts at lists + k * n (k = 1..kmax)
    int n;
    int* flags;        // flags[0] |= 1 on non-finite V
    int* uflag;        // set when a node's k differs from the expected uniform k (mode -K)
    double dt;
    R rate_scale;      // (model units -> mV) / dt: dV/dt of the k rule in mV/ms per unit difference
    const R* rrate = nullptr;   // nullable: dV/dt of each node's last reaction sub-step (model units per ms)
    R rrate_scale = (R)1;       // model units -> mV
    R vth;             // activation threshold
    int kmax;
    int adaptive;      // 0: k = 1 (OST)
    StepRef step;      // step n whose second half ends at this synchronisation
};

// Section 2's k rule from the rate of the split solution over the last step
// (reading R-k; with rrate, the reaction's rate at its last sub-step, reading
// R-k2) and the first-upward-crossing activation time (R-LAT).
// EXT: p.rrate may be set (compiled out otherwise).  vold: V of node i at the
// last synchronisation; act0(): its activation time so far, evaluated only
// when V crosses the threshold upwards (the only case that needs it).
template <typename R, bool EXT, class ActLoad>
__device__ __forceinline__ int sync_core(const SyncParams<R>& p, int i, R vnew, R vold, const ActLoad& act0) {
    int k = 1;
    if (p.adaptive) {
        R rate = (EXT && p.rrate) ? p.rrate[i] * p.rrate_scale : (vnew - vold) * p.rate_scale;
        int k0 = rate > (R)0 ? 5 : 1;
        R a = fabs(rate);
        a = a < (R)1e6 ? a : (R)1e6;          // also maps NaN to 1e6
        k = k0 + (int)floor(a);
        k = k < p.kmax ? k : p.kmax;
    }
    p.kk[i] = (uint8_t)k;
    if (vold < p.vth && vnew >= p.vth && act0() < (R)0) {
        double tprev = (double)step_index(p.step) * p.dt;
        p.act[i] = (R)(tprev + p.dt * (double)((p.vth - vold) / (vnew - vold)));
    }
    p.vsync[i] = vnew;
    if (!isfinite(vnew)) atomicOr(p.flags, 1);
    return k;
}

// The same with V at the last synchronisation (vold) and the activation
// time (a0) of node i already loaded by the caller.
template <typename R, bool EXT>
__device__ __forceinline__ int sync_node_loaded(const SyncParams<R>& p, int i, R vnew, R vold, R a0) {
    return sync_core<R, EXT>(p, i, vnew, vold, [&] { return a0; });
}

template <typename R, bool EXT>
__device__ __forceinline__ int sync_node(const SyncParams<R>& p, int i, R vnew) {
    return sync_core<R, EXT>(p, i, vnew, p.vsync[i], [&] { return p.act[i]; });
}

// Block-cooperative append of node i (valid lanes) to the list of its k
// (list k at lists + k*n): warp ranks by __match_any_sync and one shared
// atomic per (warp, k), then one global atomic per (block, k) on counts[k]
// that returns the block's positions.  Every thread of the block must call it.
__device__ __forceinline__ void block_append(int* counts, int* lists, int n, int i, int k, bool valid) {
    __shared__ int blk[DAETI_MAX_K];
    __shared__ int base[DAETI_MAX_K];
    if (threadIdx.x < DAETI_MAX_K) blk[threadIdx.x] = 0;
    __syncthreads();
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
        base[threadIdx.x] = c ? atomicAdd(&counts[threadIdx.x], c) : 0;
    }
    __syncthreads();
    if (valid) {
        const int pos = base[k] + wbase + rank;
        if (pos < n) lists[(size_t)k * n + pos] = i;
    }
}

// block_append for N nodes per thread (node i[h] with k[h] where v[h]), with
// one set of barriers.
template <int N>
__device__ __forceinline__ void block_append_n(int* counts, int* lists, int n, const int* i, const int* k,
                                               const bool* v) {
    __shared__ int blk[DAETI_MAX_K];
    __shared__ int base[DAETI_MAX_K];
    if (threadIdx.x < DAETI_MAX_K) blk[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int slot[N];
#pragma unroll
    for (int h = 0; h < N; ++h) {
        slot[h] = 0;
        const unsigned active = __ballot_sync(0xffffffffu, v[h]);
        if (v[h]) {
            const unsigned peers = __match_any_sync(active, k[h]);
            const int leader = __ffs(peers) - 1;
            int wbase = 0;
            if (lane == leader) wbase = atomicAdd(&blk[k[h]], __popc(peers));
            wbase = __shfl_sync(peers, wbase, leader);
            slot[h] = wbase + __popc(peers & ((1u << lane) - 1u));
        }
    }
    __syncthreads();
    if (threadIdx.x < DAETI_MAX_K) {
        const int c = blk[threadIdx.x];
        base[threadIdx.x] = c ? atomicAdd(&counts[threadIdx.x], c) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < N; ++h) {
        if (v[h]) {
            const int pos = base[k[h]] + slot[h];
            if (pos < n) lists[(size_t)k[h] * n + pos] = i[h];
        }
    }
}

// Bucketing at a synchronisation.  counts[0] holds the mode the previous
// step A chose: 1 = append every node to the list of its k (block_append);
// -K = that step had k = K at every node, so only check that this one does
// too (one block vote; *uflag is set if some node's k differs).  Every
// thread of the block must call it.
__device__ __forceinline__ void bucket_nodes(int* counts, int* lists, int* uflag, int n, int i, int k, bool valid) {
    const int mode = counts[0];
    if (mode < 0) {
        const int differs = __syncthreads_or(valid && k != -mode);
        if (differs && threadIdx.x == 0) atomicOr(uflag, 1);
        return;
    }
    block_append(counts, lists, n, i, k, valid);
}

// bucket_nodes for N nodes per thread.
template <int N>
__device__ __forceinline__ void bucket_nodes_n(int* counts, int* lists, int* uflag, int n, const int* i, const int* k,
                                               const bool* v) {
    const int mode = counts[0];
    if (mode < 0) {
        bool d = false;
#pragma unroll
        for (int h = 0; h < N; ++h) d = d || (v[h] && k[h] != -mode);
        if (__syncthreads_or(d) && threadIdx.x == 0) atomicOr(uflag, 1);
        return;
    }
    block_append_n<N>(counts, lists, n, i, k, v);
}

}  // namespace daeti
