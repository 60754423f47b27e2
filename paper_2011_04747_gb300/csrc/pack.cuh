// Two floats in one 64-bit register pair, with the packed FP32 instructions
// of sm_100+ (add/sub/mul/fma.rn.f32x2): each lane is rounded exactly as the
// scalar instruction would round it, so a computation on F2 gives in each
// lane what the same sequence of scalar operations gives.  Used by the float
// TP06 reaction to integrate two nodes per thread with half the FP32
// instructions; the SFU operations (2^x, log2, 1/x, 1/sqrt x) stay scalar,
// one per lane.
#pragma once

#include "common.cuh"

namespace daeti {

using ::fma;   // the scalar overloads stay visible beside the packed one below

struct F2 {
    unsigned long long v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float a, float b) {
        asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(a), "f"(b));
    }
    // both lanes equal (constants of the model); explicit, so that no scalar
    // expression turns into a packed one by conversion
    __device__ __forceinline__ explicit F2(double c) : F2((float)c, (float)c) {}
    __device__ __forceinline__ explicit F2(float c) : F2(c, c) {}
    __device__ __forceinline__ explicit F2(int c) : F2((float)c, (float)c) {}
    __device__ __forceinline__ float lo() const {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return a;
    }
    __device__ __forceinline__ float hi() const {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return b;
    }
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.lo(), -a.hi()); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}

// Lane masks of comparisons (bit 0 low lane, bit 1 high lane).
__device__ __forceinline__ int ge_mask(F2 a, float b) { return (a.lo() >= b ? 1 : 0) | (a.hi() >= b ? 2 : 0); }
__device__ __forceinline__ F2 select(int mask, F2 a, F2 b) {
    return F2((mask & 1) ? a.lo() : b.lo(), (mask & 2) ? a.hi() : b.hi());
}

template <> struct Fm<F2> {
    static __device__ __forceinline__ F2 ex2(F2 x) { return F2(Fm<float>::ex2(x.lo()), Fm<float>::ex2(x.hi())); }
    static __device__ __forceinline__ F2 lg2(F2 x) { return F2(Fm<float>::lg2(x.lo()), Fm<float>::lg2(x.hi())); }
    static __device__ __forceinline__ F2 rsq(F2 x) { return F2(Fm<float>::rsq(x.lo()), Fm<float>::rsq(x.hi())); }
    // a / b as a times the SFU reciprocal of b, per lane
    static __device__ __forceinline__ F2 dv(F2 a, F2 b) {
        float r0, r1;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(b.lo()));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(b.hi()));
        return a * F2(r0, r1);
    }
};

}  // namespace daeti
