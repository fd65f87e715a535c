// Two independent double-word values processed together ("lane x" and "lane y"), every FP32
// operation issued as one packed f32x2 instruction (add/sub/mul/fma.rn.f32x2, PTX ISA 8.6,
// sm_100 and later): two lanes per issue slot.  Each lane performs exactly the FP32
// operations of the scalar double-word routine it mirrors (dw.cuh), in the same order and
// with the same IEEE rounding, so its result is the scalar routine's, bit for bit.
//
// A packed FP32 pair lives in one 64-bit register pair (f2); a dw2 holds the high words of
// both lanes, then their low words, and is 16 bytes: one 128-bit shared-memory access moves a
// whole operand.  Negation flips both sign bits with one 64-bit xor (there is no packed neg).
#pragma once

#include <cstdint>

#include "dw.cuh"

namespace p2s {

struct f2 {
    unsigned long long v;
};

struct __align__(16) dw2 {
    f2 hi, lo;
};

__device__ __forceinline__ f2 f2_make(float x, float y) {
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d.v) : "f"(x), "f"(y));
    return d;
}
__device__ __forceinline__ float f2_x(f2 a) { return __uint_as_float((unsigned)(a.v & 0xffffffffull)); }
__device__ __forceinline__ float f2_y(f2 a) { return __uint_as_float((unsigned)(a.v >> 32)); }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{a.v ^ 0x8000000080000000ull}; }
__device__ __forceinline__ f2 f2_zero() { return f2{0ull}; }

__device__ __forceinline__ dw2 dw2_make(dw x, dw y) { return dw2{f2_make(x.hi, y.hi), f2_make(x.lo, y.lo)}; }
__device__ __forceinline__ dw2 dw2_dup(dw x) { return dw2_make(x, x); }
__device__ __forceinline__ dw2 dw2_zero() { return dw2{f2_zero(), f2_zero()}; }
__device__ __forceinline__ dw dw2_x(dw2 a) { return dw{f2_x(a.hi), f2_x(a.lo)}; }
__device__ __forceinline__ dw dw2_y(dw2 a) { return dw{f2_y(a.hi), f2_y(a.lo)}; }
__device__ __forceinline__ dw2 dw2_neg(dw2 a) { return dw2{f2_neg(a.hi), f2_neg(a.lo)}; }

// TwoSum and Fast2Sum per lane (two_sum, fast_two_sum of dw.cuh)
__device__ __forceinline__ dw2 two_sum2(f2 a, f2 b) {
    const f2 s = f2_add(a, b);
    const f2 bb = f2_sub(s, a);
    return dw2{s, f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}
__device__ __forceinline__ dw2 fast_two_sum2(f2 a, f2 b) {
    const f2 s = f2_add(a, b);
    return dw2{s, f2_sub(b, f2_sub(s, a))};
}

// dw_add_fast per lane
__device__ __forceinline__ dw2 dw2_add_fast(dw2 x, dw2 y) {
    const dw2 s = two_sum2(x.hi, y.hi);
    return fast_two_sum2(s.hi, f2_add(s.lo, f2_add(x.lo, y.lo)));
}

// dw_acc per lane: two accumulators of sums of products
struct dw2_acc {
    f2 s = f2_zero(), c = f2_zero();
    __device__ __forceinline__ void fma(dw2 a, dw2 b) {
        const f2 p = f2_mul(a.hi, b.hi);
        f2 e = f2_fma(a.hi, b.hi, f2_neg(p));
        e = f2_fma(a.hi, b.lo, e);
        e = f2_fma(a.lo, b.hi, e);
        const f2 t = f2_add(s, p);
        const f2 bp = f2_sub(t, s);
        c = f2_add(c, f2_add(f2_add(f2_sub(s, f2_sub(t, bp)), f2_sub(p, bp)), e));
        s = t;
    }
    __device__ __forceinline__ dw2 value() const { return fast_two_sum2(s, c); }
};

}  // namespace p2s
