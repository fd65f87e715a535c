// Arithmetic of the contraction kernels: plain FP64 and float-float (hi + lo FP32 pairs).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace p2s {

struct ArithF64 {
    using T = double;
    using C = double;
    __device__ static T zero() { return 0.0; }
    __device__ static T mul(C c, T x) { return c * x; }  // the first term of a sum
    __device__ static T add(T a, T b) { return a + b; }
    // a * s; the scale is given as FP64 s and as its (hi, lo) FP32 split sh, sl
    __device__ static T scaled(T a, double s, float, float) { return a * s; }
    __device__ static void fma_acc(T& acc, C c, T x) { acc = fma(c, x, acc); }
    __device__ static T finish(T acc) { return acc; }
    __device__ static double to_double(T v) { return v; }
    __device__ static double to_double_fast(T v) { return v; }
    __device__ static T load_moment(const void* p, size_t i) { return __ldg(reinterpret_cast<const double*>(p) + i); }
    __device__ static C load_coef(const void* p, int i) { return __ldg(reinterpret_cast<const double*>(p) + i); }
};

// float-float value: x = hi + lo, |lo| <= ulp(hi)/2 after finish()
struct ArithFF {
    using T = float2;
    using C = float2;
    __device__ static T zero() { return make_float2(0.f, 0.f); }
    // The first term of a sum: c * x as (leading product, its exact FMA error plus the
    // cross terms) -- what fma_acc gives from a zero accumulator, without the TwoSum.
    __device__ static T mul(C c, T x) {
        const float p = c.x * x.x;
        return make_float2(p, fmaf(c.y, x.x, fmaf(c.x, x.y, fmaf(c.x, x.x, -p))));
    }
    // a + b of two finished values: both leading words by TwoSum, the low words and the
    // rounding error joined, renormalised (accurate double-word sum, Joldes, Muller and
    // Popescu 2017)
    __device__ static T add(T a, T b) {
        const float s = a.x + b.x, bp = s - a.x, e = (a.x - (s - bp)) + (b.x - bp);
        const float t = a.y + b.y, tp = t - a.y, f = (a.y - (t - tp)) + (b.y - tp);
        float h = s + (e + t);
        float l = (e + t) - (h - s);
        const float h2 = h + (l + f);
        l = (l + f) - (h2 - h);
        return make_float2(h2, l);
    }
    // a * s with s an FP64 scale given by its (hi, lo) FP32 split sh, sl
    __device__ static T scaled(T a, double, float sh, float sl) {
        const float p = a.x * sh;
        const float e = fmaf(a.y, sh, fmaf(a.x, sl, fmaf(a.x, sh, -p)));
        const float h = p + e;
        return make_float2(h, e - (h - p));
    }
    // acc += c * x, with the exact error of the leading product (FMA) and of the leading
    // sum (TwoSum); second-order terms go to the low word.
    __device__ static void fma_acc(T& acc, C c, T x) {
        float p = c.x * x.x;
        float e = fmaf(c.x, x.x, -p);
        e = fmaf(c.x, x.y, e);
        e = fmaf(c.y, x.x, e);
        float s = acc.x + p;
        float bp = s - acc.x;
        float err = (acc.x - (s - bp)) + (p - bp);
        acc.x = s;
        acc.y += err + e;
    }
    __device__ static T finish(T acc) {  // Fast2Sum renormalisation
        float s = acc.x + acc.y;
        float lo = acc.y - (s - acc.x);
        return make_float2(s, lo);
    }
    // FP64 bits of hi + lo without FP64 instructions: hi's double pattern plus lo in units
    // of the last place of hi's binade (lo < 2^29 such units, so no carry into the exponent;
    // a borrow below a power of two is taken in the halved units of the lower binade).
    __device__ static double to_double(T v) {
        const uint32_t hb = __float_as_uint(v.x);
        const uint32_t ah = hb & 0x7fffffffu;
        // zero and subnormal hi (|hi + lo| < 2^-126) map to a signed zero; inf/nan to a quiet nan
        if (ah < 0x00800000u) return __longlong_as_double((long long)((uint64_t)(hb & 0x80000000u) << 32));
        if (ah >= 0x7f800000u) return __longlong_as_double(0x7ff8000000000000ll);
        const uint32_t e = ah >> 23;
        uint64_t pat = ((uint64_t)((hb & 0x80000000u) | ((e + 896u) << 20) | ((hb & 0x7fffffu) >> 3)) << 32) |
                       (uint64_t)(hb << 29);
        const uint32_t lb = __float_as_uint(v.y);
        const uint32_t al = lb & 0x7fffffffu;
        if (al >= 0x00800000u) {
            const int sh = (int)(al >> 23) - (int)e + 29;
            const uint32_t lm = (al & 0x7fffffu) | 0x800000u;
            uint32_t u = sh >= 0 ? (lm << sh) : (sh > -32 ? (lm >> -sh) : 0u);
            if ((lb ^ hb) & 0x80000000u) {
                if ((hb & 0x7fffffu) == 0u) u <<= 1;
                pat -= u;
            } else {
                pat += u;
            }
        }
        return __longlong_as_double((long long)pat);
    }
    // The same value by a shorter route for the common case 2^-74 <= |hi| < 2^128: lo, scaled
    // by a power of two to units of hi's last double place (exact, |result| <= 2^29), is
    // rounded once and added to the magnitude bits of hi's double pattern.  When hi is a
    // power of two and lo reduces its magnitude, the result lies in the binade below, whose
    // places are half as large, so lo is scaled by twice as much.  Zero, tiny, subnormal,
    // infinite and NaN hi take the general route above.
    __device__ static double to_double_fast(T v) {
        const uint32_t hb = __float_as_uint(v.x);
        const uint32_t e = (hb >> 23) & 0xffu;
        if (e < 53u || e == 0xffu) return to_double(v);
        const uint64_t pat = ((uint64_t)((hb & 0x80000000u) | ((e + 896u) << 20) | ((hb & 0x7fffffu) >> 3)) << 32) |
                             (uint64_t)(hb << 29);
        const bool below = (hb & 0x7fffffu) == 0u && ((__float_as_uint(v.y) ^ hb) & 0x80000000u);
        int u = __float2int_rn(v.y * __uint_as_float((306u + (below ? 1u : 0u) - e) << 23));
        if ((int32_t)hb < 0) u = -u;
        return __longlong_as_double((long long)(pat + (uint64_t)(int64_t)u));
    }
    __device__ static T load_moment(const void* p, size_t i) { return __ldg(reinterpret_cast<const float2*>(p) + i); }
    __device__ static C load_coef(const void* p, int i) { return __ldg(reinterpret_cast<const float2*>(p) + i); }
};

}  // namespace p2s
