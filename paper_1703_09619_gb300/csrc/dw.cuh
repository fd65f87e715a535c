// Double-word ("float-float") arithmetic: a value is hi + lo with two FP32 words.
//
// Building blocks (exact transformations of FP32 operations):
//   TwoSum (Knuth), Fast2Sum (Dekker, |a| >= |b|), TwoProd with FMA.
// Composite operations follow Joldes, Muller and Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
//   add   - AccurateDWPlusDW (relative error <= 3u^2 + 13u^3, u = 2^-24),
//   mul   - DWTimesDW with FMA (the 2 FMA variant, error <= 5u^2),
//   div   - a Newton correction of the FP32 quotient,
// which keep about 44 significant bits.  FP64 appears only in the conversions at the
// boundaries (dw_from_double), which kernels do once per element, not per point.
#pragma once

#include <cuda_runtime.h>

namespace p2s {

struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_make(float hi, float lo) { return dw{hi, lo}; }
__device__ __forceinline__ dw dw_from_float(float x) { return dw{x, 0.f}; }
__device__ __forceinline__ dw dw_from_double(double x) {
    const float h = (float)x;
    return dw{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double dw_to_double(dw x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return dw{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = a + b;
    return dw{s, b - (s - a)};
}
__device__ __forceinline__ dw two_prod(float a, float b) {
    const float p = a * b;
    return dw{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dw dw_add(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    const dw t = two_sum(x.lo, y.lo);
    const dw v = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(v.hi, t.lo + v.lo);
}
__device__ __forceinline__ dw dw_neg(dw x) { return dw{-x.hi, -x.lo}; }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_add_f(dw x, float y) {
    const dw s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, s.lo + x.lo);
}
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    const dw p = two_prod(x.hi, y.hi);
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
    const dw p = two_prod(x.hi, y);
    return fast_two_sum(p.hi, fmaf(x.lo, y, p.lo));
}
__device__ __forceinline__ dw dw_fma(dw x, dw y, dw z) { return dw_add(dw_mul(x, y), z); }
__device__ __forceinline__ dw dw_div(dw x, dw y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const dw r = dw_sub(x, dw_mul_f(y, q1));  // remainder x - q1 y
    const float q2 = __fdiv_rn(r.hi, y.hi);
    const dw r2 = dw_sub(r, dw_mul_f(y, q2));
    const float q3 = __fdiv_rn(r2.hi, y.hi);
    const dw q = fast_two_sum(q1, q2);
    return dw_add_f(q, q3);
}

// Cheaper variants whose error is bounded against the operands rather than the result:
// absolute error O(u^2 (|x| + |y|)) for a sum, O(u^2 |x y|) for a product.  The coupling
// factor feeds a normwise error measure (max|dM| / max|M| per element), so cancellation in
// one of its sums may lose relative accuracy of that sum without harming the fill.
//   dw_add_fast - SloppyDWPlusDW (Joldes, Muller and Popescu 2017): the high words add with
//                 TwoSum, the low words join the rounding error, one Fast2Sum renormalises;
//   dw_mul_fast - DWTimesDW with FMA, without the final renormalisation: the pair returned
//                 has |lo| <= ~3u |hi| and every operation here accepts it as an operand;
//   dw_div_fast - an FP32 quotient from the hardware reciprocal (a few ulp) plus one Newton
//                 correction computed from the remainder (x.hi - q y.hi is exact by Sterbenz,
//                 the correction's own error is a few ulp of a term of order u |x / y|):
//                 error about 12 u^2.
__device__ __forceinline__ dw dw_add_fast(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ dw dw_sub_fast(dw x, dw y) { return dw_add_fast(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_mul_fast(dw x, dw y) {
    const float p = x.hi * y.hi;
    return dw{p, fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, fmaf(x.hi, y.hi, -p)))};
}
__device__ __forceinline__ dw dw_fma_fast(dw x, dw y, dw z) { return dw_add_fast(dw_mul_fast(x, y), z); }
__device__ __forceinline__ dw dw_div_fast(dw x, dw y) {
    const float ry = __fdividef(1.f, y.hi);
    const float q1 = x.hi * ry;
    const float ph = y.hi * q1;
    const float pl = fmaf(y.lo, q1, fmaf(y.hi, q1, -ph));
    const float r = (x.hi - ph) + (x.lo - pl);
    return fast_two_sum(q1, r * ry);
}

// Sums without the final renormalisation: (s, e + x.lo + y.lo) with s + e = x.hi + y.hi
// exactly (TwoSum).  The pair still represents the sum to O(u^2 (|x| + |y|)); its low word may
// exceed half an ulp of the high one, which every _fast and _lazy operation here accepts in
// an operand (products take both words of each operand, sums TwoSum the high words).
__device__ __forceinline__ dw dw_add_lazy(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    return dw{s.hi, s.lo + (x.lo + y.lo)};
}
__device__ __forceinline__ dw dw_sub_lazy(dw x, dw y) { return dw_add_lazy(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_fma_lazy(dw x, dw y, dw z) { return dw_add_lazy(dw_mul_fast(x, y), z); }
__device__ __forceinline__ dw dw_add_f_lazy(dw x, float y) {
    const dw s = two_sum(x.hi, y);
    return dw{s.hi, s.lo + x.lo};
}

// Accumulator for sums of products: the leading words sum with TwoSum, every rounding
// error and lower-order product term goes to the second word; renormalise at the end.
struct dw_acc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void fma(dw a, dw b) {
        const float p = a.hi * b.hi;
        float e = fmaf(a.hi, b.hi, -p);
        e = fmaf(a.hi, b.lo, e);
        e = fmaf(a.lo, b.hi, e);
        const float t = s + p;
        const float bp = t - s;
        c += ((s - (t - bp)) + (p - bp)) + e;
        s = t;
    }
    __device__ __forceinline__ void add(dw a) {
        const float t = s + a.hi;
        const float bp = t - s;
        c += ((s - (t - bp)) + (a.hi - bp)) + a.lo;
        s = t;
    }
    __device__ __forceinline__ dw value() const { return fast_two_sum(s, c); }
};

// sin of a double-word argument |x| <= ~6e3 (its words need not be normalised).  Cody-Waite
// reduction by pi/2 with a four-part constant (the first two parts have 12 significant bits,
// so n * part is exact for |n| < 2^12), then Taylor polynomials on |r| <= pi/4 (the leading
// terms in double-word, the tail, below 1e-3 in magnitude, in FP32).  The reduction is
// accurate to the last bit of the double word; its partial sums and the polynomial's sums
// skip their renormalisation except before the square (every later operation takes both
// words), and the result is returned unnormalised (absolute error a few u^2 on a result of
// magnitude <= 1).
__device__ __forceinline__ dw dw_sin(dw x) {
    // pi/2 = C1 + C2 + C3 + C4 (C1, C2 with 12 significant bits; C3, C4 FP32 roundings of the rest)
    const float C1 = 1.57080078125f;
    const float C2 = -4.4535845518112183e-06f;
    const float C3 = -8.7055157527160532e-10f;
    const float C4 = 5.721188916458728e-18f;
    const float n = rintf(x.hi * 0.63661974668502808f);
    // r = x - n (C1 + C2 + C3 + C4), n C1 and n C2 exact
    dw r = dw_add_f_lazy(x, -n * C1);
    r = dw_add_f_lazy(r, -n * C2);
    r = dw_add_lazy(r, dw_neg(two_prod(n, C3)));
    r = dw_add_f(r, -n * C4);
    const dw z = dw_mul_fast(r, r);
    const int q = ((int)n) & 3;
    // One branch-free evaluation for both quadrant parities (lanes of a warp take different
    // quadrants): res = A + B z (c1 + z (c2 + z t(z))) with
    //   sin r: A = B = r, c1 = -1/6, c2 = 1/120, t = -1/5040 + z/362880 - z^2/39916800 + z^3/6227020800;
    //   cos r: A = B = 1, c1 = -1/2, c2 = 1/24,  t = -1/720 + z/40320 - z^2/3628800 + z^3/479001600
    // (the leading terms in double word, the tail, below 1e-3 in magnitude, in FP32).
    const bool c = q & 1;
    const float zf = z.hi;
    float t = fmaf(zf, c ? 2.08767569878680990e-9f : 1.60590438368216146e-10f,
                   c ? -2.75573192239858907e-7f : -2.50521083854417188e-8f);
    t = fmaf(zf, t, c ? 2.48015873015873016e-5f : 2.75573192239858907e-6f);
    t = fmaf(zf, t, c ? -1.38888888888888889e-3f : -1.98412698412698413e-4f);
    const dw c2 = c ? dw_make(0.041666667908430099f, -1.2417634698280722e-09f)    // 1/24
                    : dw_make(0.0083333337679505348f, -4.3461720333759502e-10f);  // 1/120
    const dw c1 = c ? dw_make(-0.5f, 0.f) : dw_make(-0.1666666716337204f, 4.9670538793122887e-09f);  // -1/2, -1/6
    const dw A = c ? dw_make(1.f, 0.f) : r;
    const dw inner = dw_add_lazy(c1, dw_mul_fast(z, dw_add_f_lazy(c2, zf * t)));
    const dw res = dw_add_lazy(A, dw_mul_fast(dw_mul_fast(A, z), inner));
    return (q & 2) ? dw_neg(res) : res;
}

}  // namespace p2s
