// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers, |lo| <= ulp(hi) / 2 after normalisation: about 48 significant bits
// within the FP32 exponent range.  Built from two error-free transformations:
// Knuth's two-sum (The Art of Computer Programming, vol. 2, 4.2.2, Theorem B)
// and the exact product a b = p + e with e = fma(a, b, -p) (Dekker 1971 wrote
// the product without an FMA; with one the error term is a single rounding-
// free operation).  The _rn intrinsics are never contracted or reassociated
// by the compiler, which the transformations rely on.
#pragma once

namespace glls {

struct __align__(8) ffloat {   // 8-byte aligned: one 64-bit shared-memory access per value
    float hi, lo;
};

__device__ __forceinline__ ffloat ff_from_double(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ffloat a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth's two-sum: no condition on |a|, |b|)
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// hi + lo rewritten with |lo| <= ulp(hi) / 2 (the fast two-sum, valid when
// |hi| >= |lo| or hi = 0)
__device__ __forceinline__ ffloat ff_norm(ffloat a) {
    const float s = __fadd_rn(a.hi, a.lo);
    return {s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

// acc += a b for float-float a, b.  The exact product of the high parts plus
// the two cross terms (a.lo b.lo is below the format's precision); the sum's
// rounding error and the product's low part are collected in acc.lo, which
// is left unnormalised (a few terms in a row stay well inside its headroom).
__device__ __forceinline__ void ff_mac(ffloat& acc, ffloat a, ffloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, es;
    ff_two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(es, e));
}

// a + b and a - b, normalised
__device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
    float s, e;
    ff_two_sum(a.hi, b.hi, s, e);
    return ff_norm({s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))});
}
__device__ __forceinline__ ffloat ff_sub(ffloat a, ffloat b) { return ff_add(a, {-b.hi, -b.lo}); }

}  // namespace glls
