// Double-float arithmetic on the float32 pipes: the accurate sums and products of a value held
// as two floats, and the stage-recurrence helper of the float32 and bfloat16-storage policies.
#pragma once

#include <cuda_runtime.h>

namespace pb {

// A value held as the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2), about 48
// significant bits, computed on the float32 pipes (GB300 issues float64 at a small fraction of
// the float32 rate).  Sums follow Knuth's two-sum and Dekker's fast two-sum; products take the
// exact rounding error of hi * hi from a fused multiply-add.  Every operation is an explicit
// round-to-nearest intrinsic, so the compiler neither contracts nor reorders the error terms.
struct dfloat {
    float hi, lo;
    dfloat() = default;
    __device__ constexpr dfloat(float h) : hi(h), lo(0.f) {}
    __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// The sum's error is a small multiple of 2^-48 (|x| + |y|): relative to the operands, not to the
// result (when x and y nearly cancel the result keeps the absolute, not the relative, accuracy).
// That is the accuracy a residual of a stencil needs, whose error budget is set by the magnitude
// of the terms it sums; the low parts are therefore added in one float (no second two-sum).
__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
    const dfloat s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ double to_double(dfloat x) { return (double)x.hi + (double)x.lo; }

// Running sum of products c_i v_i with float64 coefficients c_i = hi_i + lo_i (split on the host)
// and float operands v_i, in double-float: each product's rounding error comes from a fused
// multiply-add, the leading parts are added by two-sum and every error term is gathered in e.
// The value s + e carries about 44 significant bits of the terms' magnitude, so the stage
// recurrence loses nothing to its own arithmetic (or to the float rounding of its coefficients);
// only the store of the result rounds.
struct DfAcc {
    float s, e;
    // starts the sum with c v
    __device__ __forceinline__ void set(float ch, float cl, float v) {
        s = __fmul_rn(ch, v);
        e = __fmaf_rn(cl, v, __fmaf_rn(ch, v, -s));
    }
    __device__ __forceinline__ void add(float ch, float cl, float v) {
        const float p = __fmul_rn(ch, v);
        const float err = __fmaf_rn(cl, v, __fmaf_rn(ch, v, -p));
        const dfloat t = two_sum(s, p);
        s = t.hi;
        e = __fadd_rn(e, __fadd_rn(t.lo, err));
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, e); }
};

// A per-thread sum of products a b read out as a double: in double-float on the float32 pipes
// for float operands (each product exact from a fused multiply-add, the sum about 44 bits: the
// accuracy of a float64 sum of float products, without GB300's thin float64 pipes on every
// point), a plain float64 sum for double operands.
template <typename A> struct DotAcc;
template <> struct DotAcc<float> {
    DfAcc a;
    __device__ __forceinline__ void init() { a.s = 0.f; a.e = 0.f; }
    __device__ __forceinline__ void add(float x, float y) { a.add(x, 0.f, y); }
    __device__ __forceinline__ double value() const { return (double)a.s + (double)a.e; }
};
template <> struct DotAcc<double> {
    double v;
    __device__ __forceinline__ void init() { v = 0.0; }
    __device__ __forceinline__ void add(double x, double y) { v += x * y; }
    __device__ __forceinline__ double value() const { return v; }
};

// c v rounded once, with c = hi + lo
__device__ __forceinline__ float df_scale(float ch, float cl, float v) {
    const float p = __fmul_rn(ch, v);
    float err = __fmaf_rn(ch, v, -p);
    err = __fmaf_rn(cl, v, err);
    return __fadd_rn(p, err);
}

}  // namespace pb
