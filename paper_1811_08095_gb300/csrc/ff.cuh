// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  Every operation is built from FP32 adds and
// FMAs with error-free transformations (Knuth's two-sum, the FMA two-product), so it runs on the
// FP32 pipe; on this part the FP64 pipe delivers a small fraction of the FP32 rate.  Used for the
// reliable updates of the mixed-precision CG, whose true residual b - A x must be accurate to far
// below the solver tolerance (an operation errs by about 2^-46 of its operands).
//
// The intrinsics (__fadd_rn, __fmul_rn) keep the compiler from contracting a product and a sum
// into one FMA, which would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace odwf {

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ ff(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ ff(float v) : hi(v), lo(0.f) {}
    __host__ __device__ ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));  // a.hi + b.hi - s, exact
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);  // a.hi b.hi - p, exact
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
// three quotient digits: q1 + q2 + q3 with the remainders formed in float-float
__device__ __forceinline__ ff operator/(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r1 = a - b * ff(q1);
    const float q2 = __fdiv_rn(r1.hi, b.hi);
    const ff r2 = r1 - b * ff(q2);
    const float q3 = __fdiv_rn(r2.hi, b.hi);
    return ff_fast_two_sum(q1, q2) + ff(q3);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

// conversions of stored float-float pairs to and from a kernel's arithmetic type
template <class R>
__device__ __forceinline__ R ff_to(ff v);
template <>
__device__ __forceinline__ ff ff_to<ff>(ff v) { return v; }
template <>
__device__ __forceinline__ double ff_to<double>(ff v) { return (double)v.hi + (double)v.lo; }
template <>
__device__ __forceinline__ float ff_to<float>(ff v) { return __fadd_rn(v.hi, v.lo); }

__device__ __forceinline__ ff to_ff(ff v) { return v; }
__device__ __forceinline__ ff to_ff(double v) { return ff(v); }
__device__ __forceinline__ ff to_ff(float v) { return ff(v); }

}  // namespace odwf
