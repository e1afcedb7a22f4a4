// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, i.e. a 48-bit significand.  On
// GB300 the FP64 pipe runs at a small fraction of the FP32 rate, so FP64-class
// accuracy for the outer residuals of the mixed-precision solver is cheaper
// from FP32 instructions.  The error-free transformations used are:
//   TwoSum(a, b)    s = fl(a + b), e = a + b - s exactly        (Knuth)
//   FastTwoSum(a,b) the same for |a| >= |b| in three operations (Dekker)
//   TwoProd(a, b)   p = fl(a b), e = fma(a, b, -p) = a b - p exactly
// Addition is Dekker's form: TwoSum of the high parts, the low parts added in
// FP32, one renormalisation -- an error below ~2^-46 (|a| + |b|), i.e. small
// against the operands rather than against the (possibly cancelled) result.
// That is the bound the library needs: a residual b - A x is wanted to an
// absolute accuracy far below tol * |b|, never to full relative accuracy of a
// tiny difference.  The compiler must not reassociate these operations (nvcc
// does not by default; fast-math flags must stay off for this file's users).
#pragma once

#include <cuda_runtime.h>

namespace wl {

// Exact-match overloads: code in namespace wl that calls fma on float or
// double must keep the hardware FMA, not convert to df64 below.
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

struct df64 {
    float hi, lo;

    __host__ __device__ df64() : hi(0.f), lo(0.f) {}
    __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
    __device__ df64(int v) : hi((float)v), lo(0.f) {}
    __device__ df64(float v) : hi(v), lo(0.f) {}
    // nearest df64 to an FP64 value: hi = fl32(v), lo = fl32(v - hi)
    __device__ df64(double v)
    {
        hi = __double2float_rn(v);
        lo = __double2float_rn(v - (double)hi);
    }
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df64 r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df64 r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }

}  // namespace wl
