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

// Conversions between binary64 and binary32 by integer operations on the
// IEEE 754 encodings.  GB300 runs the FP64 pipe, and with it the hardware
// conversions between the two formats, at a small fraction of the integer
// rate, so the conversion of whole fields between FP64 and df64 is done here
// from the formats' definitions; values outside the common range take the
// hardware conversions.  Both give the same bits.

// binary32 -> binary64, exact: a normal float's biased exponent e (bias 127)
// becomes e + 896 (bias 1023) and its 23 fraction bits the top of the 52;
// zeros keep their sign.  Subnormals, infinities and NaNs: hardware.
__device__ __forceinline__ double widen_f32(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned mag = u & 0x7fffffffu;
    if ((mag >> 23) - 1u >= 254u) {  // biased exponent 0 or 255
        if (mag == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
        return (double)f;
    }
    const unsigned long long bits =
        ((unsigned long long)(u & 0x80000000u) << 32) | (((unsigned long long)mag << 29) + (896ull << 52));
    return __longlong_as_double((long long)bits);
}

struct df64 {
    float hi, lo;

    __host__ __device__ df64() : hi(0.f), lo(0.f) {}
    __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
    __device__ df64(int v) : hi((float)v), lo(0.f) {}
    __device__ df64(float v) : hi(v), lo(0.f) {}
    // nearest df64 to an FP64 value: hi = RN32(v), lo = RN32(v - hi), where
    // v - hi is exact in binary64.  For zeros and for biased exponents E in
    // [949, 1149] (2^-74 <= |v| < 2^127) from the encoding: hi is v's 53-bit
    // significand rounded to 24 bits, ties to even, a carry running into the
    // exponent field as the format provides; v - hi is the signed remainder r
    // of that rounding (|r| <= 2^28) times 2^(E-1075), whose nearest float is
    // RN32(r) 2^(E-1075) -- the scaling by a power of two is exact because the
    // product stays a normal float for every nonzero r in this range.
    __device__ df64(double v)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
        const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
        if (E - 949u > 200u) {
            if ((b << 1) == 0ull) {  // +-0: hi keeps the sign, lo = v - hi = +0
                hi = __uint_as_float(sign);
                lo = 0.f;
            } else {
                hi = __double2float_rn(v);
                lo = __double2float_rn(v - (double)hi);
            }
            return;
        }
        const unsigned low = (unsigned)b & 0x1fffffffu;       // the 29 fraction bits rounded off
        const unsigned up = (unsigned)(b >> 29) & 0x7fffffu;  // the 23 kept
        const unsigned rnd = (low > 0x10000000u || (low == 0x10000000u && (up & 1u))) ? 1u : 0u;
        hi = __uint_as_float(sign | ((((E - 896u) << 23) | up) + rnd));
        const int r = (int)low - (int)(rnd << 29);  // |v| - |hi| in units of 2^(E-1075)
        lo = __int2float_rn(sign ? -r : r) * __uint_as_float((E - 948u) << 23);
    }
    __device__ explicit operator double() const { return widen_f32(hi) + widen_f32(lo); }
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
