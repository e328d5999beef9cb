// Double-float ("double-word") arithmetic of the MM_F32X2 precision (its
// fields, FFTs, convolution and local terms): a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits, computed on the
// FP32 pipes (64 times the FP64 FMA rate on this GPU).
//
// Building blocks: TwoSum (Knuth, TAOCP vol. 2), Fast2Sum (Dekker, Numer.
// Math. 18 (1971) 224) and the exact product with one FMA.  Addition is the
// double-word sum that adds the two high parts exactly, the low parts with
// one rounding and renormalises ("SloppyDWPlusDW"); its error is a small
// multiple of u^2 (|a| + |b|), u = 2^-24, which is the norm-wise bound an
// FFT error analysis needs.  Multiplication is the double-word product with
// FMA ("DWTimesDW"), relative error a small multiple of u^2.  Both are
// analysed by Joldes, Muller and Popescu, ACM Trans. Math. Softw. 44 (2017)
// 15.  Intrinsics with explicit rounding keep the compiler from contracting
// the error-free transformations into FMAs.
#pragma once

#include <cuda_runtime.h>

// aligned like float2 / float4, so that loads and stores of a value (or a
// complex value) are single vector accesses in shared and global memory
struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // nearest double-word of a double (hi = rounded value, lo = rounded remainder)
    __host__ __device__ constexpr dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr dfloat(int i) : hi((float)i), lo(0.0f) {}
};

struct __align__(16) dcomplex {
    dfloat x, y;
};

#ifdef __CUDACC__
__device__ __forceinline__ dfloat df_fast2sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df_fast2sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);                 // exact: a.hi b.hi = p + e
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return df_fast2sum(p, e);
}
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { a = a + b; return a; }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { a = a - b; return a; }
__device__ __forceinline__ dfloat &operator*=(dfloat &a, dfloat b) { a = a * b; return a; }

// the double nearest to hi + lo (one rounding: the sum of two floats is exact in double)
__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

// Quotient by long division: q1 = a.hi / b.hi (correctly rounded), the
// remainder a - b q1 formed in double-word arithmetic, and one correction
// q2 = r.hi / b.hi.  The error of q1 + q2 is that of q2 (a relative 2^-24 of a
// term 2^-24 times smaller than q1) plus the double-word rounding of the
// remainder: a few units of 2^-48 relative.
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfloat r = a - b * dfloat(q1, 0.0f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_fast2sum(q1, q2);
}

// 1 / sqrt(a) for a > 0: the correctly rounded float y0 = 1/sqrt(a.hi), then
// one Newton step for f(y) = 1/y^2 - a, y1 = y0 + y0 (1 - a y0^2) / 2, with
// the residual 1 - a y0^2 in double-word arithmetic (y0^2 exact by one FMA).
// y0 has relative error <= 2^-24 (plus 2^-25 from dropping a.lo), the step
// squares it: about 2^-47 relative.
__device__ __forceinline__ dfloat df_rsqrt(dfloat a)
{
    const float y0 = __frsqrt_rn(a.hi);
    const float p = __fmul_rn(y0, y0);
    const dfloat y2(p, fmaf(y0, y0, -p));
    const dfloat e = dfloat(1.0f, 0.0f) - a * y2;
    return df_fast2sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e.hi));
}
#endif
