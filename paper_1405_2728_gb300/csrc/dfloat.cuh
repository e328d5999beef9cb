// Double-float ("double-word") arithmetic for the FFT and convolution stages
// of the MM_F32X2 precision: a value is the unevaluated sum hi + lo of two
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
#endif
