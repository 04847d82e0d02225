// Double-float arithmetic on the FP32 pipes for sm_103a.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits),
// built from the error-free transformations TwoSum (Knuth) and TwoProduct by FMA (Dekker's
// double-length arithmetic).  On this part FP32 issues about 60 times faster than FP64, so the
// few places that need more than FP32 in O(N^2) loops use these instead of FP64.  Products
// that feed an error-free step are rounded on their own (__fmul_rn) and sums use __fadd_rn /
// __fsub_rn, so that FMA contraction cannot break the transformations.
#pragma once

#include <cuda_runtime.h>

namespace frost {
namespace df {

struct dfloat {
    float h, l;
};

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat make(float h, float l)
{
    dfloat r;
    fast_two_sum(h, l, r.h, r.l);
    return r;
}

// the nearest double-float of an FP64 value (48 of its 53 bits)
__device__ __forceinline__ dfloat from_double(double v)
{
    dfloat r;
    r.h = (float)v;
    r.l = (float)(v - (double)r.h);
    return r;
}

__device__ __forceinline__ double to_double(dfloat a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ dfloat add(dfloat a, dfloat b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return make(s, e);
}

__device__ __forceinline__ dfloat neg(dfloat a)
{
    a.h = -a.h;
    a.l = -a.l;
    return a;
}

__device__ __forceinline__ dfloat sub(dfloat a, dfloat b) { return add(a, neg(b)); }

__device__ __forceinline__ dfloat mul(dfloat a, dfloat b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return make(p, e);
}

__device__ __forceinline__ dfloat mul_f(dfloat a, float b)
{
    const float p = __fmul_rn(a.h, b);
    const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
    return make(p, e);
}

// 1 / sqrt(a) for a > 0: the MUFU estimate y0 and the residual res = 1 - a y0^2 in
// double-float, then y0 (1 - res)^(-1/2) = y0 (1 + res/2 + 3 res^2/8 + ...), |res| < 2^-21
__device__ __forceinline__ dfloat rsqrt(dfloat a)
{
    const float y0 = rsqrtf(a.h);
    const float q = __fmul_rn(y0, y0), qe = fmaf(y0, y0, -q);
    const float pp = __fmul_rn(a.h, q), pe = fmaf(a.h, q, -pp);
    const float res = __fsub_rn(__fsub_rn(__fsub_rn(1.f, pp), pe), fmaf(a.h, qe, __fmul_rn(a.l, q)));
    const float c = __fmul_rn(__fmul_rn(y0, res), fmaf(0.375f, res, 0.5f));
    return make(y0, c);
}

// x = h + l + ll exactly (three FP32 parts hold the 53 bits of an FP64 value)
__device__ __forceinline__ void split3(double v, float &h, float &l, float &ll)
{
    h = (float)v;
    const double r = v - (double)h;
    l = (float)r;
    ll = (float)(r - (double)l);
}

// x_j - x_i from three-part splits: the two larger differences are exact (TwoSum), the
// smallest parts' difference is rounded once.  The result is renormalised (TwoSum of the
// high word and the collected tail): with splits of 12 + 12 + 24 bits (the gradient records)
// a pair closer than ~2^-24 |x| has equal or one-unit-apart high and middle parts, so the
// tail can be as large as the high word, and the products of df::mul, which drop lo x lo,
// need |lo| <= ulp(hi) / 2.
__device__ __forceinline__ dfloat sep(float jh, float jl, float jll, float ih, float il, float ill)
{
    float a, e1, b, e2, h, e4;
    two_sum(jh, -ih, a, e1);
    two_sum(jl, -il, b, e2);
    two_sum(a, b, h, e4);
    const float tail = __fadd_rn(e4, __fadd_rn(e1, __fadd_rn(e2, __fsub_rn(jll, ill))));
    dfloat r;
    two_sum(h, tail, r.h, r.l);
    return r;
}

}  // namespace df
}  // namespace frost
