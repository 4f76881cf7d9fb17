// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two float32 numbers
// (about 48 significant bits), built from error-free float32 transformations: the exact product
// error by FMA (Dekker 1971) and the exact sum error by TwoSum (Knuth, TAOCP vol. 2, 4.2.2).
// Every operation uses the _rn intrinsics, so that the compiler neither contracts nor reorders it.
// Used where float32 is too coarse and the GPU's float64 rate is the bound (the fusion-centre
// step, the gauge terms of the LM kernels).
#pragma once

#include <cuda_runtime.h>

namespace calib {

struct DF { float hi, lo; };

// s += a * b with a, b float32.
__device__ __forceinline__ void df_add_prod(DF& s, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);  // a*b - p, exact
    const float t = __fadd_rn(s.hi, p);
    const float z = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));  // s.hi + p - t, exact
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float t = __fadd_rn(a.hi, b.hi);
    const float z = __fsub_rn(t, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, z)), __fsub_rn(b.hi, z));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
    const float hi = __fadd_rn(t, lo);
    return DF{hi, __fsub_rn(lo, __fsub_rn(hi, t))};
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
// a * b: the exact product of the leading parts plus the cross terms, renormalised.
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float hi = __fadd_rn(p, e);
    return DF{hi, __fsub_rn(e, __fsub_rn(hi, p))};
}
// a * b + c
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) { return df_add(df_mul(a, b), c); }
// a * b for float32 a and b, exactly.
__device__ __forceinline__ DF df_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_load(const float2* p) {
    const float2 v = *p;
    return DF{v.x, v.y};
}

// The double-float nearest a float64 value (host side: tables prepared once).
inline float2 df_split(double x) {
    const float hi = (float)x;
    return float2{hi, (float)(x - (double)hi)};
}

}  // namespace calib
