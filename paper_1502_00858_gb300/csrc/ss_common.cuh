// Shared pieces of the sufficient-statistics sweeps (ss.cu, ss_hessvec.cu): the copy-ring
// constants, complex FMA chains on float2/float4 and the work partition (see ss.cu).
#pragma once

#include "calib_internal.cuh"
#include "tma.cuh"

namespace calib {
namespace ss {

// One stage = one whole diagonal; one stage in flight while the other is computed (3 and 4 stages
// measured no faster for the Hessian pass).
template <bool HV> __host__ __device__ constexpr int nst() { return 2; }
constexpr int BAR_BYTES = 64;  // barrier area, keeps what follows 16-byte aligned
constexpr int HV1_KMAX = 5;    // largest K of the one-thread-per-slot Hessian kernel (register budget)


__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// acc += s * q
__device__ __forceinline__ void cmac(float2& acc, float2 s, float2 q) {
    acc.x = fmaf(s.x, q.x, fmaf(-s.y, q.y, acc.x));
    acc.y = fmaf(s.x, q.y, fmaf(s.y, q.x, acc.y));
}
// acc + a[0] conj(b[0]) + a[1] conj(b[1]) for complex pairs packed as (re, im, re, im), one FMA chain
// per component (a conj(b) = (a.x b.x + a.y b.y, a.y b.x - a.x b.y)).
__device__ __forceinline__ float2 cdot2_acc(float2 acc, float4 a, float4 b) {
    float re = fmaf(a.x, b.x, acc.x);
    re = fmaf(a.y, b.y, re);
    re = fmaf(a.z, b.z, re);
    re = fmaf(a.w, b.w, re);
    float im = fmaf(a.y, b.x, acc.y);
    im = fmaf(-a.x, b.y, im);
    im = fmaf(a.w, b.z, im);
    im = fmaf(-a.z, b.w, im);
    return make_float2(re, im);
}
// acc + sg (x0 b0 + x1 b1) (complex products; sg = +1 or -1 folded into the FMAs).
__device__ __forceinline__ float2 cmul2_acc(float2 acc, float sg, float2 x0, float2 b0, float2 x1, float2 b1) {
    float re = fmaf(sg * x0.x, b0.x, acc.x);
    re = fmaf(-sg * x0.y, b0.y, re);
    re = fmaf(sg * x1.x, b1.x, re);
    re = fmaf(-sg * x1.y, b1.y, re);
    float im = fmaf(sg * x0.x, b0.y, acc.y);
    im = fmaf(sg * x0.y, b0.x, im);
    im = fmaf(sg * x1.x, b1.y, im);
    im = fmaf(sg * x1.y, b1.x, im);
    return make_float2(re, im);
}
// acc + sg (conj(x0) b0 + conj(x1) b1); conj(x) b = (x.x b.x + x.y b.y, x.x b.y - x.y b.x).
__device__ __forceinline__ float2 cmul2c_acc(float2 acc, float sg, float2 x0, float2 b0, float2 x1, float2 b1) {
    float re = fmaf(sg * x0.x, b0.x, acc.x);
    re = fmaf(sg * x0.y, b0.y, re);
    re = fmaf(sg * x1.x, b1.x, re);
    re = fmaf(sg * x1.y, b1.y, re);
    float im = fmaf(sg * x0.x, b0.y, acc.y);
    im = fmaf(-sg * x0.y, b0.x, im);
    im = fmaf(sg * x1.x, b1.y, im);
    im = fmaf(-sg * x1.y, b1.x, im);
    return make_float2(re, im);
}
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
// value of the partner lane (lane ^ 1: the other row of the same slot)
__device__ __forceinline__ float2 shfl2x(float2 v) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1));
}

// Register bucket of the statistics sweeps for K directions (the dispatch in ss.cu).
__host__ __device__ constexpr int ss_bucket(int K) {
    return K <= 6 ? K : (K <= 8 ? 8 : (K <= 10 ? 10 : (K <= 12 ? 12 : 16)));
}
// From bucket 10 on, the trial pass reads U (each entry once) from global memory instead of staging
// it with the S statistics: a stage of one diagonal's U and S at K = 10 (47 KB) leaves shared memory
// for one CTA per SM, the S stage alone (27 KB) for two.
__host__ __device__ constexpr bool ss_u_global(bool hessvec, int kb) { return !hessvec && kb >= 10; }

// CTA holding item i of W items split into G equal contiguous ranges (start(c) = floor(c W / G)).
__device__ __forceinline__ long long cta_of_item(long long i, long long W, long long G) { return ((i + 1) * G - 1) / W; }

}  // namespace ss
}  // namespace calib
