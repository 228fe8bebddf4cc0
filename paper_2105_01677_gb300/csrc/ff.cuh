// ff.cuh -- double-single ("float-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2 (about 48
// significant bits).  On GB300 an FP64 warp instruction occupies the FP64 pipe for ~64
// cycles per SM sub-partition, so pair terms that need more than FP32 accuracy are
// evaluated here instead, from the classical error-free transformations:
//   TwoSum      (Knuth, TAOCP vol. 2): s = fl(a + b) and the exact error of that sum;
//   FastTwoSum  (Dekker 1971):         the same when |a| >= |b|;
//   TwoProd     (with a fused multiply-add): p = fl(a b) and its exact error fma(a, b, -p).
// The reciprocal square root starts from the FP32 hardware estimate and takes Newton steps
// y <- y + y (1 - x y^2)/2 with the residual 1 - x y^2 formed exactly; two steps give a
// relative error of a few 1e-15.
#pragma once

#include <cuda_runtime.h>

namespace mps {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.h, b.h);
    return ff_fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = ff_two_sum(a.h, b);
    return ff_fast_two_sum(s.h, s.l + a.l);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = ff_two_prod(a.h, b.h);
    p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
    return ff_fast_two_sum(p.h, p.l);
}

// difference of two coordinates given as (hi, lo) pairs: (bh + bl) - (ah + al)
__device__ __forceinline__ ff ff_diff(float ah, float al, float bh, float bl) {
    const ff s = ff_two_sum(bh, -ah);
    return ff_fast_two_sum(s.h, s.l + (bl - al));
}

// square without the final normalisation (the caller sums three of them)
__device__ __forceinline__ ff ff_sqr_raw(ff a) {
    ff p = ff_two_prod(a.h, a.h);
    p.l = fmaf(2.0f * a.h, a.l, p.l);
    return p;
}

// dx^2 + dy^2 + dz^2 of a float-float displacement
__device__ __forceinline__ ff ff_dist2(ff dx, ff dy, ff dz) {
    const ff x = ff_sqr_raw(dx), y = ff_sqr_raw(dy), z = ff_sqr_raw(dz);
    const ff s1 = ff_two_sum(x.h, y.h);
    const ff s2 = ff_two_sum(s1.h, z.h);
    return ff_fast_two_sum(s2.h, ((s1.l + s2.l) + (x.l + y.l)) + z.l);
}

// one Newton step for y ~ 1/sqrt(x), y given as float-float
__device__ __forceinline__ ff ff_rsqrt_step(ff x, ff y) {
    // t = y^2, u = x t (both to ~2^-48), h = 1 - u, y <- y + y h / 2
    const ff t = ff_mul(y, y);
    ff u = ff_two_prod(x.h, t.h);
    u.l = fmaf(x.h, t.l, fmaf(x.l, t.h, u.l));
    const float hres = (1.0f - u.h) - u.l;
    return ff_add_f(y, 0.5f * y.h * hres);
}

__device__ __forceinline__ ff ff_rsqrt(ff x) {
    const ff y0 = {rsqrtf(x.h), 0.0f};
    return ff_rsqrt_step(x, ff_rsqrt_step(x, y0));
}

// one Newton step only: relative error ~1e-13 (the FP32 estimate's error squared)
__device__ __forceinline__ ff ff_rsqrt1(ff x) {
    const ff y0 = {rsqrtf(x.h), 0.0f};
    return ff_rsqrt_step(x, y0);
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// float -> double by moving the bits (exact for normal floats; zero and subnormal floats
// give a signed zero, an error below 1.2e-38), on the integer pipes
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (e == 0u) return __longlong_as_double((long long)sign);
    if (e == 0xffu) return (double)f;   // infinities and NaN keep their meaning
    const unsigned long long bits =
        sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// float-float -> double with a single FP64 operation (the conversions are bit moves)
__device__ __forceinline__ double ff_to_double_fast(ff a) { return f2d_bits(a.h) + f2d_bits(a.l); }

__host__ inline ff ff_from_double(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

}  // namespace mps
