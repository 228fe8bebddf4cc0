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

// ---------------------------------------------------------------- packed pairs
// The same transformations on two independent values at once with the FP32x2 instructions
// (sm_100 and later): lane x and lane y never mix.  Every operation is an explicit
// round-to-nearest intrinsic, so none of them is contracted into a fused multiply-add.
struct ff2 {
    float2 h, l;
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ ff2 ff2_two_sum(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    const float2 e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff2 ff2_fast_two_sum(float2 a, float2 b) {
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ ff2 ff2_two_prod(float2 a, float2 b) {
    const float2 p = mul2(a, b);
    return {p, fma2(a, b, neg2(p))};
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
    const ff2 s = ff2_two_sum(a.h, b.h);
    return ff2_fast_two_sum(s.h, add2(s.l, add2(a.l, b.l)));
}

__device__ __forceinline__ ff2 ff2_add_f(ff2 a, float2 b) {
    const ff2 s = ff2_two_sum(a.h, b);
    return ff2_fast_two_sum(s.h, add2(s.l, a.l));
}

__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
    ff2 p = ff2_two_prod(a.h, b.h);
    p.l = fma2(a.h, b.l, fma2(a.l, b.h, p.l));
    return ff2_fast_two_sum(p.h, p.l);
}

// (bh + bl) - (ah + al) for two coordinate pairs b against one a
__device__ __forceinline__ ff2 ff2_diff(float ah, float al, float2 bh, float2 bl) {
    const ff2 s = ff2_two_sum(bh, f2(-ah));
    return ff2_fast_two_sum(s.h, add2(s.l, sub2(bl, f2(al))));
}

__device__ __forceinline__ ff2 ff2_sqr_raw(ff2 a) {
    ff2 p = ff2_two_prod(a.h, a.h);
    p.l = fma2(add2(a.h, a.h), a.l, p.l);
    return p;
}

__device__ __forceinline__ ff2 ff2_dist2(ff2 dx, ff2 dy, ff2 dz) {
    const ff2 x = ff2_sqr_raw(dx), y = ff2_sqr_raw(dy), z = ff2_sqr_raw(dz);
    const ff2 s1 = ff2_two_sum(x.h, y.h);
    const ff2 s2 = ff2_two_sum(s1.h, z.h);
    return ff2_fast_two_sum(s2.h, add2(add2(add2(s1.l, s2.l), add2(x.l, y.l)), z.l));
}

__device__ __forceinline__ ff2 ff2_rsqrt_step(ff2 x, ff2 y) {
    const ff2 t = ff2_mul(y, y);
    ff2 u = ff2_two_prod(x.h, t.h);
    u.l = fma2(x.h, t.l, fma2(x.l, t.h, u.l));
    const float2 hres = sub2(sub2(f2(1.0f), u.h), u.l);
    return ff2_add_f(y, mul2(mul2(f2(0.5f), y.h), hres));
}

// one Newton step from the FP32 estimate (relative error ~1e-13).  The start y0 has no low
// part, so y0^2 is a single exact product, and the correction y0 h / 2 (|h| ~ 1e-7) is
// added by FastTwoSum: the values of the general step taken from (y0, 0), in fewer operations
__device__ __forceinline__ ff2 ff2_rsqrt1(ff2 x) {
    const float2 y0 = make_float2(rsqrtf(x.h.x), rsqrtf(x.h.y));
    const ff2 t = ff2_two_prod(y0, y0);
    ff2 u = ff2_two_prod(x.h, t.h);
    u.l = fma2(x.h, t.l, fma2(x.l, t.h, u.l));
    const float2 hres = sub2(sub2(f2(1.0f), u.h), u.l);
    return ff2_fast_two_sum(y0, mul2(mul2(f2(0.5f), y0), hres));
}

// a b + c with the product's low part carried into the sum unnormalised (one FastTwoSum
// fewer than ff2_add(ff2_mul(a, b), c); the same ~2^-46 relative error)
__device__ __forceinline__ ff2 ff2_mul_add(ff2 a, ff2 b, ff2 c) {
    ff2 p = ff2_two_prod(a.h, b.h);
    p.l = fma2(a.h, b.l, fma2(a.l, b.h, p.l));
    const ff2 s = ff2_two_sum(p.h, c.h);
    return ff2_fast_two_sum(s.h, add2(s.l, add2(p.l, c.l)));
}

// 2/x for x > 0: the correctly rounded FP32 reciprocal y0 of x.h and one Newton step
// y = y0 + y0 (1 - x y0) with the residual formed from an exact product (relative error
// ~1e-14), doubled exactly
__device__ __forceinline__ ff2 ff2_two_over(ff2 x) {
    const float2 y0 = make_float2(__frcp_rn(x.h.x), __frcp_rn(x.h.y));
    const ff2 t = ff2_two_prod(x.h, y0);
    const float2 e = sub2(sub2(sub2(f2(1.0f), t.h), t.l), mul2(x.l, y0));
    const ff2 y = ff2_add_f({y0, f2(0.f)}, mul2(y0, e));
    return {add2(y.h, y.h), add2(y.l, y.l)};
}

// 1 - a and a^3 of packed float-float values
__device__ __forceinline__ ff2 ff2_one_minus(ff2 a) {
    return ff2_add_f({neg2(a.h), neg2(a.l)}, f2(1.0f));
}
__device__ __forceinline__ ff2 ff2_cube(ff2 a) { return ff2_mul(ff2_mul(a, a), a); }

__device__ __forceinline__ ff ff2_lo(const ff2& a) { return {a.h.x, a.l.x}; }
__device__ __forceinline__ ff ff2_hi(const ff2& a) { return {a.h.y, a.l.y}; }

__host__ inline ff ff_from_double(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

}  // namespace mps
