// df2.cuh -- the FP32-pair arithmetic of df.cuh on two independent values at
// once, in the packed FP32x2 instructions of sm_100+ (one instruction per
// two adds, multiplies or FMAs).  Component x is one value, component y the
// other.  Every function performs the operations of its df.cuh namesake in
// the same order, each rounded once to nearest per component, so each
// component is bit for bit the scalar result; divisions, square roots and
// reciprocal square roots have no packed form and run per component.
#pragma once

#include "df.cuh"

struct df2 {
    float2 hi, lo;  // (x, y) components of two double-words
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// per component: cx ? a.x : b.x, cy ? a.y : b.y
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b)
{
    return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}

__device__ __forceinline__ df2 df2_make(float2 a) { return {a, f2(0.0f)}; }
__device__ __forceinline__ df2 df2_neg(df2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ df2 df2_sel(bool cx, bool cy, df2 a, df2 b)
{
    return {sel2(cx, cy, a.hi, b.hi), sel2(cx, cy, a.lo, b.lo)};
}

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    const float2 e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return {s, e};
}

__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ df2 two_prod2(float2 a, float2 b)
{
    const float2 p = mul2(a, b);
    return {p, fma2(a, b, neg2(p))};
}

__device__ __forceinline__ df2 df2_add(df2 x, df2 y)
{
    const df2 s = two_sum2(x.hi, y.hi);
    const df2 t = two_sum2(x.lo, y.lo);
    const float2 c = add2(s.lo, t.hi);
    const df2 v = fast_two_sum2(s.hi, c);
    const float2 w = add2(t.lo, v.lo);
    return fast_two_sum2(v.hi, w);
}

__device__ __forceinline__ df2 df2_sub(df2 x, df2 y) { return df2_add(x, df2_neg(y)); }

__device__ __forceinline__ df2 df2_mul_f(df2 x, float2 y)
{
    const df2 c = two_prod2(x.hi, y);
    const float2 cl2 = mul2(x.lo, y);
    const df2 t = fast_two_sum2(c.hi, cl2);
    const float2 tl2 = add2(t.lo, c.lo);
    return fast_two_sum2(t.hi, tl2);
}

__device__ __forceinline__ df2 df2_mul(df2 x, df2 y)
{
    const df2 c = two_prod2(x.hi, y.hi);
    const float2 tl0 = mul2(x.lo, y.lo);
    const float2 tl1 = fma2(x.hi, y.lo, tl0);
    const float2 cl2 = fma2(x.lo, y.hi, tl1);
    const float2 cl3 = add2(c.lo, cl2);
    return fast_two_sum2(c.hi, cl3);
}

__device__ __forceinline__ float2 div2(float2 a, float2 b)
{
    return make_float2(__fdiv_rn(a.x, b.x), __fdiv_rn(a.y, b.y));
}

__device__ __forceinline__ df2 df2_div(df2 x, df2 y)
{
    const float2 q1 = div2(x.hi, y.hi);
    const df2 r = df2_sub(x, df2_mul_f(y, q1));
    const float2 q2 = div2(r.hi, y.hi);
    return fast_two_sum2(q1, q2);
}

// a component whose hi is not positive gives 0, as df_sqrt / df_rsqrt
__device__ __forceinline__ df2 df2_sqrt(df2 x)
{
    const bool px = x.hi.x > 0.0f, py = x.hi.y > 0.0f;
    const float2 s = make_float2(__fsqrt_rn(px ? x.hi.x : 1.0f), __fsqrt_rn(py ? x.hi.y : 1.0f));
    const df2 r = df2_sub(x, two_prod2(s, s));
    const float2 e = div2(r.hi, mul2(f2(2.0f), s));
    return df2_sel(px, py, fast_two_sum2(s, e), df2_make(f2(0.0f)));
}

__device__ __forceinline__ df2 df2_rsqrt(df2 x)
{
    const bool px = x.hi.x > 0.0f, py = x.hi.y > 0.0f;
    float2 r0 = make_float2(rsqrtf(px ? x.hi.x : 1.0f), rsqrtf(py ? x.hi.y : 1.0f));
    r0 = mul2(r0, fma2(mul2(f2(-0.5f), mul2(x.hi, r0)), r0, f2(1.5f)));
    const df2 xr2 = df2_mul_f(df2_mul_f(x, r0), r0);
    const float2 e = sub2(sub2(f2(1.0f), xr2.hi), xr2.lo);
    return df2_sel(px, py, fast_two_sum2(r0, mul2(mul2(f2(0.5f), r0), e)), df2_make(f2(0.0f)));
}

__device__ __forceinline__ df2 df2_recip(df2 y) { return df2_div(df2_make(f2(1.0f)), y); }

struct df3_2 {
    df2 x, y, z;
};

__device__ __forceinline__ df2 df2_dot(df3_2 a, df3_2 b)
{
    return df2_add(df2_add(df2_mul(a.x, b.x), df2_mul(a.y, b.y)), df2_mul(a.z, b.z));
}

__device__ __forceinline__ df3_2 df2_cross(df3_2 a, df3_2 b)
{
    return {df2_sub(df2_mul(a.y, b.z), df2_mul(a.z, b.y)), df2_sub(df2_mul(a.z, b.x), df2_mul(a.x, b.z)),
            df2_sub(df2_mul(a.x, b.y), df2_mul(a.y, b.x))};
}

__device__ __forceinline__ df3_2 df3_2_sub(df3_2 a, df3_2 b)
{
    return {df2_sub(a.x, b.x), df2_sub(a.y, b.y), df2_sub(a.z, b.z)};
}
__device__ __forceinline__ df3_2 df3_2_add(df3_2 a, df3_2 b)
{
    return {df2_add(a.x, b.x), df2_add(a.y, b.y), df2_add(a.z, b.z)};
}
__device__ __forceinline__ df3_2 df3_2_scale(df3_2 a, df2 s) { return {df2_mul(a.x, s), df2_mul(a.y, s), df2_mul(a.z, s)}; }
__device__ __forceinline__ df3_2 df3_2_neg(df3_2 a) { return {df2_neg(a.x), df2_neg(a.y), df2_neg(a.z)}; }
__device__ __forceinline__ df3_2 df3_2_sel(bool cx, bool cy, df3_2 a, df3_2 b)
{
    return {df2_sel(cx, cy, a.x, b.x), df2_sel(cx, cy, a.y, b.y), df2_sel(cx, cy, a.z, b.z)};
}
