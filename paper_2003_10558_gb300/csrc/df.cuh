// df.cuh -- FP32-pair ("double-float", double-word) arithmetic for the
// per-triangle set-up and the per-tile centring terms.
//
// A value is hi + lo with |lo| <= ulp(hi)/2.  The building blocks are the
// classical error-free transformations:
//   TwoSum      (Knuth, TAOCP vol. 2)          s + e = a + b exactly
//   FastTwoSum  (Dekker 1971, needs |a| >= |b|) s + e = a + b exactly
//   TwoProd     (with FMA)                      p + e = a * b exactly
// and the double-word algorithms of M. Joldes, J.-M. Muller, V. Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017 (DWPlusDW "accurate", DWTimesDW,
// DWTimesFP), plus one Newton step for the quotient and the square root.
// Every operation uses the explicitly rounded intrinsics (__fadd_rn,
// __fmul_rn, __fmaf_rn) so the compiler cannot contract or reassociate them.
#pragma once

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.0f}; }

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fadd_rn(s, -a);
    float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fadd_rn(b, -__fadd_rn(s, -a));
    return {s, e};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// DWPlusDW (accurate version)
__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    df t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    df v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// DWTimesFP
__device__ __forceinline__ df df_mul_f(df x, float y)
{
    df c = two_prod(x.hi, y);
    float cl2 = __fmul_rn(x.lo, y);
    df t = fast_two_sum(c.hi, cl2);
    float tl2 = __fadd_rn(t.lo, c.lo);
    return fast_two_sum(t.hi, tl2);
}

// DWTimesDW
__device__ __forceinline__ df df_mul(df x, df y)
{
    df c = two_prod(x.hi, y.hi);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(c.lo, cl2);
    return fast_two_sum(c.hi, cl3);
}

// quotient: q1 = x.hi / y.hi, one correction step with the double-word residual
__device__ __forceinline__ df df_div(df x, df y)
{
    float q1 = __fdiv_rn(x.hi, y.hi);
    df r = df_sub(x, df_mul_f(y, q1));
    float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

// square root of a positive double-word: s = sqrt(hi), e = (x - s^2) / (2 s)
__device__ __forceinline__ df df_sqrt(df x)
{
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    float s = __fsqrt_rn(x.hi);
    df r = df_sub(x, two_prod(s, s));
    float e = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
    return fast_two_sum(s, e);
}

// 1/sqrt(x) of a positive double-word: r0 = rsqrt(hi), one Newton step
// r = r0 + r0 (1 - x r0^2) / 2 with the residual in double-word arithmetic.
__device__ __forceinline__ df df_rsqrt(df x)
{
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    float r0 = rsqrtf(x.hi);
    r0 = __fmul_rn(r0, __fmaf_rn(__fmul_rn(-0.5f, __fmul_rn(x.hi, r0)), r0, 1.5f));  // ~1 ulp
    df xr2 = df_mul_f(df_mul_f(x, r0), r0);
    float e = __fadd_rn(__fadd_rn(1.0f, -xr2.hi), -xr2.lo);
    return fast_two_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), e));
}

// reciprocal of a double-word
__device__ __forceinline__ df df_recip(df y) { return df_div(df_make(1.0f), y); }

struct df3 {
    df x, y, z;
};

__device__ __forceinline__ df df_dot(df3 a, df3 b) { return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z)); }

__device__ __forceinline__ df3 df_cross(df3 a, df3 b)
{
    return {df_sub(df_mul(a.y, b.z), df_mul(a.z, b.y)), df_sub(df_mul(a.z, b.x), df_mul(a.x, b.z)),
            df_sub(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}

__device__ __forceinline__ df3 df3_sub(df3 a, df3 b) { return {df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_add(df3 a, df3 b) { return {df_add(a.x, b.x), df_add(a.y, b.y), df_add(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_scale(df3 a, df s) { return {df_mul(a.x, s), df_mul(a.y, s), df_mul(a.z, s)}; }
__device__ __forceinline__ df3 df3_div(df3 a, df s) { return {df_div(a.x, s), df_div(a.y, s), df_div(a.z, s)}; }
__device__ __forceinline__ df3 df3_neg(df3 a) { return {df_neg(a.x), df_neg(a.y), df_neg(a.z)}; }

// a . (b_hi + b_lo) for an FP32 vector a and a double-word vector b
// (Ogita-Rump-Oishi style compensated dot product), rounded to one float.
__device__ __forceinline__ float dot_f_df(float ax, float ay, float az, df3 b)
{
    df p = two_prod(ax, b.x.hi);
    df q = two_prod(ay, b.y.hi);
    df r = two_prod(az, b.z.hi);
    df s = two_sum(p.hi, q.hi);
    df t = two_sum(s.hi, r.hi);
    float err = __fadd_rn(__fadd_rn(__fadd_rn(p.lo, q.lo), __fadd_rn(r.lo, s.lo)), t.lo);
    float lo = __fmaf_rn(ax, b.x.lo, __fmaf_rn(ay, b.y.lo, __fmul_rn(az, b.z.lo)));
    return __fadd_rn(t.hi, __fadd_rn(err, lo));
}
