// stage.cuh -- shared-memory staging of binned triangles for one tile, and
// the per-(pixel, triangle) plane distances, shared by the coverage kernel
// (raster.cu) and the fragment-list kernels of the differentiable path
// (grad.cu) so that both classify every pair with the same FP32 arithmetic.
//
// Distances are re-centred on the tile's cone axis a (Sec. 1.1.2 equation,
// evaluated as G.n = a.n + (G - a).n): a.n is formed once per (tile,
// triangle) from the FP32-pair normals in a compensated dot product; the
// per-pixel part is a 3-term FMA chain on |G - a| <= the tile radius.
#pragma once

#include "df.cuh"
#include "vsr_internal.cuh"

constexpr int STAGE_CHUNK = 128;  // triangles staged per pass

struct __align__(16) Stage {
    float4 s0[STAGE_CHUNK];  // S-hat.hi xyz, tie flags (bits)
    float4 s1[STAGE_CHUNK];  // sin rho, 2(1 - cos rho), 1/(2 sin rho), A'.N-hat
    float4 s2[STAGE_CHUNK];  // n1.hi xyz, a.n1
    float4 s3[STAGE_CHUNK];  // n2.hi xyz, a.n2
    float4 s4[STAGE_CHUNK];  // n3.hi xyz, a.n3
    float4 s5[STAGE_CHUNK];  // N-hat.hi xyz, a.N-hat
    float4 s6[STAGE_CHUNK];  // S-hat - a (tile axis) xyz, triangle index (bits)
};

constexpr uint32_t STAGE_EMPTY = 0xffffffffu;  // s6.w of a slot that holds no triangle

// Stage triangle t (a valid record index) into slot j for the tile axis a.
__device__ __forceinline__ void stage_triangle(const float4* __restrict__ rec, size_t TT, uint32_t t, float ax,
                                               float ay, float az, Stage& st, int j)
{
    const float4 cp = rec[RF_CAP * TT + t];
    const float4 cp2 = rec[RF_CAP2 * TT + t];
    const float4 n1 = rec[RF_N1 * TT + t], n2 = rec[RF_N2 * TT + t], n3 = rec[RF_N3 * TT + t];
    const float4 pl = rec[RF_PL * TT + t];
    const float4 l1 = rec[RF_N1L * TT + t], l2 = rec[RF_N2L * TT + t], l3 = rec[RF_N3L * TT + t];
    const float4 ll = rec[RF_PLL * TT + t];
    const float c1 = dot_f_df(ax, ay, az, {{n1.x, l1.x}, {n1.y, l1.y}, {n1.z, l1.z}});
    const float c2 = dot_f_df(ax, ay, az, {{n2.x, l2.x}, {n2.y, l2.y}, {n2.z, l2.z}});
    const float c3 = dot_f_df(ax, ay, az, {{n3.x, l3.x}, {n3.y, l3.y}, {n3.z, l3.z}});
    const float cN = dot_f_df(ax, ay, az, {{pl.x, ll.x}, {pl.y, ll.y}, {pl.z, ll.z}});
    st.s0[j] = make_float4(cp.x, cp.y, cp.z, n1.w);
    st.s1[j] = make_float4(cp2.x, cp2.y, cp2.z, pl.w);
    st.s2[j] = make_float4(n1.x, n1.y, n1.z, c1);
    st.s3[j] = make_float4(n2.x, n2.y, n2.z, c2);
    st.s4[j] = make_float4(n3.x, n3.y, n3.z, c3);
    st.s5[j] = make_float4(pl.x, pl.y, pl.z, cN);
    // S-hat - a from the pair S-hat (exact differences, then one rounding)
    const df dsx = df_add(two_sum(cp.x, -ax), df_make(l1.w));
    const df dsy = df_add(two_sum(cp.y, -ay), df_make(l2.w));
    const df dsz = df_add(two_sum(cp.z, -az), df_make(l3.w));
    st.s6[j] = make_float4(__fadd_rn(dsx.hi, dsx.lo), __fadd_rn(dsy.hi, dsy.lo), __fadd_rn(dsz.hi, dsz.lo),
                           __uint_as_float(t));
}

// |G|^2 - 1, error-free (TwoProd / TwoSum): the chord form of the miter
// distance equals (G.S-hat - cos rho)/sin rho for any G only with this term,
// and FP32 map directions are unit to ~1e-7, not exactly.
__device__ __forceinline__ float norm2_minus_one(float x, float y, float z)
{
    const df px2 = two_prod(x, x), py2 = two_prod(y, y), pz2 = two_prod(z, z);
    const df s1 = two_sum(px2.hi, py2.hi);
    const df s2 = two_sum(s1.hi, pz2.hi);
    const float tail = __fadd_rn(__fadd_rn(__fadd_rn(px2.lo, py2.lo), __fadd_rn(pz2.lo, s1.lo)), s2.lo);
    return __fadd_rn(__fadd_rn(s2.hi, -1.0f), tail);
}

// Miter distance in the chord form (4 sin^2(rho/2) - |G - S-hat|^2 +
// |G|^2 - 1) / (2 sin rho) from the tile-relative pixel direction dg = G - a,
// the staged e = S-hat - a, b = s1 and eg = |G|^2 - 1.
__device__ __forceinline__ float miter_distance(float dgx, float dgy, float dgz, const float4& e, const float4& b,
                                                float eg)
{
    const float mx = dgx - e.x, my = dgy - e.y, mz = dgz - e.z;
    const float q = fmaf(mx, mx, fmaf(my, my, mz * mz));
    return ((b.y - q) + eg) * b.z;
}

// Edge (or plane) distance G.n = a.n + (G - a).n from a staged (n.hi, a.n).
__device__ __forceinline__ float plane_distance(float dgx, float dgy, float dgz, const float4& n)
{
    return fmaf(dgx, n.x, fmaf(dgy, n.y, fmaf(dgz, n.z, n.w)));
}

// The same two distances for two pixels at once (x: the first pixel, y: the
// second) in the packed FP32x2 arithmetic of sm_100+: one instruction per
// two FMAs, adds or multiplies.  Each component is the scalar
// function's IEEE result bit for bit -- the same operations in the same
// order, each rounded once -- so packed and scalar kernels classify every
// (pixel, triangle) pair identically.
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 miter_distance2(float2 dgx, float2 dgy, float2 dgz, const float4& e, const float4& b,
                                                  float2 eg)
{
    const float2 mx = __fadd2_rn(dgx, bcast2(-e.x)), my = __fadd2_rn(dgy, bcast2(-e.y)),
                 mz = __fadd2_rn(dgz, bcast2(-e.z));
    const float2 q = __ffma2_rn(mx, mx, __ffma2_rn(my, my, __fmul2_rn(mz, mz)));
    // b.y - q as fma(q, -1, b.y): the exact difference, rounded once
    return __fmul2_rn(__fadd2_rn(__ffma2_rn(q, bcast2(-1.0f), bcast2(b.y)), eg), bcast2(b.z));
}

__device__ __forceinline__ float2 plane_distance2(float2 dgx, float2 dgy, float2 dgz, const float4& n)
{
    return __ffma2_rn(dgx, bcast2(n.x), __ffma2_rn(dgy, bcast2(n.y), __ffma2_rn(dgz, bcast2(n.z), bcast2(n.w))));
}

// Coverage in 2^-22 fixed point.  m in [0, 1]: fma(m, 2^22, 2^23) lies in
// [2^23, 2^24), where the float spacing is 1, so its single rounding leaves
// round-to-nearest(m 2^22) in the low mantissa bits.  Sums of these terms
// saturate at COV_ONE (coverage 1): min(a + b, C) composes over any grouping
// of non-negative terms, so the result does not depend on how the terms were
// split between CTAs.
constexpr uint32_t COV_ONE = 1u << 22;
__device__ __forceinline__ uint32_t cov_fixed(float m)
{
    return __float_as_uint(fmaf(m, 4194304.0f, 8388608.0f)) - 0x4B000000u;
}

// Centre-inside test (bstep on g_1..3, exact zeros by the tie rule);
// g3m = min(g1, g2, g3).
__device__ __forceinline__ bool centre_inside(float g1, float g2, float g3, float g3m, unsigned ties)
{
    bool in = g3m > 0.0f;
    if (g3m == 0.0f)
        in = (g1 > 0.0f || (g1 == 0.0f && (ties & 1u))) && (g2 > 0.0f || (g2 == 0.0f && (ties & 2u))) &&
             (g3 > 0.0f || (g3 == 0.0f && (ties & 4u)));
    return in;
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
    for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
