// setup.cu -- per-triangle set-up in FP32-pair arithmetic.
//
// For each world-space triangle ABC and camera (O, M):
//   A' = M (A - O)                                 camera space (exact pairs)
//   edge-plane normals  n_AB = s ||A' x B'||, n_BC, n_CA          (Sec. 1.1)
//     with s = sign(A'.(B' x C')) so the triangle is on the positive side of
//     all three (two-sided triangles), and each edge's cross product taken
//     with its vertices in a canonical order (the lexicographic order of the
//     FP32 bit patterns of the world coordinates) and negated when the
//     triangle lists them the other way -- neighbours sharing an edge get
//     bit-for-bit opposite normals, which makes the centre test watertight.
//   miter cap: smallest circle over the projected vertices   (Sec. 1.1.2)
//     a^2 = |B-C|^2, b^2 = |C-A|^2, c^2 = |A-B|^2 of the unit vertices,
//     O_s = a^2(b^2+c^2-a^2), O_t = b^2(c^2+a^2-b^2), O_p = c^2(a^2+b^2-c^2),
//     S = midpoint of the side opposite the first non-positive O, else the
//     circumcentre (O_s A + O_t B + O_p C)/(O_s + O_t + O_p);
//     kept as S-hat, cos rho = |S|, sin rho, 2(1 - cos rho), 1/(2 sin rho).
//   plane: N = (A'-B') x (C'-B') (Sec. 1.1.4), kept as N-hat and A'.N-hat.
// Culled: a vertex at the eye, A'.(B' x C') = 0, or sin rho = 0.
//
// Everything is FP32 arithmetic; the pairs (Dekker / Knuth error-free
// transformations, see df.cuh) keep the normals accurate to ~2^-44 so that the
// anti-aliasing ramp, whose slope is the global delta (hundreds per radian),
// is placed to ~1e-6 of a pixel.
#include "df.cuh"
#include "df2.cuh"
#include "vsr_internal.cuh"

namespace {

struct Cam {
    float O[3];
    float M[9];
};

__device__ __forceinline__ bool vless(const float* P, const float* Q)
{
    for (int c = 0; c < 3; ++c) {
        unsigned a = __float_as_uint(P[c]), b = __float_as_uint(Q[c]);
        if (a != b) return a < b;
    }
    return false;
}

// resident CTAs per SM the pair kernel is compiled for (its register cap)
#ifndef VSR_SETUP_PAIR_CTAS
#define VSR_SETUP_PAIR_CTAS 1
#endif

// The set-up of two triangles per thread, every double-word step in packed
// FP32x2 arithmetic (component x: triangle t0, y: t1 = t0 + 1; df2.cuh), so
// each record is bit for bit what the scalar double-word algorithms of
// df.cuh give for its triangle.  What would branch per triangle is a
// per-component select: the canonical operand order of each edge, the miter
// case (every case is formed), the invalid triangles.
__device__ __forceinline__ df3_2 normalize3_2(df3_2 v) { return df3_2_scale(v, df2_rsqrt(df2_dot(v, v))); }

__device__ __forceinline__ df3_2 edge_normal2(const float* P0, const float* Q0, const float* P1, const float* Q1,
                                              const df3_2& P, const df3_2& Q, bool flip0, bool flip1)
{
    const bool s0 = vless(Q0, P0), s1 = vless(Q1, P1);  // per triangle: cross the canonical order, then negate
    const df3_2 a = df3_2_sel(s0, s1, Q, P), b = df3_2_sel(s0, s1, P, Q);
    df3_2 x = df2_cross(a, b);
    x = df3_2_sel(s0, s1, df3_2_neg(x), x);
    const df3_2 n = normalize3_2(x);
    return df3_2_sel(flip0, flip1, df3_2_neg(n), n);
}

__device__ __forceinline__ unsigned first_positive_c(float x, float y, float z)
{
    if (x != 0.0f) return x > 0.0f;
    if (y != 0.0f) return y > 0.0f;
    return z > 0.0f;
}

// VIEWS: blockIdx.y is a view; its camera is read from cams_dev (12 floats)
// and its records go to rec + view * REC_F * T.
template <bool VIEWS>
__global__ void __launch_bounds__(128, VSR_SETUP_PAIR_CTAS) setup_pair_kernel(const float* __restrict__ tris, int T,
                                                                             Cam cam, const float* __restrict__ cams_dev,
                                                                             float4* __restrict__ rec)
{
    const int t0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (t0 >= T) return;
    if (VIEWS) {
        const float* cv = cams_dev + 12 * blockIdx.y;
#pragma unroll
        for (int q = 0; q < 3; ++q) cam.O[q] = cv[q];
#pragma unroll
        for (int q = 0; q < 9; ++q) cam.M[q] = cv[3 + q];
        rec += (size_t)blockIdx.y * REC_F * (size_t)T;
    }
    const bool has1 = t0 + 1 < T;
    const int t1 = has1 ? t0 + 1 : t0;
    float w0[9], w1[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        w0[q] = tris[(size_t)t0 * 9 + q];
        w1[q] = tris[(size_t)t1 * 9 + q];
    }
    // an identity rotation (the common camera) needs only the exact
    // differences A - O: the pair products by 1 and sums with 0 of the
    // general transform return those pairs unchanged
    bool ident = true;
#pragma unroll
    for (int q = 0; q < 9; ++q) ident = ident && cam.M[q] == ((q % 4 == 0) ? 1.0f : 0.0f);
    df3_2 V[3];
    bool eye0 = false, eye1 = false;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const df2 d0 = two_sum2(make_float2(w0[3 * q + 0], w1[3 * q + 0]), f2(-cam.O[0]));
        const df2 d1 = two_sum2(make_float2(w0[3 * q + 1], w1[3 * q + 1]), f2(-cam.O[1]));
        const df2 d2 = two_sum2(make_float2(w0[3 * q + 2], w1[3 * q + 2]), f2(-cam.O[2]));
        df2 c[3] = {d0, d1, d2};
        if (!ident) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
                c[r] = df2_add(df2_add(df2_mul_f(d0, f2(cam.M[3 * r + 0])), df2_mul_f(d1, f2(cam.M[3 * r + 1]))),
                               df2_mul_f(d2, f2(cam.M[3 * r + 2])));
        }
        V[q] = {c[0], c[1], c[2]};
        eye0 |= (c[0].hi.x == 0.0f && c[1].hi.x == 0.0f && c[2].hi.x == 0.0f);
        eye1 |= (c[0].hi.y == 0.0f && c[1].hi.y == 0.0f && c[2].hi.y == 0.0f);
    }
    const df2 det = df2_dot(V[0], df2_cross(V[1], V[2]));
    bool bad0 = eye0 || det.hi.x == 0.0f || !isfinite(det.hi.x);
    bool bad1 = eye1 || det.hi.y == 0.0f || !isfinite(det.hi.y);
    const bool flip0 = det.hi.x < 0.0f, flip1 = det.hi.y < 0.0f;
    const df3_2 n1 = edge_normal2(w0 + 0, w0 + 3, w1 + 0, w1 + 3, V[0], V[1], flip0, flip1);
    const df3_2 n2 = edge_normal2(w0 + 3, w0 + 6, w1 + 3, w1 + 6, V[1], V[2], flip0, flip1);
    const df3_2 n3 = edge_normal2(w0 + 6, w0 + 0, w1 + 6, w1 + 0, V[2], V[0], flip0, flip1);

    // miter: smallest circle over the unit vertices; every case formed, the
    // triangle's own selected
    const df3_2 U0 = normalize3_2(V[0]), U1 = normalize3_2(V[1]), U2 = normalize3_2(V[2]);
    const df3_2 ea = df3_2_sub(U1, U2), eb = df3_2_sub(U2, U0), ec = df3_2_sub(U0, U1);
    const df2 a2 = df2_dot(ea, ea), b2 = df2_dot(eb, eb), c2 = df2_dot(ec, ec);
    const df2 Os = df2_mul(a2, df2_sub(df2_add(b2, c2), a2));
    const df2 Ot = df2_mul(b2, df2_sub(df2_add(c2, a2), b2));
    const df2 Op = df2_mul(c2, df2_sub(df2_add(a2, b2), c2));
    const df2 half = df2_make(f2(0.5f));
    const df3_2 num = df3_2_add(df3_2_add(df3_2_scale(U0, Os), df3_2_scale(U1, Ot)), df3_2_scale(U2, Op));
    df3_2 S = df3_2_scale(num, df2_recip(df2_add(df2_add(Os, Ot), Op)));
    const bool p0 = Op.hi.x <= 0.0f, p1 = Op.hi.y <= 0.0f;
    S = df3_2_sel(p0, p1, df3_2_scale(df3_2_add(U0, U1), half), S);
    const bool q0 = Ot.hi.x <= 0.0f, q1 = Ot.hi.y <= 0.0f;
    S = df3_2_sel(q0, q1, df3_2_scale(df3_2_add(U2, U0), half), S);
    const bool r0 = Os.hi.x <= 0.0f, r1 = Os.hi.y <= 0.0f;
    S = df3_2_sel(r0, r1, df3_2_scale(df3_2_add(U1, U2), half), S);
    const df2 s2len = df2_dot(S, S);
    const df2 rs = df2_rsqrt(s2len);
    const df2 slen = df2_mul(s2len, rs);
    const df2 one = df2_make(f2(1.0f));
    const df2 omc = df2_sub(one, slen);
    const df2 sr = df2_sqrt(df2_mul(omc, df2_add(one, slen)));
    bad0 = bad0 || !(slen.hi.x > 0.0f) || !(sr.hi.x > 0.0f);
    bad1 = bad1 || !(slen.hi.y > 0.0f) || !(sr.hi.y > 0.0f);
    const df3_2 Sh = df3_2_scale(S, rs);
    const float2 K = mul2(f2(2.0f), omc.hi);
    const float2 inv2sr = div2(f2(1.0f), mul2(f2(2.0f), sr.hi));

    // plane
    const df3_2 N = df2_cross(df3_2_sub(V[0], V[1]), df3_2_sub(V[2], V[1]));
    const df3_2 Nh = normalize3_2(N);
    const df2 dN = df2_dot(V[0], Nh);

    const size_t TT = (size_t)T;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (c == 1 && !has1) break;
        const int t = t0 + c;
        const bool bad = c ? bad1 : bad0;
        auto pick = [c](float2 v) { return c ? v.y : v.x; };
        if (bad) {
#pragma unroll
            for (int f = 0; f < REC_F; ++f) rec[f * TT + t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            continue;
        }
        const unsigned ties = first_positive_c(pick(n1.x.hi), pick(n1.y.hi), pick(n1.z.hi)) |
                              (first_positive_c(pick(n2.x.hi), pick(n2.y.hi), pick(n2.z.hi)) << 1) |
                              (first_positive_c(pick(n3.x.hi), pick(n3.y.hi), pick(n3.z.hi)) << 2);
        rec[RF_CAP * TT + t] = make_float4(pick(Sh.x.hi), pick(Sh.y.hi), pick(Sh.z.hi), pick(slen.hi));
        rec[RF_CAP2 * TT + t] = make_float4(pick(sr.hi), pick(K), pick(inv2sr), 1.0f);
        rec[RF_N1 * TT + t] = make_float4(pick(n1.x.hi), pick(n1.y.hi), pick(n1.z.hi), __uint_as_float(ties));
        rec[RF_N2 * TT + t] = make_float4(pick(n2.x.hi), pick(n2.y.hi), pick(n2.z.hi), 0.0f);
        rec[RF_N3 * TT + t] = make_float4(pick(n3.x.hi), pick(n3.y.hi), pick(n3.z.hi), 0.0f);
        rec[RF_PL * TT + t] = make_float4(pick(Nh.x.hi), pick(Nh.y.hi), pick(Nh.z.hi), pick(dN.hi));
        rec[RF_N1L * TT + t] = make_float4(pick(n1.x.lo), pick(n1.y.lo), pick(n1.z.lo), pick(Sh.x.lo));
        rec[RF_N2L * TT + t] = make_float4(pick(n2.x.lo), pick(n2.y.lo), pick(n2.z.lo), pick(Sh.y.lo));
        rec[RF_N3L * TT + t] = make_float4(pick(n3.x.lo), pick(n3.y.lo), pick(n3.z.lo), pick(Sh.z.lo));
        rec[RF_PLL * TT + t] = make_float4(pick(Nh.x.lo), pick(Nh.y.lo), pick(Nh.z.lo), 0.0f);
    }
}

}  // namespace

vsr_status launch_setup(const float* tris, int T, const float cam[12], float4* rec, cudaStream_t st)
{
    if (T == 0) return VSR_OK;
    Cam c;
    for (int q = 0; q < 3; ++q) c.O[q] = cam[q];
    for (int q = 0; q < 9; ++q) c.M[q] = cam[3 + q];
    const int pairs = (T + 1) / 2;
    setup_pair_kernel<false><<<(pairs + 127) / 128, 128, 0, st>>>(tris, T, c, nullptr, rec);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_setup_views(const float* tris, int T, const float* cams_dev, int nviews, float4* rec,
                              cudaStream_t st)
{
    if (T == 0 || nviews == 0) return VSR_OK;
    Cam c = {};
    const int pairs = (T + 1) / 2;
    setup_pair_kernel<true><<<dim3((pairs + 127) / 128, nviews), 128, 0, st>>>(tris, T, c, cams_dev, rec);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}
