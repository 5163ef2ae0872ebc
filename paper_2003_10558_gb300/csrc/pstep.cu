// pstep.cu -- coverage / depth / visibility with the per-fragment pixel
// step (Sec. 1.1.1): each of the four plane distances g of the
// rasterization equation ramps over its own fwidth,
//   w = |d_i g| + |d_j g|,  d g = n . d G  (edges),  (S-hat . d G)/sin(rho)
//   (miter, whose distance carries the same 1/sin(rho)),
// with d_i G, d_j G the map's own central differences (stored with the map),
// instead of the map-wide global delta:
//   fragment iff every g > -w/2 (bpxstep),  m^f = min clamp(g/w + 1/2, 0, 1)
// Everything else -- tile-centred distances, the order-free merge, the
// visibility key -- is the coverage kernel's (raster.cu).  A variant of
// quality, not of speed: one CTA per tile over its whole bin.
#include "stage.cuh"

namespace {

constexpr int PT = 128;  // threads per CTA: one 16x16 tile, two pixels per thread
constexpr int PPT = 2;
static_assert(PT == STAGE_CHUNK && PT * PPT == TILE_PIX, "tile layout");

__device__ __forceinline__ float absdot(const float4& n, const float3& d)
{
    return fabsf(fmaf(n.x, d.x, fmaf(n.y, d.y, n.z * d.z)));
}

__global__ void __launch_bounds__(PT) raster_pstep_kernel(RasterView v, const float4* __restrict__ deriv,
                                                           int* __restrict__ status)
{
    __shared__ Stage st;
    const int tile = blockIdx.x;
    const int W = v.W, H = v.H, T = v.T;
    const size_t TT = (size_t)T;
    const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = tx * TILE + (warp & 1) * 8 + (lane & 7);
    const int py0 = ty * TILE + (warp >> 1) * 8 + (lane >> 3);
    const Cone tc = v.tiles[tile];
    const float ax = tc.c0.x, ay = tc.c0.y, az = tc.c0.z;

    float gx[PPT], gy[PPT], gz[PPT], dgx[PPT], dgy[PPT], dgz[PPT], hp[PPT], eg[PPT];
    float3 di[PPT], dj[PPT];
    bool pv[PPT], inimg[PPT];
    uint32_t acc[PPT];
    unsigned long long key[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int py = py0 + 4 * p;
        inimg[p] = px < W && py < H;
        const size_t o = (size_t)py * W + px;
        float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f), a = g, b = g;
        if (inimg[p]) {
            g = v.map[o];
            a = deriv[2 * o];
            b = deriv[2 * o + 1];
        }
        pv[p] = g.w > 0.0f;
        gx[p] = g.x;
        gy[p] = g.y;
        gz[p] = g.z;
        di[p] = make_float3(a.x, a.y, a.z);
        dj[p] = make_float3(b.x, b.y, b.z);
        // the widest ramp half-width of any distance at this pixel
        hp[p] = pv[p] ? 0.5f * (sqrtf(fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z))) +
                                sqrtf(fmaf(b.x, b.x, fmaf(b.y, b.y, b.z * b.z)))) * 1.000001f
                      : 0.0f;
        eg[p] = pv[p] ? norm2_minus_one(g.x, g.y, g.z) : 0.0f;
        dgx[p] = g.x - ax;
        dgy[p] = g.y - ay;
        dgz[p] = g.z - az;
        acc[p] = 0u;
        key[p] = ~0ull;
    }

    // the warp's view cone (its 8x8 pixels), widened by the widest ramp
    float sx = 0.0f, sy = 0.0f, sz = 0.0f, cn = 0.0f, hw = 0.0f;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
        if (pv[p]) {
            sx += gx[p];
            sy += gy[p];
            sz += gz[p];
            cn += 1.0f;
            hw = fmaxf(hw, hp[p]);
        }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    sz = warp_sum(sz);
    const float wcnt = warp_sum(cn);
    const float wh = warp_max(hw);
    const float wl = sqrtf(sx * sx + sy * sy + sz * sz);
    const bool wdeg = !(wl > 1e-6f * fmaxf(wcnt, 1.0f));
    const float wax = wdeg ? 0.0f : sx / wl, way = wdeg ? 0.0f : sy / wl, waz = wdeg ? 1.0f : sz / wl;
    float cm = 2.0f;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
        if (pv[p]) cm = fminf(cm, gx[p] * wax + gy[p] * way + gz[p] * waz);
    float wcos = fmaxf(-1.0f, fminf(1.0f, warp_min(cm) - 2e-6f));
    if (wdeg) wcos = -1.0f;
    const float wsin = sqrtf(fmaxf(0.0f, 1.0f - wcos * wcos));
    const bool warp_active = wcnt > 0.0f;

    uint32_t b0 = 0, b1 = 0;
    if (tc.c1.z > 0.0f) {
        b0 = v.offsets[tile];
        b1 = v.ends ? v.ends[tile] : v.offsets[tile + 1];
        if (b1 > v.cap) {
            if (threadIdx.x == 0) raise_status(status, VSR_ERR_BIN_OVERFLOW);
            b1 = v.cap;
            b0 = min(b0, v.cap);
        }
    }
    for (uint32_t base = b0; base < b1; base += STAGE_CHUNK) {
        const int n = (int)min((uint32_t)STAGE_CHUNK, b1 - base);
#pragma unroll
        for (int p = 0; p < PPT; ++p) acc[p] = min(acc[p], COV_ONE);
        __syncthreads();
        if ((int)threadIdx.x < n) {
            const uint32_t t = v.ids[base + threadIdx.x];
            if (t >= (uint32_t)T) {
                raise_status(status, VSR_ERR_BIN_OVERFLOW);
                st.s6[threadIdx.x] = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(STAGE_EMPTY));
            } else {
                stage_triangle(v.rec, TT, t, ax, ay, az, st, threadIdx.x);
            }
        }
        __syncthreads();
        if (!warp_active) continue;
        for (int gbase = 0; gbase < n; gbase += 32) {
            bool keep = false;
            const int jj = gbase + lane;
            if (jj < n && __float_as_uint(st.s6[jj].w) != STAGE_EMPTY) {
                const float4 a = st.s0[jj];
                const float4 b = st.s1[jj];
                const float2 cap = pstep_cap(1.0f - 0.5f * b.y, b.x, wh);
                keep = cap_hits_cone(make_float3(a.x, a.y, a.z), cap.x, cap.y, make_float3(wax, way, waz), wcos, wsin,
                                     0.0f);
                const float lim = -(wh + wsin + (1.0f - wcos) + 1e-6f);
                const float4 n1 = st.s2[jj], n2 = st.s3[jj], n3 = st.s4[jj];
                keep = keep && fmaf(wax, n1.x, fmaf(way, n1.y, waz * n1.z)) > lim &&
                       fmaf(wax, n2.x, fmaf(way, n2.y, waz * n2.z)) > lim &&
                       fmaf(wax, n3.x, fmaf(way, n3.y, waz * n3.z)) > lim;
            }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            while (mask) {
                const int j = gbase + __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 a = st.s0[j], b = st.s1[j], e = st.s6[j];
                const float4 n1 = st.s2[j], n2 = st.s3[j], n3 = st.s4[j], pl = st.s5[j];
                const float inv_sr = 2.0f * b.z;
                const unsigned ties = __float_as_uint(a.w);
                const unsigned long long tbits = (unsigned long long)__float_as_uint(e.w);
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const float g1 = plane_distance(dgx[p], dgy[p], dgz[p], n1);
                    const float g2 = plane_distance(dgx[p], dgy[p], dgz[p], n2);
                    const float g3 = plane_distance(dgx[p], dgy[p], dgz[p], n3);
                    const float g4 = miter_distance(dgx[p], dgy[p], dgz[p], e, b, eg[p]);
                    const float w1 = absdot(n1, di[p]) + absdot(n1, dj[p]);
                    const float w2 = absdot(n2, di[p]) + absdot(n2, dj[p]);
                    const float w3 = absdot(n3, di[p]) + absdot(n3, dj[p]);
                    const float w4 = (absdot(a, di[p]) + absdot(a, dj[p])) * inv_sr;
                    const bool frag = pv[p] && g1 > -0.5f * w1 && g2 > -0.5f * w2 && g3 > -0.5f * w3 &&
                                      g4 > -0.5f * w4;
                    const float D = plane_distance(dgx[p], dgy[p], dgz[p], pl);
                    const float r = __fdividef(b.w, D);
                    const bool f = frag && __float_as_uint(r) - 1u < 0x7f7fffffu;  // 0 < r < inf
                    const float m = fminf(fminf(__saturatef(__fdividef(g1, fmaxf(w1, 1e-30f)) + 0.5f),
                                                __saturatef(__fdividef(g2, fmaxf(w2, 1e-30f)) + 0.5f)),
                                          fminf(__saturatef(__fdividef(g3, fmaxf(w3, 1e-30f)) + 0.5f),
                                                __saturatef(__fdividef(g4, fmaxf(w4, 1e-30f)) + 0.5f)));
                    acc[p] += f ? cov_fixed(m) : 0u;
                    const bool in = f && centre_inside(g1, g2, g3, fminf(fminf(g1, g2), g3), ties);
                    const unsigned long long k = ((unsigned long long)__float_as_uint(r) << 32) | tbits;
                    key[p] = in && k < key[p] ? k : key[p];
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (!inimg[p]) continue;
        const size_t o = (size_t)(py0 + 4 * p) * W + px;
        const bool hit = key[p] != ~0ull;
        if (v.out_id) v.out_id[o] = hit ? (uint32_t)(key[p] & 0xffffffffull) : 0xffffffffu;
        if (v.out_depth) v.out_depth[o] = hit ? __uint_as_float((uint32_t)(key[p] >> 32)) : INFINITY;
        if (v.out_cov) v.out_cov[o] = (float)min(acc[p], COV_ONE) * (1.0f / (float)COV_ONE);
    }
}

}  // namespace

vsr_status launch_raster_pstep(const RasterView& view, const float4* deriv, int* status, cudaStream_t st)
{
    const int ntiles = view.tiles_x * ((view.H + TILE - 1) / TILE);
    if (ntiles == 0) return VSR_OK;
    raster_pstep_kernel<<<ntiles, PT, 0, st>>>(view, deriv, status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}
