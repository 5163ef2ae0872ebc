// map.cu -- perspective-map generation (Universal perspective 2D->3D,
// Sec. 2 "Transformation of 2D->3D coordinates"; global delta, Sec. 1.1.1)
// and the per-tile view cones used by the binner.
//
// One CTA per 16x16 tile.  The map function is evaluated once per pixel
// centre of the tile plus a one-pixel halo into shared memory (18x18 = 324
// evaluations for 256 pixels), the global delta comes from central
// differences of those values, and the tile's view cone is reduced in the
// same CTA, so the map is written exactly once (16 B/px, HBM-write bound).
#include <math.h>

#include "vsr_internal.cuh"

namespace {

struct MapP {
    float k, l;
    float inv_k;   // 1 / k (k != 0)
    float tk;      // tan(k Omega/2)              (k > 0)
    float sk;      // sin(k Omega/2)              (k < 0)
    float half;    // Omega/2 in radians
    float inv_ls;  // 1 / (l (1 - s) + s)
    float sc;      // view-coordinate scale: x = (2i + 1 - W) sc, y = (2j + 1 - H) sc
    int kind;      // 1: k > 0, 0: k == 0, -1: k < 0
};

// Universal perspective direction of view coordinates (x, y).
__device__ __forceinline__ bool universal_dir(float x, float y, const MapP& p, float3& v)
{
    float R = sqrtf(fmaf(x, x, p.l * y * y));
    float th;
    float lim;  // lim_{R -> 0} sin(theta)/R
    if (p.kind > 0) {
        th = atanf(p.tk * R) * p.inv_k;
        lim = p.tk * p.inv_k;
    } else if (p.kind == 0) {
        th = p.half * R;
        lim = p.half;
    } else {
        float arg = p.sk * R;
        if (arg > 1.0f || arg < -1.0f) return false;
        th = asinf(arg) * p.inv_k;
        lim = p.sk * p.inv_k;
    }
    float st, ct;
    sincosf(th, &st, &ct);
    const float sor = R > 0.0f ? __fdividef(st, R) : lim;
    float wx = x * sor, wy = y * sor * p.inv_ls, wz = ct;
    float inv = rsqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    // one Newton step on the reciprocal square root keeps |v| = 1 to ~1 ulp
    float n2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
    inv = inv * fmaf(-0.5f * n2 * inv, inv, 1.5f);
    v = make_float3(wx * inv, wy * inv, wz * inv);
    return true;
}

// Map function at pixel centre (i, j) (may lie outside the picture).
__device__ __forceinline__ bool map_fn(int i, int j, int W, int H, const MapP& p, float3& v)
{
    const float x = (float)(2 * i + 1 - W) * p.sc;
    const float y = (float)(2 * j + 1 - H) * p.sc;
    return universal_dir(x, y, p, v);
}

// Tile cone from per-pixel (valid, G, h), reduced by the TILE_PIX / P pixel
// threads of a CTA, each holding P pixels (threads 0 .. TILE_PIX/P - 1, all
// of which must call it; other threads of the CTA must not) on named
// barrier 1: two rounds of warp shuffles, each closed by one barrier.  Every
// thread forms the axis itself from the warp partials (the same sums in the
// same order, so the same bits everywhere), so no single thread's work sits
// between the barriers.
template <int NT>
__device__ __forceinline__ void cone_barrier()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// h_gen (optional): the map's widest-ramp word, (generation << 32) | float
// bits of the largest ramp half-width; thread 0 raises it to this tile's
// with generation gen (a 64-bit maximum: a word left by an earlier
// generation is below every value of this one, so nothing clears it).
template <int P>
__device__ void reduce_cone(const bool (&valid)[P], const float3 (&G)[P], const float (&hp)[P], Cone* out,
                            float4* geom, unsigned long long* h_gen = nullptr, uint32_t gen = 0)
{
    constexpr int NT = TILE_PIX / P, CONE_WARPS = NT / 32;
    static_assert(NT % 32 == 0, "whole warps of pixel threads");
    __shared__ float4 part[CONE_WARPS];
    __shared__ float2 part2[CONE_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float sx = 0.0f, sy = 0.0f, sz = 0.0f, cnt = 0.0f;
#pragma unroll
    for (int q = 0; q < P; ++q)
        if (valid[q]) {
            sx += G[q].x;
            sy += G[q].y;
            sz += G[q].z;
            cnt += 1.0f;
        }
    for (int o = 16; o; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) part[warp] = make_float4(sx, sy, sz, cnt);
    cone_barrier<NT>();
    float a = 0.0f, b = 0.0f, c = 0.0f, n = 0.0f;
#pragma unroll
    for (int w = 0; w < CONE_WARPS; ++w) {
        const float4 q = part[w];
        a += q.x;
        b += q.y;
        c += q.z;
        n += q.w;
    }
    const float len = sqrtf(a * a + b * b + c * c);
    float ax = 0.0f, ay = 0.0f, az = 1.0f;
    if (len > 1e-6f * fmaxf(n, 1.0f)) {
        const float inv = 1.0f / len;
        ax = a * inv;
        ay = b * inv;
        az = c * inv;
    }
    float cmin = 2.0f, hmax = 0.0f;
#pragma unroll
    for (int q = 0; q < P; ++q)
        if (valid[q]) {
            cmin = fminf(cmin, G[q].x * ax + G[q].y * ay + G[q].z * az);
            hmax = fmaxf(hmax, hp[q]);
        }
    for (int o = 16; o; o >>= 1) {
        cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
        hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    }
    if (lane == 0) part2[warp] = make_float2(cmin, hmax);
    cone_barrier<NT>();
    if (threadIdx.x == 0) {
        float cm = 2.0f, hh = 0.0f;
#pragma unroll
        for (int w = 0; w < CONE_WARPS; ++w) {
            cm = fminf(cm, part2[w].x);
            hh = fmaxf(hh, part2[w].y);
        }
        // widen by a margin that covers the FP32 rounding of the dot products
        float ca = fmaxf(-1.0f, fminf(1.0f, cm - 2e-6f));
        if (n == 0.0f) ca = 1.0f;
        const float sa = sqrtf(fmaxf(0.0f, 1.0f - ca * ca));
        const Cone cone{make_float4(ax, ay, az, ca), make_float4(sa, hh, n, 0.0f)};
        *out = cone;
        // the tile's half-angle and the latitude / longitude of its axis, for
        // the tile index (the same functions the index would apply)
        const float4 g =
            make_float4(acosf(ca), asinf(fmaxf(-1.0f, fminf(1.0f, ay))), atan2f(ax, az), n > 0.0f ? hh : -1.0f);
        *geom = g;
        if (h_gen && g.w >= 0.0f) atomicMax(h_gen, ((unsigned long long)gen << 32) | __float_as_uint(hh));
    }
}

constexpr int HW = TILE + 2;
constexpr int MAP_THREADS = ((HW * HW + 31) / 32) * 32;  // one halo evaluation per thread
// threads and resident CTAs of the map kernel with P pixels per thread: one
// halo evaluation per thread at P = 1, else the tile's TILE_PIX / P pixel
// threads evaluate the halo in turns
constexpr int map_threads(int P) { return P == 1 ? MAP_THREADS : TILE_PIX / P; }
constexpr int map_ctas(int P) { return P == 1 ? 5 : (P == 2 ? 10 : 16); }
// pixels per thread of the map kernel: 2 (measured on the 1080p frame:
// map || set-up 68.4 -> 61.7 us, a new lens's map + tile index 67.9 -> 61.5
// us against 1; 4: 65.4 / 62.4 us) -- half the pixel threads share the cone
// reduction's shuffles and barriers, and no register spills
#ifndef VSR_MAP_PPT
#define VSR_MAP_PPT 2
#endif

// One pixel of the tile (li, lj) from the staged map values: the global
// delta from central differences over neighbours of the same chart
// (one-sided next to an unusable neighbour), the map row and, with deriv,
// the differences; returns whether the pixel is valid, its direction and its
// ramp half-width.
__device__ __forceinline__ void map_pixel(const float4* sv, int li, int lj, int i, int j, int W, int H, float4* map,
                                          float4* deriv, bool& valid, float3& G, float& h)
{
    const int c = (lj + 1) * HW + (li + 1);
    valid = false;
    G = make_float3(0.0f, 0.0f, 0.0f);
    h = 0.0f;
    if (i < W && j < H) {
        float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 qc = sv[c];
        const float cc = qc.w;
        if (cc != 0.0f) {
            const float3 vc = make_float3(qc.x, qc.y, qc.z);
            const float4 qL = sv[c - 1], qR = sv[c + 1], qU = sv[c - HW], qD = sv[c + HW];
            const bool uL = qL.w == cc, uR = qR.w == cc, uU = qU.w == cc, uD = qD.w == cc;
            float fw = 0.0f;
            float dv[6];
            if (uL && uR && uU && uD) {
                // every neighbour usable (almost every pixel): central differences
                const float a[3] = {qR.x - qL.x, qR.y - qL.y, qR.z - qL.z};
                const float b[3] = {qD.x - qU.x, qD.y - qU.y, qD.z - qU.z};
#pragma unroll
                for (int comp = 0; comp < 3; ++comp) {
                    dv[comp] = a[comp] * 0.5f;
                    dv[3 + comp] = b[comp] * 0.5f;
                    fw = fmaxf(fw, fabsf(dv[comp]) + fabsf(dv[3 + comp]));
                }
            } else {
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                auto get = [&](const float4& q) { return comp == 0 ? q.x : (comp == 1 ? q.y : q.z); };
                const float vcc = comp == 0 ? vc.x : (comp == 1 ? vc.y : vc.z);
                float di, dj;
                if (uL && uR)
                    di = (get(qR) - get(qL)) * 0.5f;
                else if (uR)
                    di = get(qR) - vcc;
                else if (uL)
                    di = vcc - get(qL);
                else
                    di = 0.0f;
                if (uU && uD)
                    dj = (get(qD) - get(qU)) * 0.5f;
                else if (uD)
                    dj = get(qD) - vcc;
                else if (uU)
                    dj = vcc - get(qU);
                else
                    dj = 0.0f;
                fw = fmaxf(fw, fabsf(di) + fabsf(dj));
                dv[comp] = di;
                dv[3 + comp] = dj;
            }
            }
            if (fw > 0.0f) {
                o = make_float4(vc.x, vc.y, vc.z, __frcp_rn(fw));
                valid = true;
                G = vc;
                h = 0.5f / o.w;  // exactly the raster kernel's ramp half-width
                if (deriv) {
                    // pstep ramp half-width bound for any unit normal n:
                    // (|n.d_i G| + |n.d_j G|)/2 <= (|d_i G| + |d_j G|)/2
                    const float ni = sqrtf(fmaf(dv[0], dv[0], fmaf(dv[1], dv[1], dv[2] * dv[2])));
                    const float nj = sqrtf(fmaf(dv[3], dv[3], fmaf(dv[4], dv[4], dv[5] * dv[5])));
                    h = fmaxf(h, 0.5f * (ni + nj) * 1.000001f);
                }
            }
            if (deriv) {
                deriv[2 * ((size_t)j * W + i)] = valid ? make_float4(dv[0], dv[1], dv[2], 0.0f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                deriv[2 * ((size_t)j * W + i) + 1] = valid ? make_float4(dv[3], dv[4], dv[5], 0.0f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        map[(size_t)j * W + i] = o;
    }
}

// One 16x16 tile of a map: the map function F at every pixel centre of the
// tile and its one-pixel halo (F(i, j, v) returns 0 where the map is
// undefined, else 1 + the pixel's chart -- the face of a cube map, 0 for
// single-chart maps), then map_pixel for each pixel of the tile, P pixels
// per thread (rows lj and lj + 16/P ...), and the tile cone.
// deriv (optional): the differences (d_i G, d_j G) the delta is formed
// from, 2 float4 per pixel, for the per-fragment pixel step; the tile
// cones then carry the widest ramp of either step.
template <class F, int P>
__global__ void __launch_bounds__(map_threads(P), map_ctas(P)) map_kernel(int W, int H, F fn, float4* __restrict__ map,
                                                                         Cone* __restrict__ tiles,
                                                                         float4* __restrict__ geom,
                                                                         float4* __restrict__ deriv,
                                                                         unsigned long long* h_gen, uint32_t gen)
{
    // map values of the tile and its halo: direction xyz, w = F's return value
    __shared__ float4 sv[HW * HW];
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int i0 = tx * TILE - 1, j0 = ty * TILE - 1;
    for (int q = threadIdx.x; q < HW * HW; q += map_threads(P)) {
        const int qi = q % HW, qj = q / HW;
        float3 v = make_float3(0.0f, 0.0f, 0.0f);
        const int ok = fn(i0 + qi, j0 + qj, W, H, v);
        sv[q] = make_float4(v.x, v.y, v.z, (float)ok);
    }
    __syncthreads();
    constexpr int NT = TILE_PIX / P;
    if (threadIdx.x >= NT) return;  // halo-only threads: done
    const int li = threadIdx.x % TILE, lj0 = threadIdx.x / TILE;
    bool valid[P];
    float3 G[P];
    float h[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int lj = lj0 + q * (TILE / P);
        map_pixel(sv, li, lj, tx * TILE + li, ty * TILE + lj, W, H, map, deriv, valid[q], G[q], h[q]);
    }
    const int t = ty * gridDim.x + tx;
    reduce_cone<P>(valid, G, h, &tiles[t], &geom[t], h_gen, gen);
}

// The Universal perspective map function.
struct UniversalFn {
    MapP p;
    __device__ __forceinline__ int operator()(int i, int j, int W, int H, float3& v) const
    {
        return map_fn(i, j, W, H, p, v) ? 1 : 0;
    }
};

__device__ __forceinline__ float3 normalized(float x, float y, float z)
{
    const float n2 = fmaf(x, x, fmaf(y, y, z * z));
    float inv = rsqrtf(n2);
    inv = inv * fmaf(-0.5f * n2 * inv, inv, 1.5f);  // one Newton step: |v| = 1 to ~1 ulp
    return make_float3(x * inv, y * inv, z * inv);
}

// The other projections of Sec. 2.2 and the Brown-Conrady distortion of the
// view coordinates (Sec. 2.3), see vsr_map_spec.
struct SpecFn {
    int kind;
    MapP p;          // Universal lens; p.sc = view-coordinate scale of the AOV type
    float cot_half;  // rectilinear: cot(Omega/2)
    float d[6];      // k1, k2, p1, p2, q1, q2
    float a[4];      // panorama: Omega_h (rad), height; dome: compression + pi/2 (rad), cos tilt, sin tilt, offset

    __device__ __forceinline__ int operator()(int i, int j, int W, int H, float3& v) const
    {
        if (kind == VSR_MAP_UNIVERSAL || kind == VSR_MAP_RECTILINEAR) {
            const float x = (float)(2 * i + 1 - W) * p.sc, y = (float)(2 * j + 1 - H) * p.sc;
            const float r2 = fmaf(x, x, y * y);
            const float rad = fmaf(d[1] * r2, r2, fmaf(d[0], r2, 1.0f));
            const float pr = fmaf(d[2], x, d[3] * y);
            const float xd = fmaf(x, rad, fmaf(x, pr, d[4] * r2));
            const float yd = fmaf(y, rad, fmaf(y, pr, d[5] * r2));
            if (kind == VSR_MAP_UNIVERSAL) return universal_dir(xd, yd, p, v) ? 1 : 0;
            v = normalized(xd, yd, cot_half);
            return 1;
        }
        const float fs = ((float)i + 0.5f) / (float)W, ft = ((float)j + 0.5f) / (float)H;
        if (kind == VSR_MAP_PANORAMA) {
            float sx, cx;
            sincosf(a[0] * (fs - 0.5f), &sx, &cx);
            v = normalized(sx, a[1] * (ft - 0.5f), cx);
            return 1;
        }
        if (kind == VSR_MAP_DOME) {
            const float fx = 2.0f * fs - 1.0f, fy = 1.0f - 2.0f * ft;
            const float R = sqrtf(fmaf(fx, fx, fy * fy));
            if (R > 1.0f) return 0;
            float st, ct;
            sincosf(R * a[0], &st, &ct);
            const float sor = R > 0.0f ? st / R : a[0];
            const float3 w = normalized(fx * sor, ct, fmaf(fy, sor, a[3]));
            v = make_float3(w.x, fmaf(w.y, a[1], w.z * a[2]), fmaf(-w.y, a[2], w.z * a[1]));
            return 1;
        }
        if (kind == VSR_MAP_EQUIRECT) {
            float sx, cx, sy, cy;
            sincospif(2.0f * fs - 1.0f, &sx, &cx);
            sincospif(ft, &sy, &cy);
            v = make_float3(sx * sy, -cy, cx * sy);
            return 1;
        }
        // cube: face = floor(6 f_s), rows of the face rotation (world = M u)
        const float s6 = 6.0f * fs;
        const int face = (int)floorf(s6);
        if (face < 0 || face > 5) return 0;  // beyond the strip
        const float3 u = normalized(s6 - (float)face - 0.5f, ft - 0.5f, 0.5f);
        switch (face) {
        case 0: v = make_float3(u.z, -u.x, -u.y); break;   // [ Z, -X, -Y]
        case 1: v = make_float3(-u.z, u.x, -u.y); break;   // [-Z,  X, -Y]
        case 2: v = make_float3(u.x, -u.y, -u.z); break;   // [ X, -Y, -Z]
        case 3: v = u; break;                               // [ X,  Y,  Z]: the front face
        case 4: v = make_float3(u.x, u.z, -u.y); break;    // [ X,  Z, -Y]
        default: v = make_float3(-u.x, -u.z, -u.y); break; // [-X, -Z, -Y]
        }
        return 1 + face;
    }
};

// Cones of a map supplied by the caller.
__global__ void __launch_bounds__(TILE_PIX) cone_kernel(const float4* __restrict__ map, int W, int H,
                                                         Cone* __restrict__ tiles, float4* __restrict__ geom,
                                                         unsigned long long* h_gen, uint32_t gen)
{
    const int li = threadIdx.x % TILE, lj = threadIdx.x / TILE;
    const int i = blockIdx.x * TILE + li, j = blockIdx.y * TILE + lj;
    bool valid = false;
    float3 G = make_float3(0.0f, 0.0f, 0.0f);
    float h = 0.0f;
    if (i < W && j < H) {
        float4 o = map[(size_t)j * W + i];
        if (o.w > 0.0f) {
            valid = true;
            G = make_float3(o.x, o.y, o.z);
            h = 0.5f / o.w;
        }
    }
    const bool vv[1] = {valid};
    const float3 gg[1] = {G};
    const float hh[1] = {h};
    const int t = blockIdx.y * gridDim.x + blockIdx.x;
    reduce_cone<1>(vv, gg, hh, &tiles[t], &geom[t], h_gen, gen);
}

}  // namespace

namespace {

// per-map scalars, formed once in double precision and rounded to float
MapP make_params(int W, int H, int aov, float k, float l, float s, float omega_deg)
{
    MapP p;
    double half = (double)omega_deg * M_PI / 360.0;
    p.k = k;
    p.l = l;
    p.kind = k > 0.0f ? 1 : (k < 0.0f ? -1 : 0);
    p.inv_k = k != 0.0f ? (float)(1.0 / (double)k) : 0.0f;
    p.tk = (float)tan((double)k * half);
    p.sk = (float)sin((double)k * half);
    p.half = (float)half;
    p.inv_ls = (float)(1.0 / ((double)l * (1.0 - (double)s) + (double)s));
    switch (aov) {
    case VSR_AOV_DIAGONAL: p.sc = (float)(1.0 / sqrt((double)W * W + (double)H * H)); break;
    case VSR_AOV_VERTICAL: p.sc = (float)(1.0 / H); break;
    case VSR_AOV_H4X3: p.sc = (float)(0.75 / H); break;
    default: p.sc = (float)(1.0 / W); break;
    }
    return p;
}

}  // namespace

vsr_status launch_map(int W, int H, int aov, float k, float l, float s, float omega_deg, float4* map, Cone* tiles,
                      float4* geom, unsigned long long* h_gen, uint32_t gen, cudaStream_t st)
{
    const MapP p = make_params(W, H, aov, k, l, s, omega_deg);
    dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE);
    map_kernel<UniversalFn, VSR_MAP_PPT>
        <<<grid, map_threads(VSR_MAP_PPT), 0, st>>>(W, H, UniversalFn{p}, map, tiles, geom, nullptr, h_gen, gen);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_map_spec(const vsr_map_spec& sp, float4* map, Cone* tiles, float4* geom, float4* deriv,
                           unsigned long long* h_gen, uint32_t gen, cudaStream_t st)
{
    SpecFn f;
    f.kind = sp.kind;
    f.p = make_params(sp.W, sp.H, sp.aov, sp.param[0], sp.param[1], sp.param[2], sp.param[3]);
    f.cot_half = (float)(1.0 / tan((double)sp.param[0] * M_PI / 360.0));
    for (int q = 0; q < 6; ++q) f.d[q] = sp.distortion[q];
    for (int q = 0; q < 4; ++q) f.a[q] = 0.0f;
    if (sp.kind == VSR_MAP_PANORAMA) {
        f.a[0] = (float)((double)sp.param[0] * M_PI / 180.0);
        f.a[1] = sp.param[1];
    } else if (sp.kind == VSR_MAP_DOME) {
        f.a[0] = (float)((double)sp.param[0] * M_PI / 180.0 + 0.5 * M_PI);
        f.a[1] = (float)cos((double)sp.param[1] * M_PI / 180.0);
        f.a[2] = (float)sin((double)sp.param[1] * M_PI / 180.0);
        f.a[3] = sp.param[2];
    }
    dim3 grid((sp.W + TILE - 1) / TILE, (sp.H + TILE - 1) / TILE);
    map_kernel<SpecFn, VSR_MAP_PPT>
        <<<grid, map_threads(VSR_MAP_PPT), 0, st>>>(sp.W, sp.H, f, map, tiles, geom, deriv, h_gen, gen);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_map_cones(const float4* map, int W, int H, Cone* tiles, float4* geom, unsigned long long* h_gen,
                            uint32_t gen, cudaStream_t st)
{
    dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE);
    cone_kernel<<<grid, TILE_PIX, 0, st>>>(map, W, H, tiles, geom, h_gen, gen);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}


// ---------------------------------------------------------------------------
// Map adjoint: the lens gradient dL/d(k, l, s, Omega in degrees) from the
// per-pixel gradients (dG, d delta) of the map, by forward-mode tangents of
// the map function (the chain rule through the 2D->3D transform of Sec. 2)
// and of the global delta (reading of fwidth as central differences,
// Sec. 1.1.1), contracted per pixel and reduced per CTA; a one-CTA pass sums
// the CTA partials in double precision in a fixed order.
//
//   R = sqrt(x^2 + l y^2)                      dR/dl = y^2/(2R)
//   k > 0: theta = atan(tan(a) R)/k, a = k Omega/2
//   k = 0: theta = (Omega/2) R                 (flat in k: both branches agree
//                                               to second order at k = 0)
//   k < 0: theta = asin(sin(a) R)/k
//   w = (x sin(theta)/R, y sin(theta)/R / (l(1-s)+s), cos(theta)), v = w/|w|
//   delta = 1/fw, fw = max_c (|d_i v_c| + |d_j v_c|): the derivative of the
//   maximising component (first maximum) with the signs of its differences.
// The gradient is the one of the map at its effective parameters (after the
// parameter limits).
namespace {

struct TanP {
    MapP p;
    float s;
    float ck;  // cos(k Omega/2)
};

constexpr float DEG_HALF = 0.00872664625997164788f;  // d(Omega/2 in rad)/d(Omega in deg) = pi/360

// tangents dv[q] = dv/dparam_q (q = k, l, s, Omega) at pixel centre (i, j);
// false where the map is undefined
__device__ __forceinline__ bool map_tangent(int i, int j, int W, int H, const TanP& tp, float3& v, float3 dv[4])
{
    const MapP& p = tp.p;
    if (!map_fn(i, j, W, H, p, v)) return false;
#pragma unroll
    for (int q = 0; q < 4; ++q) dv[q] = make_float3(0.0f, 0.0f, 0.0f);
    const float x = (float)(2 * i + 1 - W) * p.sc;
    const float y = (float)(2 * j + 1 - H) * p.sc;
    const float R = sqrtf(fmaf(x, x, p.l * y * y));
    if (!(R > 0.0f)) return true;  // the optical axis: v = (0, 0, 1) for every lens
    const float dR[4] = {0.0f, y * y / (2.0f * R), 0.0f, 0.0f};
    float th, dth[4];
    if (p.kind > 0) {
        const float u = p.tk * R;
        th = atanf(u) * p.inv_k;
        const float sec2 = fmaf(p.tk, p.tk, 1.0f);
        const float dtk[4] = {sec2 * p.half, 0.0f, 0.0f, sec2 * p.k * DEG_HALF};
        const float w = p.inv_k / fmaf(u, u, 1.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q) dth[q] = fmaf(dtk[q], R, p.tk * dR[q]) * w;
        dth[0] -= th * p.inv_k;
    } else if (p.kind == 0) {
        th = p.half * R;
        dth[0] = 0.0f;
        dth[1] = p.half * dR[1];
        dth[2] = 0.0f;
        dth[3] = DEG_HALF * R;
    } else {
        const float u = p.sk * R;
        th = asinf(u) * p.inv_k;
        const float dsk[4] = {tp.ck * p.half, 0.0f, 0.0f, tp.ck * p.k * DEG_HALF};
        const float w = p.inv_k * rsqrtf(fmaxf(fmaf(-u, u, 1.0f), 1e-30f));
#pragma unroll
        for (int q = 0; q < 4; ++q) dth[q] = fmaf(dsk[q], R, p.sk * dR[q]) * w;
        dth[0] -= th * p.inv_k;
    }
    float st, ct;
    sincosf(th, &st, &ct);
    const float sor = st / R;
    const float il = p.inv_ls;
    const float dil[4] = {0.0f, -il * il * (1.0f - tp.s), -il * il * (1.0f - p.l), 0.0f};
    const float wx = x * sor, wy = y * sor * il, wz = ct;
    const float n = sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    const float inv = 1.0f / n;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float dsor = (ct * dth[q] - sor * dR[q]) / R;
        const float dwx = x * dsor;
        const float dwy = y * fmaf(dsor, il, sor * dil[q]);
        const float dwz = -st * dth[q];
        const float pr = (wx * dwx + wy * dwy + wz * dwz) * inv * inv;
        dv[q] = make_float3((dwx - wx * pr) * inv, (dwy - wy * pr) * inv, (dwz - wz * pr) * inv);
    }
    return true;
}

__global__ void __launch_bounds__(MAP_THREADS) map_backward_kernel(int W, int H, TanP tp,
                                                                    const float4* __restrict__ dmap,
                                                                    float* __restrict__ partials)
{
    __shared__ float3 sv[HW * HW];
    __shared__ float3 sd[4][HW * HW];
    __shared__ unsigned char sok[HW * HW];
    __shared__ float red[4][MAP_THREADS / 32];
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int i0 = tx * TILE - 1, j0 = ty * TILE - 1;
    if (threadIdx.x < HW * HW) {
        const int q = threadIdx.x, qi = q % HW, qj = q / HW;
        float3 v = make_float3(0.0f, 0.0f, 0.0f), dv[4];
        const bool ok = map_tangent(i0 + qi, j0 + qj, W, H, tp, v, dv);
        sv[q] = v;
        sok[q] = ok;
#pragma unroll
        for (int k = 0; k < 4; ++k) sd[k][q] = ok ? dv[k] : make_float3(0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (threadIdx.x < TILE_PIX) {
        const int li = threadIdx.x % TILE, lj = threadIdx.x / TILE;
        const int i = tx * TILE + li, j = ty * TILE + lj;
        const int c = (lj + 1) * HW + (li + 1);
        if (i < W && j < H && sok[c]) {
            const float4 dm = dmap[(size_t)j * W + i];
            const int L = c - 1, Rr = c + 1, U = c - HW, D = c + HW;
            // the map kernel's fwidth, with the maximising component's tangent
            float fw = 0.0f, dfw[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                auto get = [&](const float3& a) { return comp == 0 ? a.x : (comp == 1 ? a.y : a.z); };
                int ia = c, ib = c, ja = c, jb = c;  // di = (v[ia] - v[ib]) * fi, dj likewise
                float fi = 0.0f, fj = 0.0f;
                if (sok[L] && sok[Rr]) { ia = Rr; ib = L; fi = 0.5f; }
                else if (sok[Rr]) { ia = Rr; fi = 1.0f; }
                else if (sok[L]) { ib = L; fi = 1.0f; }
                if (sok[U] && sok[D]) { ja = D; jb = U; fj = 0.5f; }
                else if (sok[D]) { ja = D; fj = 1.0f; }
                else if (sok[U]) { jb = U; fj = 1.0f; }
                const float di = fi == 0.0f ? 0.0f : (fi == 0.5f ? (get(sv[ia]) - get(sv[ib])) * 0.5f
                                                                 : get(sv[ia]) - get(sv[ib]));
                const float dj = fj == 0.0f ? 0.0f : (fj == 0.5f ? (get(sv[ja]) - get(sv[jb])) * 0.5f
                                                                 : get(sv[ja]) - get(sv[jb]));
                const float f = fabsf(di) + fabsf(dj);
                if (f > fw) {
                    fw = f;
                    const float si = di > 0.0f ? fi : (di < 0.0f ? -fi : 0.0f);
                    const float sj = dj > 0.0f ? fj : (dj < 0.0f ? -fj : 0.0f);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        dfw[k] = si * (get(sd[k][ia]) - get(sd[k][ib])) + sj * (get(sd[k][ja]) - get(sd[k][jb]));
                }
            }
            if (fw > 0.0f) {
                const float dd = -dm.w / (fw * fw);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float3 t = sd[k][c];
                    acc[k] = fmaf(dm.x, t.x, fmaf(dm.y, t.y, fmaf(dm.z, t.z, dd * dfw[k])));
                }
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float a = acc[k];
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[k][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float a = 0.0f;
        for (int w = 0; w < MAP_THREADS / 32; ++w) a += red[threadIdx.x][w];
        partials[(size_t)(ty * gridDim.x + tx) * 4 + threadIdx.x] = a;
    }
}

__global__ void __launch_bounds__(256) lens_reduce_kernel(const float* __restrict__ partials, int nblocks,
                                                          double* __restrict__ dlens)
{
    __shared__ double red[4][256];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += 256)
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] += (double)partials[(size_t)b * 4 + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) dlens[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

size_t map_backward_partials(int W, int H)
{
    return (size_t)((W + TILE - 1) / TILE) * (size_t)((H + TILE - 1) / TILE) * 4;
}

vsr_status launch_map_backward(int W, int H, int aov, float k, float l, float s, float omega_deg,
                               const float4* dmap, float* partials, double* dlens, cudaStream_t st)
{
    TanP tp;
    tp.p = make_params(W, H, aov, k, l, s, omega_deg);
    tp.s = s;
    tp.ck = (float)cos((double)k * (double)omega_deg * M_PI / 360.0);
    dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE);
    map_backward_kernel<<<grid, MAP_THREADS, 0, st>>>(W, H, tp, dmap, partials);
    VSR_CUDA_TRY(cudaGetLastError());
    lens_reduce_kernel<<<1, 256, 0, st>>>(partials, (int)(grid.x * grid.y), dlens);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}
