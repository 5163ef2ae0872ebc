// grad.cu -- the differentiable path: per-pixel fragment lists, the
// front-to-back merge of a shade pass, and its hand-written adjoint.
//
// Forward (vsr_raster_shaded).  The image is the paper's front-to-back mask
// merge (Sec. 1.4) applied to a shade pass, shade_t = c_t |N-hat_t . G|
// (the hard normal of Sec. 1.1.4):
//   over the fragments of a pixel in ascending (r, t):
//     m^fc = min(m^f, 1 - m^b);  I += m^fc shade;  m^b += m^fc
// Unlike coverage, the image depends on the order, so every fragment is
// kept: a count pass and a fill pass over the tile bins (the same template,
// so both see exactly the same fragments), an exclusive scan of the
// per-pixel counts in between, and each thread sorts and merges its own
// pixels' lists after the fill.  A fragment record is the float4
// (r, t, m^f, shade).
//
// Backward (vsr_raster_backward).  Per pixel, with upstream gradients dI,
// dcov, ddepth: the merge takes m^fc = m^f until the first fragment f* with
// m^f > 1 - m^b, which takes 1 - m^b and saturates the pixel, so
//   dI/d shade_f = m^fc_f,
//   dI/d m^f_f   = shade_f - shade_f* (f < f*; shade_f when nothing
//                  saturates), 0 from f* on,
//   dcov/d m^f_f = 1 when nothing saturates, else 0;
// m^f = clamp(delta min_i g_i + 1/2, 0, 1) (gpstep on the four plane
// distances) passes d g_i* = delta dm and d delta = g_i* dm to the
// minimising distance while the clamp is open; g_1..3 = G.n_i, g_4 =
// (G.S-hat - cos rho)/sin rho; depth r = (A'.N-hat)/(G.N-hat).  The
// per-triangle record gradients accumulate with float4 atomics; the
// per-pixel (dG, d delta) go to the map adjoint (map.cu), and the set-up
// adjoint below takes the record gradients to the world vertices.
#include "stage.cuh"

namespace {

constexpr int FT = 128;  // threads of a fragment-kernel CTA: one 16x16 tile, two pixels per thread
constexpr int PPT = 2;
static_assert(FT == STAGE_CHUNK && FT * PPT == TILE_PIX, "tile layout");

struct FragView {
    const float4* map;
    int W, H;
    const Cone* tiles;
    int tiles_x;
    const float4* rec;
    int T;
    const uint32_t* offsets;  // tile bins
    const uint32_t* ids;
    uint32_t cap;
    const float* colors;      // per triangle, NULL = 1
    uint32_t* counts;         // count pass: fragments per pixel
    const uint32_t* foff;     // fill pass: first fragment of each pixel (W*H + 1, exclusive scan)
    float4* frags;            // fill pass: (r, t bits, m^f, shade)
    uint32_t fcap;
    float* image;
    float* cov;
    uint32_t* out_id;
    float* out_depth;
    const uint32_t* ends;     // as RasterView::ends
};

__device__ __forceinline__ bool frag_less(const float4& a, const float4& b)
{
    return a.x < b.x || (a.x == b.x && __float_as_uint(a.y) < __float_as_uint(b.y));
}

template <bool FILL>
__global__ void __launch_bounds__(FT) frag_kernel(FragView v, int* __restrict__ status)
{
    __shared__ Stage st;
    __shared__ float scol[STAGE_CHUNK];
    const int tile = blockIdx.x;
    const int W = v.W, H = v.H, T = v.T;
    const size_t TT = (size_t)T;
    const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = tx * TILE + (warp & 1) * 8 + (lane & 7);
    const int py0 = ty * TILE + (warp >> 1) * 8 + (lane >> 3);

    const Cone tc = v.tiles[tile];
    const float ax = tc.c0.x, ay = tc.c0.y, az = tc.c0.z;

    float gx[PPT], gy[PPT], gz[PPT], dgx[PPT], dgy[PPT], dgz[PPT], delta[PPT], h[PPT], eg[PPT];
    bool pv[PPT], inimg[PPT];
    uint32_t cnt[PPT], room[PPT];
    size_t fbase[PPT];
    unsigned long long key[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int py = py0 + 4 * p;
        inimg[p] = px < W && py < H;
        const size_t o = (size_t)py * W + px;
        float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (inimg[p]) g = v.map[o];
        pv[p] = g.w > 0.0f;
        gx[p] = g.x;
        gy[p] = g.y;
        gz[p] = g.z;
        delta[p] = g.w;
        h[p] = pv[p] ? 0.5f / g.w : 0.0f;
        eg[p] = pv[p] ? norm2_minus_one(g.x, g.y, g.z) : 0.0f;
        dgx[p] = g.x - ax;
        dgy[p] = g.y - ay;
        dgz[p] = g.z - az;
        cnt[p] = 0u;
        key[p] = ~0ull;
        fbase[p] = 0;
        room[p] = 0u;
        if (FILL && inimg[p]) {
            fbase[p] = v.foff[o];
            room[p] = v.foff[o + 1] - v.foff[o];
        }
    }

    // the warp's own view cone (its 8x8 pixels), as in the coverage kernel
    float sx = 0.0f, sy = 0.0f, sz = 0.0f, cn = 0.0f, hw = 0.0f;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
        if (pv[p]) {
            sx += gx[p];
            sy += gy[p];
            sz += gz[p];
            cn += 1.0f;
            hw = fmaxf(hw, h[p]);
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
    // the thread's two pixels side by side for the packed FP32x2 distances
    // (bit for bit the scalar ones, so the classification is the coverage
    // kernel's)
    static_assert(PPT == 2, "packed pairs hold the thread's two pixels");
    const float2 dgx2 = make_float2(dgx[0], dgx[1]), dgy2 = make_float2(dgy[0], dgy[1]),
                 dgz2 = make_float2(dgz[0], dgz[1]), eg2 = make_float2(eg[0], eg[1]);

    for (uint32_t base = b0; base < b1; base += STAGE_CHUNK) {
        const int n = (int)min((uint32_t)STAGE_CHUNK, b1 - base);
        __syncthreads();
        if ((int)threadIdx.x < n) {
            const uint32_t t = v.ids[base + threadIdx.x];
            if (t >= (uint32_t)T) {
                raise_status(status, VSR_ERR_BIN_OVERFLOW);
                st.s6[threadIdx.x] = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(STAGE_EMPTY));
            } else {
                stage_triangle(v.rec, TT, t, ax, ay, az, st, threadIdx.x);
                scol[threadIdx.x] = v.colors ? v.colors[t] : 1.0f;
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
                keep = cap_hits_cone(make_float3(a.x, a.y, a.z), 1.0f - 0.5f * b.y, b.x, make_float3(wax, way, waz),
                                     wcos, wsin, wh);
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
                const float4 a = st.s0[j];
                const float4 b = st.s1[j];
                const float4 e = st.s6[j];
                const float2 g4p = miter_distance2(dgx2, dgy2, dgz2, e, b, eg2);
                const float g4[PPT] = {g4p.x, g4p.y};
                bool p4[PPT], any4 = false;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    p4[p] = pv[p] && g4[p] > -h[p];
                    any4 |= p4[p];
                }
                if (!__any_sync(0xffffffffu, any4)) continue;
                const float2 g1p = plane_distance2(dgx2, dgy2, dgz2, st.s2[j]);
                const float2 g2p = plane_distance2(dgx2, dgy2, dgz2, st.s3[j]);
                const float2 g3p = plane_distance2(dgx2, dgy2, dgz2, st.s4[j]);
                const float g1[PPT] = {g1p.x, g1p.y}, g2[PPT] = {g2p.x, g2p.y}, g3[PPT] = {g3p.x, g3p.y};
                float g3m[PPT], gm[PPT];
                bool frag[PPT], anyf = false;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    g3m[p] = fminf(fminf(g1[p], g2[p]), g3[p]);
                    gm[p] = fminf(g3m[p], g4[p]);
                    frag[p] = p4[p] && gm[p] > -h[p];
                    anyf |= frag[p];
                }
                if (!__any_sync(0xffffffffu, anyf)) continue;
                const float2 Dp = plane_distance2(dgx2, dgy2, dgz2, st.s5[j]);
                const float D2[PPT] = {Dp.x, Dp.y};
                const unsigned ties = __float_as_uint(a.w);
                const uint32_t t = __float_as_uint(e.w);
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const float D = D2[p];
                    const float r = __fdividef(b.w, D);
                    const bool f = frag[p] && __float_as_uint(r) - 1u < 0x7f7fffffu;  // 0 < r < inf
                    if (!f) continue;
                    if (FILL) {
                        const float m = __saturatef(fmaf(gm[p], delta[p], 0.5f));
                        if (cnt[p] < room[p])
                            v.frags[fbase[p] + cnt[p]] =
                                make_float4(r, __uint_as_float(t), m, scol[j] * fabsf(D));
                        const unsigned long long k = ((unsigned long long)__float_as_uint(r) << 32) | t;
                        if (centre_inside(g1[p], g2[p], g3[p], g3m[p], ties) && k < key[p]) key[p] = k;
                    }
                    ++cnt[p];
                }
            }
        }
    }

#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (!inimg[p]) continue;
        const size_t o = (size_t)(py0 + 4 * p) * W + px;
        if (!FILL) {
            v.counts[o] = cnt[p];
            continue;
        }
        if (cnt[p] != room[p]) raise_status(status, VSR_ERR_FRAG_OVERFLOW);  // counts of another frame
        const uint32_t n = min(cnt[p], room[p]);
        float4* F = v.frags + fbase[p];
        // insertion sort by (r, t): lists are a few fragments long
        for (uint32_t q = 1; q < n; ++q) {
            const float4 x = F[q];
            uint32_t u = q;
            while (u > 0 && frag_less(x, F[u - 1])) {
                F[u] = F[u - 1];
                --u;
            }
            F[u] = x;
        }
        float mb = 0.0f, img = 0.0f;
        for (uint32_t q = 0; q < n && mb < 1.0f; ++q) {
            const float4 x = F[q];
            const float mfc = fminf(x.z, 1.0f - mb);
            img = fmaf(mfc, x.w, img);
            mb += mfc;
        }
        const bool hit = key[p] != ~0ull;
        if (v.image) v.image[o] = img;
        if (v.cov) v.cov[o] = mb;
        if (v.out_id) v.out_id[o] = hit ? (uint32_t)(key[p] & 0xffffffffull) : 0xffffffffu;
        if (v.out_depth) v.out_depth[o] = hit ? __uint_as_float((uint32_t)(key[p] >> 32)) : INFINITY;
    }
}

// ---------------------------------------------------------------------------
// Backward, per pixel.

struct BackView {
    const float4* map;
    int W, H;
    const float4* rec;
    int T;
    const float* colors;
    const uint32_t* foff;
    const float4* frags;
    const uint32_t* id;
    const float* dimage;
    const float* dcov;
    const float* ddepth;
    float4* grad;  // GF_COUNT x T, field-major
    float4* dmap;  // per pixel (dG, d delta)
};

__device__ __forceinline__ float dot3f(float ax, float ay, float az, const float4& b)
{
    return fmaf(ax, b.x, fmaf(ay, b.y, az * b.z));
}

__global__ void __launch_bounds__(TILE_PIX) frag_backward_kernel(BackView v)
{
    const int i = blockIdx.x * TILE + (threadIdx.x % TILE);
    const int j = blockIdx.y * TILE + (threadIdx.x / TILE);
    if (i >= v.W || j >= v.H) return;
    const size_t o = (size_t)j * v.W + i;
    const float4 g = v.map[o];
    float4 dG = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (!(g.w > 0.0f)) {
        v.dmap[o] = dG;
        return;
    }
    const size_t TT = (size_t)v.T;
    const float dI = v.dimage ? v.dimage[o] : 0.0f;
    const float dC = v.dcov ? v.dcov[o] : 0.0f;
    const float dD = v.ddepth ? v.ddepth[o] : 0.0f;
    const uint32_t b0 = v.foff[o], n = v.foff[o + 1] - b0;
    const float4* __restrict__ F = v.frags + b0;

    // the saturating fragment, replaying the forward merge's arithmetic
    uint32_t fstar = n;
    float sstar = 0.0f, mb = 0.0f;
    for (uint32_t q = 0; q < n; ++q) {
        const float4 x = F[q];
        if (x.z > 1.0f - mb) {
            fstar = q;
            sstar = x.w;
            break;
        }
        mb += x.z;
    }
    const float beta = fstar < n ? -dI * sstar : dC;
    const uint32_t last = fstar < n ? fstar + 1 : n;
    mb = 0.0f;
    for (uint32_t q = 0; q < last; ++q) {
        const float4 x = F[q];
        const uint32_t t = __float_as_uint(x.y);
        float dm, dsh;
        if (q == fstar) {
            dm = 0.0f;
            dsh = dI * (1.0f - mb);
        } else {
            dm = fmaf(dI, x.w, beta);
            dsh = dI * x.z;
            mb += x.z;
        }
        if (dm != 0.0f && x.z > 0.0f && x.z < 1.0f) {
            // the minimising distance (any one of equal minima is a valid
            // subgradient); the forward's g_min from its own m^f
            const float4 n1 = v.rec[RF_N1 * TT + t], n2 = v.rec[RF_N2 * TT + t], n3 = v.rec[RF_N3 * TT + t];
            const float4 cp = v.rec[RF_CAP * TT + t], cp2 = v.rec[RF_CAP2 * TT + t];
            const float g1 = dot3f(g.x, g.y, g.z, n1), g2 = dot3f(g.x, g.y, g.z, n2), g3 = dot3f(g.x, g.y, g.z, n3);
            const float mx = g.x - cp.x, my = g.y - cp.y, mz = g.z - cp.z;
            const float g4 = (cp2.y - fmaf(mx, mx, fmaf(my, my, mz * mz))) * cp2.z;
            int is = 0;
            float gmin = g1;
            if (g2 < gmin) { gmin = g2; is = 1; }
            if (g3 < gmin) { gmin = g3; is = 2; }
            if (g4 < gmin) { gmin = g4; is = 3; }
            const float gm = (x.z - 0.5f) / g.w;
            const float dg = dm * g.w;
            dG.w = fmaf(dm, gm, dG.w);
            if (is < 3) {
                const float4 nn = is == 0 ? n1 : (is == 1 ? n2 : n3);
                atomicAdd(&v.grad[(GF_N1 + is) * TT + t], make_float4(dg * g.x, dg * g.y, dg * g.z, 0.0f));
                dG.x = fmaf(dg, nn.x, dG.x);
                dG.y = fmaf(dg, nn.y, dG.y);
                dG.z = fmaf(dg, nn.z, dG.z);
            } else {
                const float sr = cp2.x, c = cp.w;
                const float q4 = dg / sr;
                atomicAdd(&v.grad[GF_CAP * TT + t],
                          make_float4(q4 * g.x, q4 * g.y, q4 * g.z, q4 * fmaf(g4 / sr, c, -1.0f)));
                dG.x = fmaf(q4, cp.x, dG.x);
                dG.y = fmaf(q4, cp.y, dG.y);
                dG.z = fmaf(q4, cp.z, dG.z);
            }
        }
        if (dsh != 0.0f) {
            const float4 pl = v.rec[RF_PL * TT + t];
            const float u = dot3f(g.x, g.y, g.z, pl);
            const float col = v.colors ? v.colors[t] : 1.0f;
            const float du = u > 0.0f ? dsh * col : (u < 0.0f ? -dsh * col : 0.0f);
            atomicAdd(&v.grad[GF_PL * TT + t], make_float4(du * g.x, du * g.y, du * g.z, dsh * fabsf(u)));
            dG.x = fmaf(du, pl.x, dG.x);
            dG.y = fmaf(du, pl.y, dG.y);
            dG.z = fmaf(du, pl.z, dG.z);
        }
    }
    if (dD != 0.0f && v.id) {
        const uint32_t t = v.id[o];
        if (t < (uint32_t)v.T) {
            const float4 pl = v.rec[RF_PL * TT + t];
            const float u = dot3f(g.x, g.y, g.z, pl);
            const float r = pl.w / u;
            const float dGN = -dD * r / u;
            atomicAdd(&v.grad[GF_PL * TT + t], make_float4(dGN * g.x, dGN * g.y, dGN * g.z, 0.0f));
            atomicAdd(&v.grad[GF_D * TT + t].x, dD / u);
            dG.x = fmaf(dGN, pl.x, dG.x);
            dG.y = fmaf(dGN, pl.y, dG.y);
            dG.z = fmaf(dGN, pl.z, dG.z);
        }
    }
    v.dmap[o] = dG;
}

// ---------------------------------------------------------------------------
// Set-up adjoint, per triangle: record gradients -> world vertices.
//   n_e = sigma x/|x|, x = P' x Q'  =>  dx = sigma (dn - x^ (x^.dn))/|x|,
//                                       dP' += Q' x dx, dQ' += dx x P'
//   S-hat = S/|S|, c = |S|          =>  dS = (dS^ - S^ (S^.dS^))/|S| + S^ dc
//   S = midpoint or (Os A^ + Ot B^ + Op C^)/(Os + Ot + Op) of the unit
//   vertices U = V/|V| (Sec. 1.1.2), differentiated through the squared
//   chords a^2, b^2, c^2
//   N-hat = N/|N|, N = (A' - B') x (C' - B'), d' = A'.N-hat
//   X' = M (X - O)                  =>  dX = M^T dX'
// Plain FP32 throughout: the forward quantities are recomputed from the
// world vertices, sigma is read off the stored normal.

struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(F3 a, F3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ F3 cross(F3 a, F3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ F3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
// gradient of u = x/|x| pulled back to x
__device__ __forceinline__ F3 unit_back(F3 u, float len, F3 du) { return (1.0f / len) * (du - dot(u, du) * u); }

struct CamF {
    float O[3];
    float M[9];
};

__global__ void __launch_bounds__(128) setup_backward_kernel(const float* __restrict__ tris, int T, CamF cam,
                                                              const float4* __restrict__ rec,
                                                              const float4* __restrict__ grad,
                                                              float* __restrict__ dtris, float* __restrict__ dcolors)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const size_t TT = (size_t)T;
    const float4 cp2 = rec[RF_CAP2 * TT + t];
    float* out = dtris ? dtris + (size_t)t * 9 : nullptr;
    const float4 gpl = grad[GF_PL * TT + t];
    if (dcolors) dcolors[t] = cp2.w != 0.0f ? gpl.w : 0.0f;
    if (!out) return;
    if (cp2.w == 0.0f) {  // culled at set-up: no fragments, no gradient
#pragma unroll
        for (int q = 0; q < 9; ++q) out[q] = 0.0f;
        return;
    }
    F3 V[3], dV[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float d0 = tris[(size_t)t * 9 + 3 * q] - cam.O[0];
        const float d1 = tris[(size_t)t * 9 + 3 * q + 1] - cam.O[1];
        const float d2 = tris[(size_t)t * 9 + 3 * q + 2] - cam.O[2];
        V[q] = f3(fmaf(cam.M[0], d0, fmaf(cam.M[1], d1, cam.M[2] * d2)),
                  fmaf(cam.M[3], d0, fmaf(cam.M[4], d1, cam.M[5] * d2)),
                  fmaf(cam.M[6], d0, fmaf(cam.M[7], d1, cam.M[8] * d2)));
        dV[q] = f3(0.0f, 0.0f, 0.0f);
    }
    // edge normals
    const float4 n1s = rec[RF_N1 * TT + t];
    const F3 x0 = cross(V[0], V[1]);
    const float sigma = dot(xyz(n1s), x0) < 0.0f ? -1.0f : 1.0f;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int P = e, Q = e == 2 ? 0 : e + 1;
        const F3 x = cross(V[P], V[Q]);
        const float len = sqrtf(dot(x, x));
        const F3 dn = xyz(grad[(GF_N1 + e) * TT + t]);
        const F3 dx = sigma * unit_back((1.0f / len) * x, len, dn);
        dV[P] = dV[P] + cross(V[Q], dx);
        dV[Q] = dV[Q] + cross(dx, V[P]);
    }
    // miter
    const float4 gcap = grad[GF_CAP * TT + t];
    if (gcap.x != 0.0f || gcap.y != 0.0f || gcap.z != 0.0f || gcap.w != 0.0f) {
        F3 U[3];
        float Ul[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Ul[q] = sqrtf(dot(V[q], V[q]));
            U[q] = (1.0f / Ul[q]) * V[q];
        }
        const F3 ea = U[1] - U[2], eb = U[2] - U[0], ec = U[0] - U[1];
        const float a2 = dot(ea, ea), b2 = dot(eb, eb), c2 = dot(ec, ec);
        const float Os = a2 * (b2 + c2 - a2), Ot = b2 * (c2 + a2 - b2), Op = c2 * (a2 + b2 - c2);
        F3 S;
        const bool mid = Os <= 0.0f || Ot <= 0.0f || Op <= 0.0f;
        const int ma = Os <= 0.0f ? 1 : (Ot <= 0.0f ? 2 : 0);
        const int mbi = Os <= 0.0f ? 2 : (Ot <= 0.0f ? 0 : 1);
        const float sum = Os + Ot + Op;
        if (mid)
            S = 0.5f * (U[ma] + U[mbi]);
        else
            S = (1.0f / sum) * (Os * U[0] + Ot * U[1] + Op * U[2]);
        const float slen = sqrtf(dot(S, S));
        const F3 Sh = (1.0f / slen) * S;
        const F3 dS = unit_back(Sh, slen, xyz(gcap)) + gcap.w * Sh;
        F3 dU[3] = {f3(0.0f, 0.0f, 0.0f), f3(0.0f, 0.0f, 0.0f), f3(0.0f, 0.0f, 0.0f)};
        if (mid) {
            dU[ma] = 0.5f * dS;
            dU[mbi] = 0.5f * dS;
        } else {
            const float Oq[3] = {Os, Ot, Op};
            float dO[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dO[q] = dot(dS, U[q] - S) / sum;
                dU[q] = (Oq[q] / sum) * dS;
            }
            const float da2 = dO[0] * (b2 + c2 - 2.0f * a2) + dO[1] * b2 + dO[2] * c2;
            const float db2 = dO[0] * a2 + dO[1] * (c2 + a2 - 2.0f * b2) + dO[2] * c2;
            const float dc2 = dO[0] * a2 + dO[1] * b2 + dO[2] * (a2 + b2 - 2.0f * c2);
            dU[1] = dU[1] + (2.0f * da2) * ea;
            dU[2] = dU[2] - (2.0f * da2) * ea;
            dU[2] = dU[2] + (2.0f * db2) * eb;
            dU[0] = dU[0] - (2.0f * db2) * eb;
            dU[0] = dU[0] + (2.0f * dc2) * ec;
            dU[1] = dU[1] - (2.0f * dc2) * ec;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) dV[q] = dV[q] + unit_back(U[q], Ul[q], dU[q]);
    }
    // plane: shade uses N-hat, depth r = d'/(G.N-hat) with d' = A'.N-hat
    const float dd = grad[GF_D * TT + t].x;
    const F3 e1 = V[0] - V[1], e2 = V[2] - V[1];
    const F3 N = cross(e1, e2);
    const float nl = sqrtf(dot(N, N));
    const F3 Nh = (1.0f / nl) * N;
    const F3 dNh = xyz(gpl) + dd * V[0];
    dV[0] = dV[0] + dd * Nh;
    const F3 dN = unit_back(Nh, nl, dNh);
    const F3 de1 = cross(e2, dN), de2 = cross(dN, e1);
    dV[0] = dV[0] + de1;
    dV[2] = dV[2] + de2;
    dV[1] = dV[1] - (de1 + de2);
    // world: dX = M^T dX'
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        out[3 * q + 0] = fmaf(cam.M[0], dV[q].x, fmaf(cam.M[3], dV[q].y, cam.M[6] * dV[q].z));
        out[3 * q + 1] = fmaf(cam.M[1], dV[q].x, fmaf(cam.M[4], dV[q].y, cam.M[7] * dV[q].z));
        out[3 * q + 2] = fmaf(cam.M[2], dV[q].x, fmaf(cam.M[5], dV[q].y, cam.M[8] * dV[q].z));
    }
}

}  // namespace

vsr_status launch_frag_count(const FragArgs& a, cudaStream_t st)
{
    const int tx = (a.W + TILE - 1) / TILE, ty = (a.H + TILE - 1) / TILE;
    FragView v{a.map, a.W, a.H, a.tiles, tx, a.rec, a.T, a.offsets, a.ids, a.cap, a.colors, a.counts,
               nullptr, nullptr, 0u, nullptr, nullptr, nullptr, nullptr, a.ends};
    frag_kernel<false><<<tx * ty, FT, 0, st>>>(v, a.status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_frag_fill(const FragArgs& a, cudaStream_t st)
{
    const int tx = (a.W + TILE - 1) / TILE, ty = (a.H + TILE - 1) / TILE;
    FragView v{a.map,    a.W,   a.H,     a.tiles, tx,    a.rec,   a.T,      a.offsets, a.ids, a.cap,
               a.colors, nullptr, a.foff, a.frags, a.fcap, a.image, a.cov, a.out_id, a.out_depth, a.ends};
    frag_kernel<true><<<tx * ty, FT, 0, st>>>(v, a.status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_frag_backward(const FragArgs& a, const uint32_t* id, const float* dimage, const float* dcov,
                                const float* ddepth, float4* grad, float4* dmap, cudaStream_t st)
{
    BackView v{a.map, a.W, a.H, a.rec, a.T, a.colors, a.foff, a.frags, id, dimage, dcov, ddepth, grad, dmap};
    dim3 grid((a.W + TILE - 1) / TILE, (a.H + TILE - 1) / TILE);
    frag_backward_kernel<<<grid, TILE_PIX, 0, st>>>(v);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_setup_backward(const float* tris, int T, const float cam[12], const float4* rec, const float4* grad,
                                 float* dtris, float* dcolors, cudaStream_t st)
{
    if (T == 0) return VSR_OK;
    CamF c;
    for (int q = 0; q < 3; ++q) c.O[q] = cam[q];
    for (int q = 0; q < 9; ++q) c.M[q] = cam[3 + q];
    setup_backward_kernel<<<(T + 127) / 128, 128, 0, st>>>(tris, T, c, rec, grad, dtris, dcolors);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}
