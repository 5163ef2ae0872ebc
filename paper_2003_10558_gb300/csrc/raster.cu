// raster.cu -- per-tile coverage / depth / visibility kernel.
//
// One CTA of 128 threads per 16x16 tile; warp w covers the 8x8 pixel block
// (w & 1, w >> 1) of the tile and each lane two pixels of it, (x, y) and
// (x, y + 4), so every shared-memory load, vote and branch per triangle
// serves two pixels.  For every pixel G (unit direction, global delta) and
// every triangle t of the tile's bin the kernel evaluates the four plane
// distances of the rasterization equation (Sec. 1.1.2):
//   g_1..3 = G.n_i                   edge planes through the eye (Sec. 1.1)
//   g_4    = (G.S-hat - cos rho)/sin rho   miter cap, in the same angular
//            units as the edge distances, computed in the chord form
//            (4 sin^2(rho/2) - |G - S-hat|^2 + |G|^2 - 1) / (2 sin rho),
//            which keeps its accuracy for caps far below a pixel
// then   fragment   iff min g_i > -1/(2 delta) and r > 0   (gbpxstep)
//        m^f        = clamp(delta min g_i + 1/2, 0, 1)       (gpstep)
//        r          = (A'.N-hat)/(G.N-hat)                    (Sec. 1.1.4)
//        centre-inside iff g_1..3 >= 0 (tie rule via the normal's sign)
// and merges front to back (Sec. 1.4).  The merge
//   m^fc = min(m^f, 1 - m^b),  m^b = m^b + m^fc
// equals m^b = min(1, sum m^f) by induction, independent of the order, so
// each pixel keeps a saturating 2^-22 fixed-point sum and the 64-bit key
// (bits(r) << 32 | t) of its nearest centre-inside triangle.
//
// Accuracy in FP32: every distance is re-centred on the tile's cone axis a,
//   G.n = a.n + (G - a).n,
// with a.n formed once per (tile, triangle) from the FP32-pair normals in a
// compensated dot product.  The per-pixel part is a plain 3-term FMA chain
// on |G - a| <= the tile's angular radius, so its rounding error in units of
// the ramp is ~(tile size in pixels) x 2^-23, a few 1e-6 of coverage.
//
// Work culling (the paper's low-resolution region mask, Sec. 1.1.3, at the
// granularity of a warp's 8x8 pixels): the triangles of a staged chunk are
// first tested lane-parallel (lane j <-> triangle j) against each warp's
// view cone, cap and edge planes alike; the survivors are then evaluated for
// all 64 pixels, one triangle per step for the whole warp.  A culled pair is
// never a fragment, and both the coverage sum and the visibility key are
// order-free, so the result does not depend on the cull.
#include <type_traits>

#include "stage.cuh"

namespace {

constexpr int RT = 128;          // threads per CTA (one 16x16 tile)
constexpr int PPT = 2;           // pixels per thread: (x, y) and (x, y + 4) of the warp's 8x8 block
constexpr int CHUNK = RT;        // triangles staged per pass
static_assert(CHUNK == STAGE_CHUNK, "one staging slot per thread");
static_assert(RT * PPT == TILE_PIX, "one CTA covers one tile");
// resident CTAs per SM the timed kernel is compiled for (its register cap)
#ifndef VSR_RASTER_CTAS_PER_SM
#define VSR_RASTER_CTAS_PER_SM 8
#endif

// One 16x16 tile of one view.  Called by every thread of a CTA of RT
// threads; `st` is the CTA's staging area (reusable across calls: every use
// is fenced by the barriers of the chunk loop).
// Split tiles: a tile whose bin is longer than split_max triangles (a
// multiple of CHUNK) is processed as several work items of at most
// split_max triangles each.  The
// items of one tile add their coverage (2^-22 fixed point) and take the
// minimum of their visibility keys in the tile's accumulator slot with
// atomics -- both are order-free, so the result is exactly that of one item
// -- and the item that arrives last (atomic counter, nothing waits) writes
// the outputs and clears the slot for the next frame.
struct SplitAcc {
    unsigned long long* acc;  // [slot][TILE_PIX], zero between frames (64 bits: many partials)
    unsigned long long* key;  // [slot][TILE_PIX], ~0 between frames
    uint32_t* done;           // [slot], zero between frames
};

// A cone (axis, cos, sin, widest ramp half-width) may hold a fragment of the
// staged triangle (cap a, b; edge normals n1..n3): the cap test, and unless
// counting algorithmic tests (defined by the cap alone) the edge planes.
// Every pixel G of the cone is within alpha of the axis c, so
// G.n <= c.n + sin(alpha) + (1 - cos(alpha)) for a unit normal n; a triangle
// with some edge plane below -h there has no fragment.
__device__ __forceinline__ bool cone_may_hit(const float4& a, const float4& b, const float4& n1, const float4& n2,
                                             const float4& n3, const float4& c0, const float4& c1, bool count_alg)
{
    bool keep = cap_hits_cone(make_float3(a.x, a.y, a.z), 1.0f - 0.5f * b.y, b.x, make_float3(c0.x, c0.y, c0.z),
                              c0.w, c1.x, c1.y);
    const float lim = -(c1.y + c1.x + (1.0f - c0.w) + 1e-6f);
    return keep && (count_alg || (fmaf(c0.x, n1.x, fmaf(c0.y, n1.y, c0.z * n1.z)) > lim &&
                                  fmaf(c0.x, n2.x, fmaf(c0.y, n2.y, c0.z * n2.z)) > lim &&
                                  fmaf(c0.x, n3.x, fmaf(c0.y, n3.y, c0.z * n3.z)) > lim));
}

// View cone of a group of WIDTH lanes (xor-shuffle width; 32: the warp's
// block) from the lanes' valid pixels: axis = normalised sum, cos alpha = min G.axis less a margin, h =
// the widest ramp half-width; a group without a valid pixel gets valid = 0,
// a degenerate sum the whole sphere.
template <int WIDTH>
__device__ __forceinline__ void group_cone(const float* gx, const float* gy, const float* gz, const float* h,
                                           const bool* pv, float4& c0, float4& c1)
{
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
#pragma unroll
    for (int o = 1; o < WIDTH; o <<= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        cn += __shfl_xor_sync(0xffffffffu, cn, o);
        hw = fmaxf(hw, __shfl_xor_sync(0xffffffffu, hw, o));
    }
    const float len = sqrtf(sx * sx + sy * sy + sz * sz);
    const bool deg = !(len > 1e-6f * fmaxf(cn, 1.0f));
    const float ax = deg ? 0.0f : sx / len, ay = deg ? 0.0f : sy / len, az = deg ? 1.0f : sz / len;
    float cm = 2.0f;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
        if (pv[p]) cm = fminf(cm, gx[p] * ax + gy[p] * ay + gz[p] * az);
#pragma unroll
    for (int o = 1; o < WIDTH; o <<= 1) cm = fminf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    float cs = fmaxf(-1.0f, fminf(1.0f, cm - 2e-6f));
    if (deg) cs = -1.0f;
    c0 = make_float4(ax, ay, az, cs);
    c1 = make_float4(sqrtf(fmaxf(0.0f, 1.0f - cs * cs)), hw, cn > 0.0f ? 1.0f : 0.0f, 0.0f);
}

// One lane's two pixels as the evaluation sees them.
struct PixPair {
    float2 dgx, dgy, dgz;  // G - a (tile axis) of both pixels
    float2 eg;             // |G|^2 - 1
    float delta[PPT];      // global delta (0: invalid pixel)
    float lim[PPT];        // fragment iff min distance > lim (-1/(2 delta); +inf if invalid)
    uint32_t acc[PPT];     // coverage, 2^-22 fixed point
    unsigned long long key[PPT];  // (bits(r) << 32) | t of the nearest centre-inside fragment
    int32_t cnt_in[PPT];   // centre-inside fragments (statistics)
};

// Evaluate staged slot j at the lane's two pixels and merge the fragments into the pixels' coverage and keys.
// Called by all 32 lanes of a warp together (warp votes).
template <bool STATS>
__device__ __forceinline__ void eval_slot(const Stage& st, int j, PixPair& q, uint32_t& cnt_alg)
{
    // the four distances of both pixels in packed FP32x2 arithmetic; the miter
    // in chord form, G - S-hat = (G - a) - (S-hat - a): both differences are at
    // most the tile radius, so their rounding costs ~1e-9 rad where it matters
    const float4 b = st.s1[j];
    const float4 e = st.s6[j];
    const float2 g4p = miter_distance2(q.dgx, q.dgy, q.dgz, e, b, q.eg);
    const float2 g1p = plane_distance2(q.dgx, q.dgy, q.dgz, st.s2[j]);
    const float2 g2p = plane_distance2(q.dgx, q.dgy, q.dgz, st.s3[j]);
    const float2 g3p = plane_distance2(q.dgx, q.dgy, q.dgz, st.s4[j]);
    const float g4[PPT] = {g4p.x, g4p.y};
    float g3m[PPT] = {fminf(fminf(g1p.x, g2p.x), g3p.x), fminf(fminf(g1p.y, g2p.y), g3p.y)};
    float gm[PPT];
    bool frag[PPT], anyf = false;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (STATS) cnt_alg += g4[p] > q.lim[p];
        gm[p] = fminf(g3m[p], g4[p]);
        frag[p] = gm[p] > q.lim[p];  // gbpxstep on all four distances; never on invalid pixels
        anyf |= frag[p];
    }
    if (!__any_sync(0xffffffffu, anyf)) return;
    const float2 Dp = plane_distance2(q.dgx, q.dgy, q.dgz, st.s5[j]);
    const float D2[PPT] = {Dp.x, Dp.y};
    const float dgx[PPT] = {q.dgx.x, q.dgx.y}, dgy[PPT] = {q.dgy.x, q.dgy.y}, dgz[PPT] = {q.dgz.x, q.dgz.y};
    const unsigned long long tbits = (unsigned long long)__float_as_uint(e.w);
    // The exact-zero tie rule needs its branch only where some pixel of
    // the warp has a fragment on an edge plane (rare): decide once for
    // the warp, and run a copy of the loop without the branch otherwise.
    auto post = [&](auto tie_t) {
        constexpr bool TIE = decltype(tie_t)::value;
        float rr[PPT];
        bool inn[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            // predicated: every lane computes, non-fragments add nothing
            const float r = __fdividef(b.w, D2[p]);
            // 0 < r < inf (NaN excluded) as one unsigned compare of the bits
            const bool f = frag[p] && __float_as_uint(r) - 1u < 0x7f7fffffu;
            const float m = __saturatef(fmaf(gm[p], q.delta[p], 0.5f));
            q.acc[p] += f ? cov_fixed(m) : 0u;
            // centre-inside: all three edge distances >= 0; an exact zero
            // takes the tie rule on the three distances, recomputed from
            // the staged planes (the scalar form gives the packed values
            // bit for bit), so they need not stay live in registers here
            bool in = f && g3m[p] > 0.0f;
            if (TIE && f && g3m[p] == 0.0f)
                in = centre_inside(plane_distance(dgx[p], dgy[p], dgz[p], st.s2[j]),
                                   plane_distance(dgx[p], dgy[p], dgz[p], st.s3[j]),
                                   plane_distance(dgx[p], dgy[p], dgz[p], st.s4[j]), g3m[p],
                                   __float_as_uint(st.s0[j].w));
            rr[p] = r;
            inn[p] = in;
            if (STATS) q.cnt_in[p] += in;
        }
        // the visibility keys only where some lane of the warp has a
        // centre-inside fragment
        if (__any_sync(0xffffffffu, inn[0] || inn[1])) {
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const unsigned long long k = ((unsigned long long)__float_as_uint(rr[p]) << 32) | tbits;
                q.key[p] = inn[p] && k < q.key[p] ? k : q.key[p];
            }
        }
    };
    bool z = false;
#pragma unroll
    for (int p = 0; p < PPT; ++p) z |= frag[p] && g3m[p] == 0.0f;
    if (__any_sync(0xffffffffu, z))
        post(std::true_type{});
    else
        post(std::false_type{});
}

// ROWS: the outputs go through shared memory and leave in whole tile rows
// (pinned host outputs written in place over the host link).
template <bool STATS, bool ROWS = false>
__device__ __forceinline__ void raster_tile(const RasterView& view, int tile, Stage& st, bool count_alg,
                                            uint32_t& cnt_alg, uint32_t& cnt_exec, int32_t* __restrict__ n_inside,
                                            int* __restrict__ status, int range_lo = 0, int range_hi = -1,
                                            int split_slot = -1, int nsplit = 1, SplitAcc split = SplitAcc{})
{
    const float4* __restrict__ map = view.map;
    const int W = view.W, H = view.H, tiles_x = view.tiles_x, T = view.T;
    const Cone* __restrict__ tiles = view.tiles;
    const float4* __restrict__ rec = view.rec;
    const uint32_t* __restrict__ offsets = view.offsets;
    const uint32_t* __restrict__ ids = view.ids;
    const uint32_t cap = view.cap;
    uint32_t* __restrict__ out_id = view.out_id;
    float* __restrict__ out_depth = view.out_depth;
    float* __restrict__ out_cov = view.out_cov;

    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // pixel (in tile) of this lane's first pixel; its second is four rows below
    const int lx = (warp & 1) * 8 + (lane & 7);
    const int ly0 = (warp >> 1) * 8 + (lane >> 3);
    const int px = tx * TILE + lx;
    const int py0 = ty * TILE + ly0;

    const Cone tc = tiles[tile];
    const float ax = tc.c0.x, ay = tc.c0.y, az = tc.c0.z;

    float gx[PPT], gy[PPT], gz[PPT], h[PPT];
    bool pv[PPT], inimg[PPT];
    PixPair q;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int py = py0 + 4 * p;
        inimg[p] = px < W && py < H;
        float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (inimg[p]) g = map[(size_t)py * W + px];
        pv[p] = g.w > 0.0f;
        gx[p] = g.x;
        gy[p] = g.y;
        gz[p] = g.z;
        h[p] = pv[p] ? 0.5f / g.w : 0.0f;
        q.delta[p] = g.w;
        q.lim[p] = pv[p] ? -h[p] : INFINITY;
        q.acc[p] = 0u;
        q.key[p] = ~0ull;
        q.cnt_in[p] = 0;
    }
    q.dgx = make_float2(gx[0] - ax, gx[1] - ax);
    q.dgy = make_float2(gy[0] - ay, gy[1] - ay);
    q.dgz = make_float2(gz[0] - az, gz[1] - az);
    q.eg = make_float2(pv[0] ? norm2_minus_one(gx[0], gy[0], gz[0]) : 0.0f,
                       pv[1] ? norm2_minus_one(gx[1], gy[1], gz[1]) : 0.0f);

    // the warp's own view cone (its 8x8 pixels)
    float4 wc0, wc1;
    group_cone<32>(gx, gy, gz, h, pv, wc0, wc1);
    const bool warp_active = wc1.z > 0.0f;

    uint32_t b0 = 0, b1 = 0;
    if (tc.c1.z > 0.0f) {
        b0 = offsets[tile];
        b1 = view.ends ? view.ends[tile] : offsets[tile + 1];
        if (b1 > cap) {
            if (threadIdx.x == 0) raise_status(status, VSR_ERR_BIN_OVERFLOW);
            b1 = cap;
            b0 = min(b0, cap);
        }
        if (range_hi >= 0) {  // one item of a split tile
            const uint32_t lo = b0 + (uint32_t)range_lo, hi = b0 + (uint32_t)range_hi;
            b0 = min(lo, b1);
            b1 = min(hi, b1);
        }
    }

    const size_t TT = (size_t)T;
    static_assert(PPT == 2, "packed pairs hold the thread's two pixels");

    for (uint32_t base = b0; base < b1; base += CHUNK) {
        const int n = (int)min((uint32_t)CHUNK, b1 - base);
        // saturate once per chunk: at most CHUNK terms of <= COV_ONE each were added since
#pragma unroll
        for (int p = 0; p < PPT; ++p) q.acc[p] = min(q.acc[p], COV_ONE);
        __syncthreads();
        if ((int)threadIdx.x < n) {
            const uint32_t t = ids[base + threadIdx.x];
            if (t >= (uint32_t)T) {
                // never produced by a completed binning: a stale or overflowed
                // bin must not index outside the records
                raise_status(status, VSR_ERR_BIN_OVERFLOW);
                st.s6[threadIdx.x] = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(STAGE_EMPTY));
            } else {
                stage_triangle(rec, TT, t, ax, ay, az, st, threadIdx.x);
            }
        }
        __syncthreads();
        if (!warp_active) continue;
        for (int gbase = 0; gbase < n; gbase += 32) {
            // lane-parallel cull of 32 triangles against this warp's cone
            bool keep = false;
            const int jj = gbase + lane;
            if (jj < n && __float_as_uint(st.s6[jj].w) != STAGE_EMPTY)
                keep = cone_may_hit(st.s0[jj], st.s1[jj], st.s2[jj], st.s3[jj], st.s4[jj], wc0, wc1, count_alg);
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            while (mask) {
                const int j = gbase + __ffs(mask) - 1;
                mask &= mask - 1;
                if (STATS) ++cnt_exec;
                eval_slot<STATS>(st, j, q, cnt_alg);
            }
        }
    }

#pragma unroll
    for (int p = 0; p < PPT; ++p) q.acc[p] = min(q.acc[p], COV_ONE);

    if (split_slot >= 0) {
        // merge into the tile's slot; the last item to arrive writes it out
        const int lp0 = lx + TILE * ly0;
        unsigned long long* __restrict__ sacc = split.acc + (size_t)split_slot * TILE_PIX;
        unsigned long long* __restrict__ skey = split.key + (size_t)split_slot * TILE_PIX;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if (q.acc[p]) atomicAdd(&sacc[lp0 + TILE * 4 * p], (unsigned long long)q.acc[p]);
            if (q.key[p] != ~0ull) atomicMin(&skey[lp0 + TILE * 4 * p], q.key[p]);
        }
        __threadfence();
        __syncthreads();
        __shared__ int s_last;
        if (threadIdx.x == 0) s_last = atomicAdd(&split.done[split_slot], 1u) == (unsigned)(nsplit - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            q.acc[p] = (uint32_t)min(atomicExch(&sacc[lp0 + TILE * 4 * p], 0ull), (unsigned long long)COV_ONE);
            q.key[p] = atomicExch(&skey[lp0 + TILE * 4 * p], ~0ull);
        }
        if (threadIdx.x == 0) split.done[split_slot] = 0u;
    }

    if constexpr (!ROWS) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if (!inimg[p]) continue;
            const size_t o = (size_t)(py0 + 4 * p) * W + px;
            const bool hit = q.key[p] != ~0ull;
            if (out_id) out_id[o] = hit ? (uint32_t)(q.key[p] & 0xffffffffull) : 0xffffffffu;
            if (out_depth) out_depth[o] = hit ? __uint_as_float((uint32_t)(q.key[p] >> 32)) : INFINITY;
            if (out_cov) out_cov[o] = (float)q.acc[p] * (1.0f / (float)COV_ONE);
            if (STATS && n_inside) n_inside[o] = q.cnt_in[p];
        }
    } else {
        // Through shared memory, so that each warp store covers two whole tile
        // rows (16 pixels, 64 B each) instead of four 8-pixel pieces: over the
        // host link 32-byte pieces cost about a quarter of its bandwidth.
        __shared__ uint32_t s_out[3][TILE_PIX];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int lp = lx + TILE * (ly0 + 4 * p);
            const bool hit = q.key[p] != ~0ull;
            s_out[0][lp] = hit ? (uint32_t)(q.key[p] & 0xffffffffull) : 0xffffffffu;
            s_out[1][lp] = hit ? (uint32_t)(q.key[p] >> 32) : __float_as_uint(INFINITY);
            s_out[2][lp] = __float_as_uint((float)q.acc[p] * (1.0f / (float)COV_ONE));
            if (STATS && n_inside && inimg[p]) n_inside[(size_t)(py0 + 4 * p) * W + px] = q.cnt_in[p];
        }
        __syncthreads();
#pragma unroll
        for (int i = threadIdx.x; i < TILE_PIX; i += RT) {
            const int ox = tx * TILE + (i % TILE), oy = ty * TILE + i / TILE;
            if (ox >= W || oy >= H) continue;
            const size_t o = (size_t)oy * W + ox;
            if (out_id) out_id[o] = s_out[0][i];
            if (out_depth) out_depth[o] = __uint_as_float(s_out[1][i]);
            if (out_cov) out_cov[o] = __uint_as_float(s_out[2][i]);
        }
    }
}

template <bool STATS>
__global__ void __launch_bounds__(RT, 7) raster_kernel(RasterView view, unsigned long long* __restrict__ n_alg,
                                                        unsigned long long* __restrict__ n_exec,
                                                        int32_t* __restrict__ n_inside, int* __restrict__ status)
{
    __shared__ Stage st;
    __shared__ unsigned long long red[2][RT / 32];
    uint32_t cnt_alg = 0, cnt_exec = 0;
    raster_tile<STATS>(view, blockIdx.x, st, n_alg != nullptr, cnt_alg, cnt_exec, n_inside, status);
    if (STATS && (n_alg || n_exec)) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        // cnt_exec counts warp-level evaluations: one per (warp, triangle) for 64 pixels
        unsigned long long va = cnt_alg, ve = lane == 0 ? (unsigned long long)cnt_exec * (32ull * PPT) : 0ull;
        for (int o = 16; o; o >>= 1) {
            va += __shfl_xor_sync(0xffffffffu, va, o);
            ve += __shfl_xor_sync(0xffffffffu, ve, o);
        }
        if (lane == 0) {
            red[0][warp] = va;
            red[1][warp] = ve;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long sa = 0, se = 0;
            for (int w = 0; w < RT / 32; ++w) {
                sa += red[0][w];
                se += red[1][w];
            }
            if (n_alg) atomicAdd(n_alg, sa);
            if (n_exec) atomicAdd(n_exec, se);
        }
    }
}

// Raster over work items, one CTA each.  Items 0 .. n_tiles-1 are the tiles
// themselves (the first item of a split tile); the further items of split
// tiles are listed in `extra` as (tile, k).  CTAs past the end of the list
// return at once.
template <bool ROWS>
__global__ void __launch_bounds__(RT, VSR_RASTER_CTAS_PER_SM) raster_items_kernel(RasterView view, uint32_t n_tiles,
                                                              const uint32_t* __restrict__ nsplit_of,
                                                              const int32_t* __restrict__ split_slot,
                                                              const uint2* __restrict__ extra,
                                                              const uint32_t* __restrict__ n_extra, int split_max,
                                                              SplitAcc split, int* __restrict__ status)
{
    __shared__ Stage st;
    uint32_t u, k = 0;
    if (blockIdx.x < n_tiles) {
        u = blockIdx.x;
    } else {
        const uint32_t e = blockIdx.x - n_tiles;
        if (e >= *n_extra) return;
        const uint2 uk = extra[e];
        if (uk.x == 0xffffffffu) return;
        u = uk.x;
        k = uk.y;
    }
    const int nsplit = (int)nsplit_of[u];
    uint32_t ca = 0, ce = 0;
    if (nsplit == 1)
        raster_tile<false, ROWS>(view, (int)u, st, false, ca, ce, nullptr, status);
    else
        raster_tile<false, ROWS>(view, (int)u, st, false, ca, ce, nullptr, status, (int)k * split_max,
                           (int)(k + 1) * split_max, split_slot[u], nsplit, split);
}

// The work items of several views in one persistent launch: each CTA takes
// the next item of a shared queue (an atomic counter over the views' item
// ranges, item_start[v] .. item_start[v + 1]: the view's tiles, then room
// for its extra items) until none is left, and rasterizes it exactly as
// raster_items_kernel does.  The views' items must have been assigned
// (items_kernel) on the launching stream before.
__global__ void __launch_bounds__(RT, VSR_RASTER_CTAS_PER_SM) raster_pool_kernel(const PoolView* __restrict__ views,
                                                                                 const uint32_t* __restrict__ item_start,
                                                                                 int nviews, uint32_t* __restrict__ queue,
                                                                                 int split_max, int* __restrict__ status)
{
    __shared__ Stage st;
    __shared__ uint32_t s_item;
    const uint32_t total = item_start[nviews];
    for (;;) {
        __syncthreads();  // the previous item is done with the shared memory
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= total) return;
        int v = 0;  // the last view whose items start at or before `it`
        for (int hi = nviews - 1; v < hi;) {
            const int mid = (v + hi + 1) >> 1;
            if (item_start[mid] <= it)
                v = mid;
            else
                hi = mid - 1;
        }
        const PoolView& pv = views[v];
        const uint32_t e = it - item_start[v];
        uint32_t u, k = 0;
        if (e < pv.n_tiles) {
            u = e;
        } else {
            const uint32_t x = e - pv.n_tiles;
            if (x >= *pv.n_extra) continue;
            const uint2 uk = pv.extra[x];
            if (uk.x == 0xffffffffu) continue;
            u = uk.x;
            k = uk.y;
        }
        const int nsplit = (int)pv.nsplit_of[u];
        uint32_t ca = 0, ce = 0;
        if (nsplit == 1)
            raster_tile<false>(pv.view, (int)u, st, false, ca, ce, nullptr, status);
        else
            raster_tile<false>(pv.view, (int)u, st, false, ca, ce, nullptr, status, (int)k * split_max,
                               (int)(k + 1) * split_max, pv.split_slot[u], nsplit,
                               SplitAcc{pv.acc, pv.key, pv.done});
    }
}

// Dense reference of the same rasterization: every pixel of a tile against
// every triangle of the scene, with no binning and no cull.  As in the
// oracle, the miter distance is evaluated first: a triangle whose enlarged
// cap holds none of the warp's 64 pixels is skipped after it (a warp vote),
// else the coverage kernel's own evaluation follows.  The outputs equal the
// binned path's bit for bit (the same arithmetic per pair, and the merge is
// order-free); its cost is that of W x H x T pair tests.
__global__ void __launch_bounds__(RT) raster_dense_kernel(RasterView view, int* __restrict__ status)
{
    __shared__ Stage st;
    const int tile = blockIdx.x;
    const int W = view.W, H = view.H, T = view.T;
    const int tx = tile % view.tiles_x, ty = tile / view.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = tx * TILE + (warp & 1) * 8 + (lane & 7);
    const int py0 = ty * TILE + (warp >> 1) * 8 + (lane >> 3);
    const Cone tc = view.tiles[tile];
    const float ax = tc.c0.x, ay = tc.c0.y, az = tc.c0.z;
    PixPair q;
    float gx[PPT], gy[PPT], gz[PPT];
    bool pv[PPT], inimg[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int py = py0 + 4 * p;
        inimg[p] = px < W && py < H;
        float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (inimg[p]) g = view.map[(size_t)py * W + px];
        pv[p] = g.w > 0.0f;
        gx[p] = g.x;
        gy[p] = g.y;
        gz[p] = g.z;
        q.delta[p] = g.w;
        q.lim[p] = pv[p] ? -0.5f / g.w : INFINITY;
        q.acc[p] = 0u;
        q.key[p] = ~0ull;
        q.cnt_in[p] = 0;
    }
    q.dgx = make_float2(gx[0] - ax, gx[1] - ax);
    q.dgy = make_float2(gy[0] - ay, gy[1] - ay);
    q.dgz = make_float2(gz[0] - az, gz[1] - az);
    q.eg = make_float2(pv[0] ? norm2_minus_one(gx[0], gy[0], gz[0]) : 0.0f,
                       pv[1] ? norm2_minus_one(gx[1], gy[1], gz[1]) : 0.0f);
    const bool active = tc.c1.z > 0.0f;
    const size_t TT = (size_t)T;
    uint32_t unused = 0;
    for (int base = 0; active && base < T; base += CHUNK) {
        const int n = min(CHUNK, T - base);
#pragma unroll
        for (int p = 0; p < PPT; ++p) q.acc[p] = min(q.acc[p], COV_ONE);
        __syncthreads();
        if ((int)threadIdx.x < n) {
            const uint32_t t = (uint32_t)(base + threadIdx.x);
            if (view.rec[RF_CAP2 * TT + t].w == 0.0f)  // culled at set-up
                st.s6[threadIdx.x] = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(STAGE_EMPTY));
            else
                stage_triangle(view.rec, TT, t, ax, ay, az, st, threadIdx.x);
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const float4 e = st.s6[j];
            if (__float_as_uint(e.w) == STAGE_EMPTY) continue;
            const float2 g4 = miter_distance2(q.dgx, q.dgy, q.dgz, e, st.s1[j], q.eg);
            if (!__any_sync(0xffffffffu, g4.x > q.lim[0] || g4.y > q.lim[1])) continue;
            eval_slot<false>(st, j, q, unused);
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (!inimg[p]) continue;
        const size_t o = (size_t)(py0 + 4 * p) * W + px;
        const uint32_t acc = min(q.acc[p], COV_ONE);
        const bool hit = q.key[p] != ~0ull;
        if (view.out_id) view.out_id[o] = hit ? (uint32_t)(q.key[p] & 0xffffffffull) : 0xffffffffu;
        if (view.out_depth) view.out_depth[o] = hit ? __uint_as_float((uint32_t)(q.key[p] >> 32)) : INFINITY;
        if (view.out_cov) view.out_cov[o] = (float)acc * (1.0f / (float)COV_ONE);
    }
}

// Work items per tile: ceil(bin / split_max) when a split slot and room in
// the extra list are free, else 1 (the tile runs in one CTA).
__global__ void items_kernel(const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ ends,
                             uint32_t n_tiles, int split_max, uint32_t* __restrict__ nsplit_of,
                             int32_t* __restrict__ split_slot, uint32_t* __restrict__ counters /* n_split, n_extra */,
                             uint32_t split_cap, uint2* __restrict__ extra, uint32_t extra_cap)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_tiles) return;
    const uint32_t c = (ends ? ends[u] : offsets[u + 1]) - offsets[u];
    uint32_t n = 1;
    int32_t slot = -1;
    if (c > (uint32_t)split_max) {
        const uint32_t want = (c + split_max - 1) / split_max;
        const uint32_t sl = atomicAdd(&counters[0], 1u);
        const uint32_t pos = atomicAdd(&counters[1], want - 1);
        const bool ok = sl < split_cap && pos + (want - 1) <= extra_cap;
        for (uint32_t q = 1; q < want && pos + q - 1 < extra_cap; ++q)
            extra[pos + q - 1] = ok ? make_uint2(u, q) : make_uint2(0xffffffffu, 0u);
        if (ok) {
            n = want;
            slot = (int32_t)sl;
        }
    }
    nsplit_of[u] = n;
    split_slot[u] = slot;
}

}  // namespace

vsr_status launch_raster(const float4* map, int W, int H, const Cone* tiles, const float4* rec, int T,
                         const uint32_t* offsets, const uint32_t* ids, uint32_t cap, uint32_t* id, float* depth,
                         float* cov, unsigned long long* n_alg, unsigned long long* n_exec, int32_t* n_inside,
                         int* status, cudaStream_t st, const uint32_t* ends)
{
    const int tx = (W + TILE - 1) / TILE, ty = (H + TILE - 1) / TILE;
    const RasterView v{map, W, H, tiles, tx, rec, T, offsets, ids, cap, id, depth, cov, ends};
    if (n_alg || n_exec || n_inside)
        raster_kernel<true><<<tx * ty, RT, 0, st>>>(v, n_alg, n_exec, n_inside, status);
    else
        raster_kernel<false><<<tx * ty, RT, 0, st>>>(v, nullptr, nullptr, nullptr, status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

int raster_split_items(int split_max) { return split_max < CHUNK ? CHUNK : (split_max / CHUNK) * CHUNK; }

uint32_t raster_extra_cap(uint32_t cap, const RasterWork& w, int split_max)
{
    // enough extra items for every pair of the bins, bounded by the list
    const uint64_t bound = (uint64_t)cap / (uint64_t)raster_split_items(split_max) + 1;
    return bound < w.extra_cap ? (uint32_t)bound : w.extra_cap;
}

vsr_status launch_raster_assign(const uint32_t* offsets, uint32_t n_tiles, uint32_t cap, RasterWork w, int split_max,
                                cudaStream_t st, const uint32_t* ends)
{
    if (n_tiles == 0) return VSR_OK;
    VSR_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 2 * sizeof(uint32_t), st));
    items_kernel<<<(n_tiles + 255) / 256, 256, 0, st>>>(offsets, ends, n_tiles, raster_split_items(split_max),
                                                        w.nsplit_of, w.split_slot, w.counters, w.split_cap, w.extra,
                                                        raster_extra_cap(cap, w, split_max));
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_raster_pool(const PoolView* views_dev, const uint32_t* item_start_dev, int nviews,
                              uint32_t* queue, int split_max, int* status, cudaStream_t st)
{
    if (nviews == 0) return VSR_OK;
    const int sms = sm_count();
    if (sms < 0) return VSR_ERR_CUDA;
    VSR_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(uint32_t), st));
    raster_pool_kernel<<<sms * VSR_RASTER_CTAS_PER_SM, RT, 0, st>>>(views_dev, item_start_dev, nviews, queue,
                                                                    raster_split_items(split_max), status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_raster_items(const RasterView& view, const uint32_t* offsets, uint32_t n_tiles, uint32_t cap,
                               RasterWork w, int split_max, int* status, cudaStream_t st, bool host_out)
{
    if (n_tiles == 0) return VSR_OK;
    vsr_status s = launch_raster_assign(offsets, n_tiles, cap, w, split_max, st, view.ends);
    if (s != VSR_OK) return s;
    const uint32_t extra_cap = raster_extra_cap(cap, w, split_max);
    split_max = raster_split_items(split_max);
    auto kern = host_out ? raster_items_kernel<true> : raster_items_kernel<false>;
    kern<<<n_tiles + extra_cap, RT, 0, st>>>(view, n_tiles, w.nsplit_of, w.split_slot, w.extra, w.counters + 1,
                                             split_max, SplitAcc{w.acc, w.key, w.done}, status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_raster_dense(const RasterView& view, int* status, cudaStream_t st)
{
    const int n_tiles = view.tiles_x * ((view.H + TILE - 1) / TILE);
    if (n_tiles == 0) return VSR_OK;
    raster_dense_kernel<<<n_tiles, RT, 0, st>>>(view, status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

int raster_threads_per_cta() { return RT; }

vsr_status raster_work_alloc(RasterWork* w, uint32_t n_tiles)
{
    *w = RasterWork{};
    const uint32_t cap = n_tiles < SPLIT_SLOTS ? n_tiles : SPLIT_SLOTS;
    const uint32_t xcap = EXTRA_ITEMS;
    if (cudaMalloc((void**)&w->nsplit_of, sizeof(uint32_t) * (n_tiles + 1)) != cudaSuccess ||
        cudaMalloc((void**)&w->split_slot, sizeof(int32_t) * (n_tiles + 1)) != cudaSuccess ||
        cudaMalloc((void**)&w->counters, sizeof(uint32_t) * 2) != cudaSuccess ||
        cudaMalloc((void**)&w->extra, sizeof(uint2) * xcap) != cudaSuccess ||
        cudaMalloc((void**)&w->acc, sizeof(unsigned long long) * TILE_PIX * ((size_t)cap + 1)) != cudaSuccess ||
        cudaMalloc((void**)&w->key, sizeof(unsigned long long) * TILE_PIX * ((size_t)cap + 1)) != cudaSuccess ||
        cudaMalloc((void**)&w->done, sizeof(uint32_t) * ((size_t)cap + 1)) != cudaSuccess) {
        cudaGetLastError();
        raster_work_free(w);
        return VSR_ERR_OOM;
    }
    w->split_cap = cap;
    w->extra_cap = xcap;
    if (cudaMemset(w->acc, 0, sizeof(unsigned long long) * TILE_PIX * ((size_t)cap + 1)) != cudaSuccess ||
        cudaMemset(w->key, 0xff, sizeof(unsigned long long) * TILE_PIX * ((size_t)cap + 1)) != cudaSuccess ||
        cudaMemset(w->done, 0, sizeof(uint32_t) * ((size_t)cap + 1)) != cudaSuccess) {
        raster_work_free(w);
        return VSR_ERR_CUDA;
    }
    return VSR_OK;
}

void raster_work_free(RasterWork* w)
{
    cudaFree(w->nsplit_of);
    cudaFree(w->split_slot);
    cudaFree(w->counters);
    cudaFree(w->extra);
    cudaFree(w->acc);
    cudaFree(w->key);
    cudaFree(w->done);
    *w = RasterWork{};
}
