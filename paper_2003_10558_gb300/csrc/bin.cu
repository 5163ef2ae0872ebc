// bin.cu -- tile binning: which triangles may produce a fragment in which
// 16x16 tile.
//
// A fragment of triangle t at pixel direction G needs G inside the miter
// cap enlarged by the ramp half-width (the gbpxstep test of the miter plane,
// Sec. 1.1.1 / 1.1.2): G.S-hat - cos rho > -h sin rho, h = 1/(2 delta).  A
// binner keeps (tile, t) when that enlarged cap can reach the tile's view
// cone (cap_hits_cone).  The paper's analogue is the low-resolution region
// mask widened by fwidth/2 (getPolygonRegion).
//
// Two binners with the same cap / cone test:
//  * tile-major (every frame of a scene or batch view): the frame's
//    triangles filed by the cell of their cap centre on a latitude-longitude
//    grid, then one warp per tile over the cells within its reach, in one
//    pass (tri_file_kernel, bin_tiles_kernel; see TriIndex);
//  * triangle-major (the fixed-array path, vsr_raster_noalloc): every
//    triangle visits the cells of the map's tile index within beta +
//    alpha_small_max of its cap centre (a few dozen cone tests whatever the
//    map's size; no tile is found twice); count (atomic per-tile counters)
//    -> exclusive scan -> fill (atomic per-tile cursors).
// The order of ids inside a bin is not fixed; the raster kernels' results
// do not depend on it.
#include <math.h>
#include <stddef.h>

#include <algorithm>
#include <atomic>


#include "vsr_internal.cuh"

namespace {

constexpr float PI_F = IDX_PI;

__device__ __forceinline__ float hist_upper(int b) { return exp2f((float)(b + 1) / 3.0f - 17.0f); }

// ---- tile index -------------------------------------------------------------
//
// Built from the per-tile geometry the map kernels write (TileIndex::geom:
// half-angle, axis latitude / longitude, ramp half-width) by one CTA
// (idx_fused_kernel, maps of up to IDX_FUSED_TILES tiles): the histogram of
// half-angles, the grid plan (a 64-bin walk), the per-cell counts, their
// exclusive scan and the cell-sorted copies of the small tiles' cones.

// the grid plan: cell size from the 99th percentile of the half-angles
__device__ void index_plan(const TileIndexHdr* hdr, TileIndexHdr& h)
{
    const unsigned nvalid = hdr->n_valid;
    const unsigned target = (unsigned)ceilf(0.99f * (float)nvalid);
    unsigned run = 0;
    int b = 0;
    for (; b < IDX_HIST; ++b) {
        run += hdr->hist[b];
        if (run >= target) break;
    }
    const float cut = hist_upper(min(b, IDX_HIST - 1));
    const float cell = fminf(PI_F / 8.0f, fmaxf(PI_F / IDX_NLAT_MAX, cut));
    const int nlat = min(IDX_NLAT_MAX, (int)ceilf(PI_F / cell));
    h.nlat = nlat;
    h.nlon = 2 * nlat;
    h.ncell = 2 * nlat * nlat;
    h.cell = PI_F / nlat;
    h.alpha_cut = cut;
}

// The tile loops of the one-CTA index kernels take IDX_BATCH tiles per
// thread at a time and issue each step for all of them before the next
// (geometry loads, then slots, then cone loads, then stores), so their
// memory latencies overlap instead of adding up tile after tile.
constexpr int IDX_BATCH = 4;

__device__ __forceinline__ void load_geom_batch(const float4* __restrict__ geom, int ntiles, int base, int stride,
                                                float4 (&g)[IDX_BATCH])
{
#pragma unroll
    for (int u = 0; u < IDX_BATCH; ++u) {
        const int i = base + u * stride;
        g[u] = i < ntiles ? geom[i] : make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    }
}

// Exclusive scan of n counts in shared memory, in place, by a CTA of
// NT threads (all of which call it; ends with a barrier); returns the total
// to every thread.  Warp w owns a contiguous segment of cells and walks it 32
// cells at a time, lane l on cell 32 k + l of the step (no bank conflicts),
// with a shuffle scan per step.
template <int NT>
__device__ uint32_t block_scan_smem(uint32_t* s, int n, uint32_t* s_wsum /* NT / 32 words */)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = ((n + NW - 1) / NW + 31) & ~31;
    const int b0 = min(n, warp * seg), b1 = min(n, b0 + seg);
    uint32_t tot = 0;
    for (int c = b0 + lane; c < b1; c += 32) tot += s[c];
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) s_wsum[warp] = tot;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_wsum[lane] = w;  // inclusive
    }
    __syncthreads();
    uint32_t carry = warp > 0 ? s_wsum[warp - 1] : 0u;
    const uint32_t total = s_wsum[NW - 1];
    for (int c0 = b0; c0 < b1; c0 += 32) {
        const int c = c0 + lane;
        const uint32_t v = c < b1 ? s[c] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (c < b1) s[c] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    __syncthreads();
    return total;
}

// The whole index in one CTA, for maps of at most IDX_FUSED_TILES tiles:
// the histogram, the per-cell counts and their scan in shared memory
// (IDX_CELLS_MAX counters), steps closed by barriers, and the header written
// once at the end.
constexpr int IDX_FUSED_THREADS = 1024;
constexpr int IDX_FUSED_TILES = 32768;
static_assert(IDX_CELLS_MAX <= 65535, "home cells are kept as 16-bit indices");
constexpr size_t IDX_FUSED_SMEM = sizeof(uint32_t) * IDX_CELLS_MAX + sizeof(uint16_t) * IDX_FUSED_TILES;

__global__ void __launch_bounds__(IDX_FUSED_THREADS) idx_fused_kernel(const Cone* __restrict__ tiles,
                                                                       const float4* __restrict__ geom, int ntiles,
                                                                       TileIndexHdr* __restrict__ hdr,
                                                                       uint32_t* __restrict__ cell_start,
                                                                       Cone* __restrict__ sorted,
                                                                       Cone* __restrict__ big)
{
    extern __shared__ uint32_t s_cell[];  // per-cell counts, then running slots
    // each small tile's home cell (0xffff: big or empty), from step 3 to step 5
    uint16_t* s_tcell = reinterpret_cast<uint16_t*>(s_cell + IDX_CELLS_MAX);
    __shared__ TileIndexHdr s_h;
    __shared__ uint32_t s_wsum[IDX_FUSED_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        s_h = TileIndexHdr{};
        s_h.h_gen = hdr->h_gen;  // the map kernels' word, kept
    }
    __syncthreads();
    // 1. histogram of half-angles (one add per group of equal bins in a
    // warp), valid tiles, widest ramp (one atomic per warp)
    uint32_t nv = 0u, hm = 0u, va = 0u;
    for (int base = 0; base < ntiles; base += IDX_FUSED_THREADS * IDX_BATCH) {
        float4 gb[IDX_BATCH];
        load_geom_batch(geom, ntiles, base + tid, IDX_FUSED_THREADS, gb);
#pragma unroll
        for (int u = 0; u < IDX_BATCH; ++u) {
            const float4 g = gb[u];
            const bool ok = g.w >= 0.0f;
            const int bin = ok ? hist_bin(g.x) : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (ok && lane == __ffs(peers) - 1) atomicAdd(&s_h.hist[bin], (unsigned)__popc(peers));
            nv += ok;
            hm = max(hm, ok ? __float_as_uint(g.w) : 0u);  // non-negative floats order as their bits
            if (ok) va = max(va, view_angle_bits(tiles[base + tid + u * IDX_FUSED_THREADS], g.x));
        }
    }
    for (int o = 16; o; o >>= 1) {
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, o));
        va = max(va, __shfl_xor_sync(0xffffffffu, va, o));
    }
    if (lane == 0 && nv) {
        atomicAdd(&s_h.n_valid, nv);
        atomicMax(&s_h.h_max, hm);
        atomicMax(&s_h.view_angle, va);
    }
    __syncthreads();
    // 2. the grid plan
    if (tid == 0) index_plan(&s_h, s_h);
    __syncthreads();
    const int ncell = s_h.ncell;
    for (int c = tid; c < ncell; c += IDX_FUSED_THREADS) s_cell[c] = 0u;
    __syncthreads();
    // 3. per-cell counts; big tiles to their own list
    uint32_t am = 0u;
    for (int base = tid; base < ntiles; base += IDX_FUSED_THREADS * IDX_BATCH) {
        float4 gb[IDX_BATCH];
        load_geom_batch(geom, ntiles, base, IDX_FUSED_THREADS, gb);
#pragma unroll
        for (int u = 0; u < IDX_BATCH; ++u) {
            const float4 g = gb[u];
            const int i = base + u * IDX_FUSED_THREADS;
            if (i >= ntiles) continue;
            uint16_t home = 0xffffu;
            if (g.w >= 0.0f) {
                if (g.x > s_h.alpha_cut) {
                    big[atomicAdd(&s_h.n_big, 1u)] = index_entry(tiles[i], i);
                } else {
                    const int c = home_cell_geom(g, s_h);
                    atomicAdd(&s_cell[c], 1u);
                    home = (uint16_t)c;
                    am = max(am, __float_as_uint(g.x));
                }
            }
            s_tcell[i] = home;
        }
    }
    for (int o = 16; o; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
    if (lane == 0 && am) atomicMax(&s_h.alpha_small_max, am);
    __syncthreads();
    // 4. exclusive scan of the counts (in place: they become running slots),
    // the starts out (coalesced)
    const uint32_t total = block_scan_smem<IDX_FUSED_THREADS>(s_cell, ncell, s_wsum);
    for (int c = tid; c < ncell; c += IDX_FUSED_THREADS) cell_start[c] = s_cell[c];
    if (tid == 0) cell_start[ncell] = total;
    // 5. cell-sorted copies of the small tiles (slots, then cone loads, then stores)
    for (int base = tid; base < ntiles; base += IDX_FUSED_THREADS * IDX_BATCH) {
        uint32_t slot[IDX_BATCH];
#pragma unroll
        for (int u = 0; u < IDX_BATCH; ++u) {
            const int i = base + u * IDX_FUSED_THREADS;
            const uint16_t c = i < ntiles ? s_tcell[i] : (uint16_t)0xffffu;
            slot[u] = c != 0xffffu ? atomicAdd(&s_cell[c], 1u) : 0xffffffffu;
        }
        Cone cn[IDX_BATCH];
#pragma unroll
        for (int u = 0; u < IDX_BATCH; ++u)
            if (slot[u] < (uint32_t)ntiles) cn[u] = tiles[base + u * IDX_FUSED_THREADS];
#pragma unroll
        for (int u = 0; u < IDX_BATCH; ++u)
            if (slot[u] < (uint32_t)ntiles) sorted[slot[u]] = index_entry(cn[u], base + u * IDX_FUSED_THREADS);
    }
    if (tid == 0) *hdr = s_h;
}

// ---- per-triangle binning ---------------------------------------------------
//
// The candidate tiles of a triangle are the cones of its search window: the
// index rows r0..r1 around the cap centre, each a contiguous range of the
// cell-sorted cones (two ranges where the window wraps across longitude
// +-pi), plus the big tiles.  One warp bins 32 triangles.  Phase 1, one lane
// per triangle: the cap enlarged by the widest ramp and the window.  Phase
// 2: the windows' (triangle, row range) pairs -- the big list cut into
// chunks of BIN_BIG_CHUNK cones counts as further pairs -- are concatenated
// in lane order and handed out one pair per lane per round, so the
// dependent loads of the search run on all lanes at once instead of one
// lane walking its whole window.
//
// count: counts[tile] += 1 per hit (no value returned, so nothing waits),
// and the hit is recorded as (tile, triangle) in the pair list -- staged per
// warp in shared memory and appended with one atomic per warp and round.
// fill: a map over the pair list that takes slot counts[tile] - 1 by atomic
// decrement (one pair per thread, so the atomics' latency overlaps) and
// writes ids[offsets[tile] + slot] = triangle.  When the list would overflow
// (the first binning of a new shape, whose capacity is not known yet, or a
// caller without a list) the fill searches again instead, with the same
// decrement.  The counts return to zero either way; the order of ids inside
// a bin is not fixed and the raster kernels' results do not depend on it.
// (Keeping each hit's slot -- the old value of its counter -- would spare
// the fill its atomics, but makes the count pass wait for each counter's
// return: measured 44.3 -> 58.7 us for the count against 17.2 -> 8.6 us for
// the fill on the 1080p frame.)

constexpr int BIN_BIG_CHUNK = 16;
// cones per step of the search for grids beyond one resident wave
// The longest cone range of a warp round, in steps of the flattened walk,
// above which the round walks its cones flattened across the warp.
#ifndef VSR_BIN_FLAT_RATIO
#define VSR_BIN_FLAT_RATIO 2
#endif

// triangles per warp of the large-grid shape: 16 (measured on the 1080p
// frame's 220k triangles: bin stage 65.9 us against 73.8 us at 32 and 67.7 us
// at 8) -- the grid is then two resident waves, and each warp's chain of
// dependent loads (window rows, then cones) half as long
#ifndef VSR_BIN_TPW_LARGE
#define VSR_BIN_TPW_LARGE 16
#endif

#ifndef VSR_BIN_CB_LARGE
#define VSR_BIN_CB_LARGE 1
#endif
constexpr int BIN_STAGE = 256;  // hits staged per warp (appended when half full)

// FILL: false = count + record, true = fill by searching again.
// CB: cones each lane fetches per step.  The search is bound by load latency:
// a grid larger than one resident wave hides it with warps (CB = 1: 40
// registers, 12 CTAs per SM), a smaller one with loads in flight per lane
// (CB = 4, 7 CTAs per SM).
// TPW: triangles per warp (lanes 0 .. TPW-1 run phase 1; phase 2 spreads
// their pairs over all 32 lanes).  8 for small scenes, so that they still
// give the GPU enough warps to hide the search's latency.
template <bool FILL, int CB, int TPW>
__global__ void __launch_bounds__(128, CB == 1 ? 12 : (CB == 2 ? 10 : 1)) bin_kernel(BinView v, int T,
                                                                                   uint32_t* __restrict__ ids,
                                                                     uint32_t cap, int* status)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = (int)(blockIdx.x * 4 + warp) * TPW + lane;
    if (FILL && v.pairs && *v.cursor <= v.pair_cap) return;  // the pair list is complete: bin_pairs_kernel fills
    const size_t TT = (size_t)T;
    // The index header, with every count that becomes an index clamped to
    // the arrays it indexes (identity for an index built by launch_tile_index),
    // so that no index content can make this kernel read or write out of
    // bounds.
    TileIndexHdr h;
    h.nlat = min(max(v.hdr->nlat, 1), IDX_NLAT_MAX);
    h.nlon = 2 * h.nlat;
    h.cell = v.hdr->cell;
    const int nlat = h.nlat, nlon = h.nlon;
    const float cell = h.cell;
    const float amax = __uint_as_float(v.hdr->alpha_small_max), hmax = __uint_as_float(v.hdr->h_max);
    // the map's field of view: a cone about +z of half-angle view_angle
    // holding every tile cone; a cap that misses it misses every tile (a
    // view angle of pi or more holds the whole sphere: no cap misses it)
    const float vang = __uint_as_float(v.hdr->view_angle);
    const bool fov = vang < PI_F;
    float vcos, vsin;
    sincosf(fminf(vang, PI_F), &vsin, &vcos);
    const uint32_t nbig = min(v.hdr->n_big, v.ntiles);
    const int bigpairs = (int)((nbig + BIN_BIG_CHUNK - 1) / BIN_BIG_CHUNK);
    __shared__ uint2 s_hit[4][BIN_STAGE];
    __shared__ uint32_t s_nhit[4];
    if (!FILL && lane == 0) s_nhit[warp] = 0u;
    __syncwarp();

    // phase 1: this lane's triangle
    float sx = 0.0f, sy = 0.0f, sz = 1.0f, cb = 1.0f, sb = 0.0f;
    int r0 = 0, c0i = 0, ncol = 0, segs = 1, rowpairs = 0, npairs = 0;
    if (lane < TPW && t < T) {
        const float4 q0 = v.rec[RF_CAP * TT + t];
        const float4 q1 = v.rec[RF_CAP2 * TT + t];
        if (q1.w != 0.0f) {
            sx = q0.x;
            sy = q0.y;
            sz = q0.z;
            // the cap enlarged once by the map's widest ramp (>= every tile's
            // own): cos / sin of its radius beta, so each tile test is a few FMAs
            if (v.pstep) {
                const float2 c = pstep_cap(q0.w, q1.x, hmax);
                cb = c.x;
                sb = c.y;
            } else {
                cb = fmaxf(-1.0f, fminf(1.0f, q0.w - hmax * q1.x));
                sb = sqrtf(fmaxf(0.0f, 1.0f - cb * cb));
            }
            // outside the field of view: no window, no pairs.  The cap of
            // radius beta reaches the view cone iff angle(S, +z) <= beta +
            // view angle, i.e. S.z >= cos(beta + view angle) while the sum
            // is below pi; with both angles in [0, pi) the sum is below pi
            // exactly when its sine is positive
            const float cbv = fmaf(cb, vcos, -sb * vsin), sbv = fmaf(sb, vcos, cb * vsin);
            const bool outside = fov && sbv > 0.0f && sz < cbv - 2e-6f;
            // search radius: enlarged cap + largest small tile
            const float gamma = outside ? PI_F : acosf(cb) + amax + 1e-4f;
            int r1 = nlat - 1;
            ncol = nlon;
            if (gamma < PI_F) {
                const float lat = asinf(fmaxf(-1.0f, fminf(1.0f, sy)));
                const float lon = atan2f(sx, sz);
                r0 = cell_row(lat - gamma, h);
                r1 = cell_row(lat + gamma, h);
                if (fabsf(lat) + gamma < 0.5f * PI_F - 1e-3f) {
                    // longitude half-width of a cap that holds no pole
                    const float dl = asinf(fminf(1.0f, sinf(gamma) / cosf(lat))) + 1e-4f;
                    c0i = (int)floorf((lon - dl + PI_F) / cell);
                    const int c1i = (int)floorf((lon + dl + PI_F) / cell);
                    ncol = max(1, min(nlon, c1i - c0i + 1));
                    c0i %= nlon;
                    if (c0i < 0) c0i += nlon;
                }
            }
            segs = c0i + ncol <= nlon ? 1 : 2;
            rowpairs = (r1 - r0 + 1) * segs;
            npairs = outside ? 0 : rowpairs + bigpairs;
        }
    }
    int incl = npairs;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int off = incl - npairs;

    // phase 2: one (triangle, range) pair per lane and round
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        int q = 0;  // the last lane whose pairs start at or before p
        for (int st = 16; st > 0; st >>= 1) {
            const int oc = __shfl_sync(FULL, off, q + st);
            if (oc <= p) q += st;
        }
        const int u = p - __shfl_sync(FULL, off, q);
        const float tx = __shfl_sync(FULL, sx, q), ty = __shfl_sync(FULL, sy, q), tz = __shfl_sync(FULL, sz, q);
        const float tcb = __shfl_sync(FULL, cb, q), tsb = __shfl_sync(FULL, sb, q);
        const int tr0 = __shfl_sync(FULL, r0, q), tc0 = __shfl_sync(FULL, c0i, q);
        const int tncol = __shfl_sync(FULL, ncol, q), tsegs = __shfl_sync(FULL, segs, q);
        const int trows = __shfl_sync(FULL, rowpairs, q);
        const uint32_t tt = (uint32_t)__shfl_sync(FULL, t, q);
        uint32_t a = 0, b = 0;
        const Cone* __restrict__ list = v.sorted;
        if (p < total) {
            if (u < trows) {
                const int row = tr0 + u / tsegs, seg = u - (u / tsegs) * tsegs;
                const uint32_t* __restrict__ rs = v.cell_start + (size_t)row * nlon;
                if (tsegs == 1) {
                    a = rs[tc0];
                    b = rs[tc0 + tncol];
                } else if (seg == 0) {  // the window wraps across longitude +-pi
                    a = rs[tc0];
                    b = rs[nlon];
                } else {
                    a = rs[0];
                    b = rs[tc0 + tncol - nlon];
                }
            } else {
                a = (uint32_t)(u - trows) * BIN_BIG_CHUNK;
                b = min(nbig, a + BIN_BIG_CHUNK);
                list = v.big;
            }
            b = min(b, v.ntiles);
            a = min(a, b);
        }
        // a hit: count and record it (count pass) or take a slot and fill it
        auto hit = [&](uint32_t tile, uint32_t tri) {
            if (!FILL) {
                atomicAdd(&v.counts[tile], 1u);
                if (v.pairs) {
                    const uint32_t j = atomicAdd(&s_nhit[warp], 1u);
                    if (j < BIN_STAGE) {
                        s_hit[warp][j] = make_uint2(tile, tri);
                    } else {  // a round with more hits than the stage holds: straight to the list
                        const uint32_t g = atomicAdd(v.cursor, 1u);
                        if (g < v.pair_cap) v.pairs[g] = make_uint2(tile, tri);
                    }
                }
            } else {
                const uint32_t pos = v.offsets[tile] + atomicSub(&v.counts[tile], 1u) - 1u;
                if (pos < cap && pos < v.offsets[tile + 1])
                    ids[pos] = tri;
                else
                    raise_status(status, VSR_ERR_BIN_OVERFLOW);
            }
        };
        // the cap / cone test: angle(S, axis) <= alpha + beta (always when
        // alpha + beta >= pi)
        auto reaches = [&](const Cone& c, float x, float y, float z, float cbt, float sbt) {
            const float cg = fmaf(x, c.c0.x, fmaf(y, c.c0.y, z * c.c0.z));
            return cbt + c.c0.w <= 2e-6f || cg >= fmaf(c.c0.w, cbt, -c.c1.x * sbt) - 2e-6f;
        };
        // Two ways through the round's cones.  Each lane walks its own range
        // -- as many steps as the longest range, the other lanes idle once
        // theirs ends -- or, where the ranges are very unequal, the cones are
        // numbered across the warp (lane l's range is [excl_l, excl_l +
        // len_l)) and every lane takes the next cone each step, finding the
        // lane whose range holds it by a search over the lanes.  The second
        // costs more per step (the search and the range's parameters by
        // shuffle), so it is taken when the longest range is over
        // VSR_BIN_FLAT_RATIO times its step count.
        const int len = (int)(b - a);
        int incl = len, lmax = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
            lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
        }
        const int ncones = __shfl_sync(FULL, incl, 31);
        if (lmax <= VSR_BIN_FLAT_RATIO * ((ncones + 31) / 32)) {
            for (uint32_t k0 = a; k0 < b; k0 += CB) {
                Cone cs[CB];
#pragma unroll
                for (int e = 0; e < CB; ++e)
                    if (k0 + e < b) cs[e] = list[k0 + e];
#pragma unroll
                for (int e = 0; e < CB; ++e) {
                    if (k0 + e >= b) break;
                    if (!reaches(cs[e], tx, ty, tz, tcb, tsb)) continue;
                    const uint32_t tile = __float_as_uint(cs[e].c1.z);
                    if (tile < v.ntiles) hit(tile, tt);
                }
            }
        } else {
            const int excl = incl - len;
            const int rel = (int)a - excl;  // list index = cone number + rel
            const int isbig = list == v.big;
            for (int k0 = 0; k0 < ncones; k0 += 32) {
                const int idx = k0 + lane;
                int o = 0;  // the last lane whose range starts at or before cone idx
                for (int st = 16; st > 0; st >>= 1) {
                    const int e = __shfl_sync(FULL, excl, o + st);
                    if (e <= idx) o += st;
                }
                const float ox = __shfl_sync(FULL, tx, o), oy = __shfl_sync(FULL, ty, o),
                            oz = __shfl_sync(FULL, tz, o);
                const float ocb = __shfl_sync(FULL, tcb, o), osb = __shfl_sync(FULL, tsb, o);
                const uint32_t ot = (uint32_t)__shfl_sync(FULL, (int)tt, o);
                const int orel = __shfl_sync(FULL, rel, o), obig = __shfl_sync(FULL, isbig, o);
                if (idx >= ncones) continue;
                const Cone c = (obig ? v.big : v.sorted)[idx + orel];
                if (!reaches(c, ox, oy, oz, ocb, osb)) continue;
                const uint32_t tile = __float_as_uint(c.c1.z);
                if (tile < v.ntiles) hit(tile, ot);
            }
        }
        if (!FILL && v.pairs) {
            // append the staged hits to the pair list once the stage is half
            // full (a round adds about one hit per lane), and at the end
            __syncwarp();
            const uint32_t n = min(s_nhit[warp], (uint32_t)BIN_STAGE);
            if (n >= BIN_STAGE / 2 || base + 32 >= total) {
                uint32_t g0 = 0;
                if (lane == 0 && n) g0 = atomicAdd(v.cursor, n);
                g0 = __shfl_sync(FULL, g0, 0);
                for (uint32_t j = lane; j < n; j += 32)
                    if (g0 + j < v.pair_cap) v.pairs[g0 + j] = s_hit[warp][j];
                __syncwarp();
                if (lane == 0) s_nhit[warp] = 0u;
                __syncwarp();
            }
        }
    }
}

// The fill as a map over the pair list of the count pass (when it is
// complete): slot = --counts[tile], ids[offsets[tile] + slot] = triangle.
__global__ void __launch_bounds__(256) bin_pairs_kernel(const uint2* __restrict__ pairs,
                                                         const uint32_t* __restrict__ cursor, uint32_t pair_cap,
                                                         const uint32_t* __restrict__ offsets,
                                                         uint32_t* __restrict__ counts, uint32_t* __restrict__ ids,
                                                         uint32_t cap, int* status, int overflow_here)
{
    const uint32_t n = *cursor;
    if (n > pair_cap) {
        // incomplete: the search-based fill runs instead -- or, when the list
        // holds as many pairs as the bins, the bins overflow too: report it
        if (overflow_here && blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, VSR_ERR_BIN_OVERFLOW);
        return;
    }
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint2 e = pairs[p];
        const uint32_t pos = offsets[e.x] + atomicSub(&counts[e.x], 1u) - 1u;
        if (pos < cap && pos < offsets[e.x + 1])
            ids[pos] = e.y;
        else
            raise_status(status, VSR_ERR_BIN_OVERFLOW);
    }
}

// Exclusive scan of n counts (+ extra, when not NULL) into offsets[0..n] by
// one CTA of 1024 threads:
// chunks of 4096 (four consecutive elements per thread), carried across
// chunks.  n comes from n_dev when it is not NULL.
__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t* __restrict__ counts,
                                                     const uint32_t* __restrict__ extra, int n_host,
                                                     const int* __restrict__ n_dev, uint32_t* __restrict__ offsets,
                                                     volatile uint32_t* total_host)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry_s;
    const int n = n_dev ? *n_dev : n_host;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 4096) {
        const int b = base + 4 * tid;
        uint32_t v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = b + q < n ? counts[b + q] + (extra ? extra[b + q] : 0u) : 0u;
        const uint32_t local = v[0] + v[1] + v[2] + v[3];
        uint32_t x = local;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        uint32_t run = carry_s + x - local + (warp > 0 ? warp_sums[warp - 1] : 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (b + q < n) offsets[b + q] = run;
            run += v[q];
        }
        __syncthreads();
        if (tid == 0) carry_s += warp_sums[31];
        __syncthreads();
    }
    if (tid == 0) {
        offsets[n] = carry_s;
        if (total_host) {  // the total straight into the host's pinned word (read after an event)
            *total_host = carry_s;
            __threadfence_system();
        }
    }
}

// ---- tile-major binning -----------------------------------------------------
//
// Per frame: tri_file (every triangle into its cell) -> bin_tiles (every
// tile's bin, in one pass).

constexpr float TRI_CELL0 = PI_F / TRI_NLAT0;
constexpr float TRI_CELL1 = PI_F / TRI_NLAT1;
// entries of a tile binned by its own warp (its hits staged in shared
// memory); a tile with more goes to the heavy list
constexpr uint32_t BIN_STAGE_HITS = 1024;
constexpr int BIN_HEAVY_WARPS = 16;  // warps per heavy tile
// steps of the walk whose loads are issued together: 2 (measured on the
// 1080p frame: bin stage 38.9 us against 40.7 us at 4; 12 resident CTAs
// per SM instead of 8, which caps the registers: 40.8 - 48.6 us)
#ifndef VSR_BIN_WALK_U
#define VSR_BIN_WALK_U 2
#endif
constexpr int BIN_WALK_U = VSR_BIN_WALK_U;
// resident CTAs per SM the tile pass is compiled for (its register cap)
#ifndef VSR_BIN_TILES_CTAS
#define VSR_BIN_TILES_CTAS 8
#endif

__device__ __forceinline__ int tri_row(float lat, int nlat, float cell)
{
    return min(nlat - 1, max(0, (int)floorf((lat + 0.5f * PI_F) / cell)));
}

__device__ __forceinline__ int tri_col(float lon, int nlon, float cell)
{
    int c = (int)floorf((lon + PI_F) / cell);
    c %= nlon;
    return c < 0 ? c + nlon : c;
}

// The enlarged cap of triangle t as the triangle-major search forms it: its
// centre (q0.xyz) and (cos, sin) of its radius; false for a triangle
// without a cap.
__device__ __forceinline__ bool tri_cap(const float4* __restrict__ rec, size_t TT, int t, float hmax, int pstep,
                                        float4& q0, float& cb, float& sb)
{
    q0 = rec[RF_CAP * TT + t];
    const float4 q1 = rec[RF_CAP2 * TT + t];
    if (q1.w == 0.0f) return false;
    if (pstep) {
        const float2 c = pstep_cap(q0.w, q1.x, hmax);
        cb = c.x;
        sb = c.y;
    } else {
        cb = fmaxf(-1.0f, fminf(1.0f, q0.w - hmax * q1.x));
        sb = sqrtf(fmaxf(0.0f, 1.0f - cb * cb));
    }
    return true;
}

// Every triangle into its cell (counters cleared before): the fine grid
// when its cap fits and the cell has room, else the coarse grid under the
// same conditions, else the list; each grid's largest cap radius into the
// header.
__global__ void __launch_bounds__(256) tri_file_kernel(const float4* __restrict__ rec, int T,
                                                       const TileIndexHdr* __restrict__ ihdr, TriIndex ti, int pstep)
{
    uint32_t* __restrict__ cnt = ti.counts;
    const int gt = blockIdx.x * 256 + threadIdx.x;
    unsigned b0 = 0u, b1 = 0u;  // float bits of non-negative radii order as the floats
    if (gt < T) {
        const int t = gt;
        float4 q0;
        float cb, sb;
        if (tri_cap(rec, (size_t)T, t, __uint_as_float((uint32_t)ihdr->h_gen), pstep, q0, cb, sb)) {
            const float beta = acosf(cb);
            const unsigned bb = __float_as_uint(fmaxf(beta, 1e-30f));  // nonzero: the grid holds a triangle
            uint32_t e = 0xffffffffu;
            if (beta <= 2.0f * TRI_CELL1) {
                const float lat = asinf(fmaxf(-1.0f, fminf(1.0f, q0.y)));
                const float lon = atan2f(q0.x, q0.z);
                if (beta <= 2.0f * TRI_CELL0) {
                    const int cell = tri_row(lat, TRI_NLAT0, TRI_CELL0) * TRI_NLON0 + tri_col(lon, TRI_NLON0, TRI_CELL0);
                    const uint32_t k = atomicAdd(&cnt[cell], 1u);
                    if (k < (uint32_t)TRI_K0) {
                        e = (uint32_t)cell * TRI_K0 + k;
                        b0 = bb;
                    }
                }
                if (e == 0xffffffffu) {
                    const int cell = tri_row(lat, TRI_NLAT1, TRI_CELL1) * TRI_NLON1 + tri_col(lon, TRI_NLON1, TRI_CELL1);
                    const uint32_t k = atomicAdd(&cnt[TRI_CELLS0 + cell], 1u);
                    if (k < (uint32_t)TRI_K1) {
                        e = TRI_E1 + (uint32_t)cell * TRI_K1 + k;
                        b1 = bb;
                    }
                }
            }
            if (e == 0xffffffffu) {
                // (below the list's capacity unless an earlier binning left its counters behind)
                const uint32_t k = atomicAdd(&cnt[TRI_LARGE], 1u);
                if (k < (uint32_t)ti.T) e = TRI_E2 + k;
            }
            if (e != 0xffffffffu) {
                ti.cap[e] = make_float4(q0.x, q0.y, q0.z, cb);
                ti.cs[e] = make_float2(sb, __uint_as_float((uint32_t)t));
            }
        }
    }
    for (int o = 16; o; o >>= 1) {
        b0 = max(b0, __shfl_xor_sync(0xffffffffu, b0, o));
        b1 = max(b1, __shfl_xor_sync(0xffffffffu, b1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (b0) atomicMax(&cnt[TRI_HDR], b0);
        if (b1) atomicMax(&cnt[TRI_HDR + 1], b1);
    }
}

// A window of one grid: rows r0 .. r0 + nr - 1, columns c0 .. c0 + ncol - 1
// (mod nlon).
struct TriWin {
    int r0, nr, c0, ncol;
};

// The cells holding every direction within gamma of (lat, lon).
__device__ __forceinline__ TriWin tri_window(float lat, float lon, float gamma, int nlat, float cell)
{
    const int nlon = 2 * nlat;
    TriWin w{0, nlat, 0, nlon};
    if (!(gamma < PI_F)) return w;
    const int r0 = tri_row(lat - gamma, nlat, cell), r1 = tri_row(lat + gamma, nlat, cell);
    w.r0 = r0;
    w.nr = r1 - r0 + 1;
    if (fabsf(lat) + gamma < 0.5f * PI_F - 1e-3f) {
        // longitude half-width of a cap that holds no pole
        const float dl = asinf(fminf(1.0f, sinf(gamma) / cosf(lat))) + 1e-4f;
        int c0 = (int)floorf((lon - dl + PI_F) / cell);
        const int c1 = (int)floorf((lon + dl + PI_F) / cell);
        w.ncol = max(1, min(nlon, c1 - c0 + 1));
        c0 %= nlon;
        if (c0 < 0) c0 += nlon;
        w.c0 = c0;
    }
    return w;
}

__device__ __forceinline__ TriWin shfl_win(const TriWin& w, int src)
{
    return TriWin{__shfl_sync(0xffffffffu, w.r0, src), __shfl_sync(0xffffffffu, w.nr, src),
                  __shfl_sync(0xffffffffu, w.c0, src), __shfl_sync(0xffffffffu, w.ncol, src)};
}

// The candidate triangles of one tile, as one warp sees them: the cells of
// the tile's two windows and the list, one range of sorted entries each.
struct TileWalk {
    float ax, ay, az, ca, sa;  // the tile's cone
    TriWin w0, w1;             // its windows on the fine and coarse grid
    int R0, R1, R;             // ranges: fine cells, coarse cells, then the list (none for an empty tile)

    // every lane of the warp, the same tile
    __device__ __forceinline__ void init(const float4& g, const Cone& c, const uint32_t* __restrict__ hdr, int lane)
    {
        ax = c.c0.x;
        ay = c.c0.y;
        az = c.c0.z;
        ca = c.c0.w;
        sa = c.c1.x;
        TriWin w{0, 0, 0, 1};
        R = 0;
        if (g.w >= 0.0f) {  // h < 0: an empty tile
            // lane 0 forms the fine grid's window, lane 1 the coarse grid's
            // (none for a grid that holds no triangle)
            const unsigned bm = lane < 2 ? hdr[lane] : 0u;
            if (bm)
                w = tri_window(g.y, g.z, g.x + __uint_as_float(bm) + 2e-4f, lane ? TRI_NLAT1 : TRI_NLAT0,
                               lane ? TRI_CELL1 : TRI_CELL0);
        }
        w0 = shfl_win(w, 0);
        w1 = shfl_win(w, 1);
        R0 = w0.nr * w0.ncol;
        R1 = w1.nr * w1.ncol;
        R = g.w >= 0.0f ? R0 + R1 + 1 : 0;
    }

    // range i < R: first entry and length
    __device__ __forceinline__ void range(const uint32_t* __restrict__ cnt, uint32_t listcap, int i, uint32_t& a,
                                          int& len) const
    {
        if (i < R0) {
            const int row = w0.r0 + i / w0.ncol;
            int col = w0.c0 + i % w0.ncol;
            if (col >= TRI_NLON0) col -= TRI_NLON0;
            const int cell = row * TRI_NLON0 + col;
            a = (uint32_t)cell * TRI_K0;
            len = (int)min(cnt[cell], (uint32_t)TRI_K0);
        } else if (i < R0 + R1) {
            const int j = i - R0;
            const int row = w1.r0 + j / w1.ncol;
            int col = w1.c0 + j % w1.ncol;
            if (col >= TRI_NLON1) col -= TRI_NLON1;
            const int cell = row * TRI_NLON1 + col;
            a = TRI_E1 + (uint32_t)cell * TRI_K1;
            len = (int)min(cnt[TRI_CELLS0 + cell], (uint32_t)TRI_K1);
        } else {
            a = TRI_E2;
            len = (int)min(cnt[TRI_LARGE], listcap);
        }
    }

    // entries of all ranges (every lane gets the sum)
    __device__ __forceinline__ uint32_t entries(const uint32_t* __restrict__ cnt, uint32_t listcap, int lane) const
    {
        uint32_t e = 0;
        for (int rb = 0; rb < R; rb += 32) {
            uint32_t a = 0;
            int len = 0;
            if (rb + lane < R) range(cnt, listcap, rb + lane, a, len);
            e += (uint32_t)len;
        }
        for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        return e;
    }

    // The walk, shared by nwarps warps (this one is number wr): the ranges go
    // one per lane, 32 at a time; their entries are numbered across the warp
    // and every lane tests the next one each step, finding the range that
    // holds it by a search over the lanes; the warps take the steps in turn,
    // BIN_WALK_U steps' loads at a time.  sink(hit mask, hit, triangle, this
    // warp's hits before the step) for every step with a hit, on all lanes;
    // returns this warp's hits.
    template <class Sink>
    __device__ __forceinline__ uint32_t walk(const TriIndex& ti, int lane, int wr, int nwarps, Sink sink) const
    {
        const unsigned FULL = 0xffffffffu;
        uint32_t hits = 0;
        for (int rb = 0; rb < R; rb += 32) {
            uint32_t a = 0;
            int len = 0;
            if (rb + lane < R) range(ti.counts, (uint32_t)ti.T, rb + lane, a, len);
            int incl = len;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const int excl = incl - len;
            for (int k0 = 32 * BIN_WALK_U * wr; k0 < total; k0 += 32 * BIN_WALK_U * nwarps) {
                float4 q[BIN_WALK_U];
                float2 r[BIN_WALK_U];
                bool in[BIN_WALK_U];
#pragma unroll
                for (int u = 0; u < BIN_WALK_U; ++u) {
                    const int idx = k0 + 32 * u + lane;
                    int o = 0;  // the last lane whose range starts at or before entry idx
                    for (int st = 16; st > 0; st >>= 1) {
                        const int x = __shfl_sync(FULL, excl, o + st);
                        if (x <= idx) o += st;
                    }
                    const uint32_t e = __shfl_sync(FULL, a, o) + (uint32_t)(idx - __shfl_sync(FULL, excl, o));
                    in[u] = idx < total;
                    if (in[u]) {
                        q[u] = ti.cap[e];
                        r[u] = ti.cs[e];
                    }
                }
#pragma unroll
                for (int u = 0; u < BIN_WALK_U; ++u) {
                    bool hit = false;
                    if (in[u]) {
                        // the cap / cone test of the triangle-major search, operand for operand
                        const float cg = fmaf(q[u].x, ax, fmaf(q[u].y, ay, q[u].z * az));
                        hit = q[u].w + ca <= 2e-6f || cg >= fmaf(ca, q[u].w, -sa * r[u].x) - 2e-6f;
                    }
                    const unsigned m = __ballot_sync(FULL, hit);
                    if (m) sink(m, hit, __float_as_uint(r[u].y), hits);
                    hits += (uint32_t)__popc(m);
                }
            }
        }
        return hits;
    }
};

// The tiles, one warp each (a resident grid: warp w of W takes tiles w,
// w + W, ...).  A tile whose ranges hold at most
// BIN_STAGE_HITS entries is binned here: its hits staged in shared memory,
// its range of the bins taken with one atomic on the cursor.  A larger tile
// goes to the heavy list for bin_heavy_kernel.  With no heavy tile the last
// CTA to finish stores the total.
__global__ void __launch_bounds__(128, VSR_BIN_TILES_CTAS) bin_tiles_kernel(const float4* __restrict__ geom,
                                                                            const Cone* __restrict__ tiles,
                                                                            int ntiles, TriIndex ti,
                                                                            uint32_t* __restrict__ starts,
                                                                            uint32_t* __restrict__ ends,
                                                                            uint32_t* __restrict__ ids, uint32_t cap,
                                                                            int* status, uint32_t* total_host)
{
    __shared__ uint32_t s_hit[4][BIN_STAGE_HITS];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* hdr = ti.counts + TRI_HDR;
    const uint32_t lt = (1u << lane) - 1u;
    for (int tile = blockIdx.x * 4 + warp; tile < ntiles; tile += gridDim.x * 4) {
        const float4 g = geom[tile];
        TileWalk tw;
        tw.init(g, g.w >= 0.0f ? tiles[tile] : Cone{}, hdr, lane);
        const uint32_t E = tw.entries(ti.counts, (uint32_t)ti.T, lane);
        if (E <= BIN_STAGE_HITS) {
            uint32_t* __restrict__ stage = s_hit[warp];
            const uint32_t n = tw.walk(ti, lane, 0, 1, [&](unsigned m, bool hit, uint32_t t, uint32_t before) {
                if (hit) stage[before + (uint32_t)__popc(m & lt)] = t;
            });
            uint32_t start = 0;
            if (lane == 0 && n) start = atomicAdd(&hdr[TRI_H_CURSOR], n);
            start = __shfl_sync(FULL, start, 0);
            __syncwarp();
            if (lane == 0 && (uint64_t)start + n > cap) raise_status(status, VSR_ERR_BIN_OVERFLOW);
            for (uint32_t j = lane; j < n; j += 32)
                if (start + j < cap) ids[start + j] = stage[j];
            __syncwarp();  // the stage is read before the next tile's hits
            if (lane == 0) {
                starts[tile] = start;
                ends[tile] = start + n;
            }
        } else if (lane == 0) {
            const uint32_t j = atomicAdd(&hdr[TRI_H_HEAVY], 1u);
            if (j < (uint32_t)ntiles) ti.heavy[j] = (uint32_t)tile;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&hdr[TRI_H_DONE], 1u) == gridDim.x - 1) {
            __threadfence();
            if (atomicAdd(&hdr[TRI_H_HEAVY], 0u) == 0u) {
                const uint32_t total = atomicAdd(&hdr[TRI_H_CURSOR], 0u);
                starts[ntiles] = total;
                if (total_host) {  // straight into the host's pinned word (read after an event)
                    *total_host = total;
                    __threadfence_system();
                }
            }
        }
    }
}

// The heavy tiles, one CTA of BIN_HEAVY_WARPS warps each, the CTAs taking
// the next tile of the list until none is left (a grid of resident CTAs;
// nothing waits).  The warps take the walk's steps in turn: a first walk
// counts the tile's hits, one atomic takes its range of the bins, a second
// walk writes them, each step's hits taking their places from a
// shared-memory counter.  The last CTA to finish stores the total (when the
// tile pass left it to this one) and clears the counters and the header for
// the next binning.
__global__ void __launch_bounds__(32 * BIN_HEAVY_WARPS) bin_heavy_kernel(const float4* __restrict__ geom,
                                                                        const Cone* __restrict__ tiles, int ntiles,
                                                                        TriIndex ti, uint32_t* __restrict__ starts,
                                                                        uint32_t* __restrict__ ends,
                                                                        uint32_t* __restrict__ ids, uint32_t cap,
                                                                        int* status, uint32_t* total_host)
{
    __shared__ uint32_t s_tile, s_n, s_start;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* hdr = ti.counts + TRI_HDR;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t nheavy = min(hdr[TRI_H_HEAVY], (uint32_t)ntiles);
    if (!nheavy) {
        // nothing reads the cell counters any more: each CTA clears a slice
        uint4* c4 = reinterpret_cast<uint4*>(ti.counts);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < TRI_HDR / 4; i += gridDim.x * blockDim.x)
            c4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (; nheavy;) {
        __syncthreads();  // the previous tile's counter is read
        if (threadIdx.x == 0) {
            const uint32_t j = atomicAdd(&hdr[TRI_H_NEXT], 1u);
            s_tile = j < nheavy ? ti.heavy[j] : 0xffffffffu;
            s_n = 0u;
        }
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= (uint32_t)ntiles) break;
        const float4 g = geom[tile];
        TileWalk tw;
        tw.init(g, tiles[tile], hdr, lane);
        const uint32_t mine = tw.walk(ti, lane, warp, BIN_HEAVY_WARPS, [](unsigned, bool, uint32_t, uint32_t) {});
        if (lane == 0 && mine) atomicAdd(&s_n, mine);
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t n = s_n;
            const uint32_t start = n ? atomicAdd(&hdr[TRI_H_CURSOR], n) : 0u;
            if ((uint64_t)start + n > cap) raise_status(status, VSR_ERR_BIN_OVERFLOW);
            starts[tile] = start;
            ends[tile] = start + n;
            s_start = start;
            s_n = 0u;
        }
        __syncthreads();
        const uint32_t start = s_start;
        tw.walk(ti, lane, warp, BIN_HEAVY_WARPS, [&](unsigned m, bool hit, uint32_t t, uint32_t) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&s_n, (uint32_t)__popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (hit) {
                const uint32_t pos = start + base + (uint32_t)__popc(m & lt);
                if (pos < cap) ids[pos] = t;
            }
        });
    }
    // the last CTA to finish (every tile's range is taken by then: the tile
    // pass ran before, and each CTA's own before this)
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&hdr[TRI_H_DONE2], 1u) == gridDim.x - 1;
        if (s_last && nheavy) {
            __threadfence();
            const uint32_t total = atomicAdd(&hdr[TRI_H_CURSOR], 0u);
            starts[ntiles] = total;
            if (total_host) {  // straight into the host's pinned word (read after an event)
                *total_host = total;
                __threadfence_system();
            }
        }
    }
    __syncthreads();
    if (s_last) {
        // nothing reads the counters any more: clear the rest of them (all,
        // after heavy tiles) and the header
        const int from = nheavy ? 0 : TRI_HDR / 4;
        uint4* c4 = reinterpret_cast<uint4*>(ti.counts);
        for (int i = from + threadIdx.x; i < TRI_WORDS / 4; i += blockDim.x) c4[i] = make_uint4(0u, 0u, 0u, 0u);
        if (threadIdx.x < TRI_WORDS % 4) ti.counts[(TRI_WORDS / 4) * 4 + threadIdx.x] = 0u;
    }
}

}  // namespace

vsr_status launch_scan(const uint32_t* counts, const uint32_t* extra, int n, const int* n_dev, uint32_t* offsets,
                       cudaStream_t st, uint32_t* total_host)
{
    scan_kernel<<<1, 1024, 0, st>>>(counts, extra, n, n_dev, offsets, total_host);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status tri_index_alloc(TriIndex* ti, int64_t T, int ntiles)
{
    if (!ti->counts) {
        VSR_CUDA_TRY(cudaMalloc(&ti->counts, sizeof(uint32_t) * TRI_WORDS));
        ti->dirty = true;  // cleared by the first binning
    }
    if (!ti->heavy || ntiles > ti->ntiles) {
        cudaFree(ti->heavy);
        ti->heavy = nullptr;
        ti->ntiles = 0;
        VSR_CUDA_TRY(cudaMalloc(&ti->heavy, sizeof(uint32_t) * (size_t)(ntiles > 0 ? ntiles : 1)));
        ti->ntiles = ntiles;
    }
    if (!ti->cap || T > ti->T) {
        cudaFree(ti->cap);
        cudaFree(ti->cs);
        ti->cap = nullptr;
        ti->cs = nullptr;
        ti->T = 0;
        const size_t n = (size_t)TRI_E2 + (size_t)T;
        VSR_CUDA_TRY(cudaMalloc(&ti->cap, sizeof(float4) * n));
        VSR_CUDA_TRY(cudaMalloc(&ti->cs, sizeof(float2) * n));
        ti->T = T;
    }
    return VSR_OK;
}

void tri_index_free(TriIndex* ti)
{
    cudaFree(ti->counts);
    cudaFree(ti->heavy);
    cudaFree(ti->cap);
    cudaFree(ti->cs);
    *ti = TriIndex{};
}

size_t tri_index_bytes(int64_t T, int ntiles)
{
    return sizeof(uint32_t) * ((size_t)TRI_WORDS + (size_t)ntiles) +
           (sizeof(float4) + sizeof(float2)) * ((size_t)TRI_E2 + (size_t)T);
}

vsr_status launch_bin_tiles(const float4* rec, int T, const TileIndex& idx, const Cone* tiles, int ntiles,
                            TriIndex& ti, uint32_t* starts, uint32_t* ends, uint32_t* ids, uint32_t cap, int* status,
                            uint32_t* total_host, cudaStream_t st, int pstep)
{
    if (T < 0 || (int64_t)T > ti.T || !ti.counts || !ti.cap || ntiles <= 0 || ntiles > ti.ntiles)
        return VSR_ERR_INVALID_ARG;
    // until the clearing kernel is queued, a failure leaves the counters behind
    const bool was_dirty = ti.dirty;
    ti.dirty = true;
    if (was_dirty) VSR_CUDA_TRY(cudaMemsetAsync(ti.counts, 0, sizeof(uint32_t) * TRI_WORDS, st));
    if (T > 0) {
        tri_file_kernel<<<(T + 255) / 256, 256, 0, st>>>(rec, T, idx.hdr, ti, pstep);
        VSR_CUDA_TRY(cudaGetLastError());
    }
    const int sms = sm_count();
    if (sms < 0) return VSR_ERR_CUDA;
    // one resident wave (the tile pass's occupancy, looked up once)
    static std::atomic<int> per_sm{0};
    int k = per_sm.load();
    if (k <= 0) {
        VSR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, bin_tiles_kernel, 128, 0));
        if (k <= 0) k = 1;
        per_sm.store(k);
    }
    const int grid = std::min((ntiles + 3) / 4, k * sms);
    bin_tiles_kernel<<<grid, 128, 0, st>>>(idx.geom, tiles, ntiles, ti, starts, ends, ids, cap, status, total_host);
    VSR_CUDA_TRY(cudaGetLastError());
    bin_heavy_kernel<<<sms, 32 * BIN_HEAVY_WARPS, 0, st>>>(idx.geom, tiles, ntiles, ti, starts, ends, ids, cap, status,
                                                           total_host);
    VSR_CUDA_TRY(cudaGetLastError());
    ti.dirty = false;
    return VSR_OK;
}

vsr_status launch_tile_index(const Cone* tiles, int ntiles, TileIndex idx, cudaStream_t st)
{
    if (ntiles < 0 || ntiles > IDX_FUSED_TILES) return VSR_ERR_INVALID_ARG;
    // the shared-memory opt-in of the kernel, once per device
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    VSR_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        VSR_CUDA_TRY(cudaFuncSetAttribute(idx_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)IDX_FUSED_SMEM));
        attr_set.fetch_or(bit);
    }
    idx_fused_kernel<<<1, IDX_FUSED_THREADS, IDX_FUSED_SMEM, st>>>(tiles, idx.geom, ntiles, idx.hdr, idx.cell_start,
                                                                    idx.sorted, idx.big);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    const int slot = dev & 63;
    int n = cache[slot].load();
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return -1;
    cache[slot].store(n);
    return n;
}

// The binner's launch shape for T triangles on `sms` SMs: 0 = one cone per
// step and VSR_BIN_TPW_LARGE triangles per warp (grids beyond one resident wave at 7 CTAs
// per SM), 1 = four cones per step, 2 = four cones and 8 triangles per warp
// (scenes whose 8-per-warp grid still fits that wave).
static int bin_shape(int T, int sms)
{
    if ((T + 127) / 128 > 7 * sms) return 0;
    if ((T + 31) / 32 <= 7 * sms) return 2;
    return 1;
}

vsr_status launch_bin_count(const float4* rec, int T, TileIndex idx, uint32_t* counts, uint32_t* cursor,
                            uint2* pairs, uint32_t pair_cap, cudaStream_t st, int pstep)
{
    if (T == 0) return VSR_OK;
    const BinView v{idx.hdr,  idx.cell_start, idx.sorted, idx.big, rec,   counts,
                    nullptr,  pairs,          pair_cap,   cursor,  pstep, idx.ntiles};
    const int sms = sm_count();
    if (sms < 0) return VSR_ERR_CUDA;
    switch (bin_shape(T, sms)) {
    case 0:
        bin_kernel<false, VSR_BIN_CB_LARGE, VSR_BIN_TPW_LARGE>
            <<<(T + 4 * VSR_BIN_TPW_LARGE - 1) / (4 * VSR_BIN_TPW_LARGE), 128, 0, st>>>(v, T, nullptr, 0, nullptr);
        break;
    case 1: bin_kernel<false, 4, 32><<<(T + 127) / 128, 128, 0, st>>>(v, T, nullptr, 0, nullptr); break;
    default: bin_kernel<false, 4, 8><<<(T + 31) / 32, 128, 0, st>>>(v, T, nullptr, 0, nullptr); break;
    }
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_bin_fill(const float4* rec, int T, TileIndex idx, const uint32_t* offsets, uint32_t* counts,
                           const uint32_t* cursor, const uint2* pairs, uint32_t pair_cap, uint32_t* ids, uint32_t cap,
                           int* status, cudaStream_t st, int pstep)
{
    if (T == 0) return VSR_OK;
    const BinView v{idx.hdr, idx.cell_start, idx.sorted, idx.big, rec, counts, offsets, const_cast<uint2*>(pairs),
                    pair_cap, const_cast<uint32_t*>(cursor), pstep, idx.ntiles};
    // a pair list as long as the bins is complete unless the bins overflow,
    // so the search-based fill is needed only without one or with a shorter one
    const bool search = !pairs || pair_cap < cap;
    if (pairs) {
        constexpr int BIN_PAIR_BLOCKS = 152 * 8;
        bin_pairs_kernel<<<BIN_PAIR_BLOCKS, 256, 0, st>>>(pairs, cursor, pair_cap, offsets, counts, ids, cap,
                                                          status, search ? 0 : 1);
        VSR_CUDA_TRY(cudaGetLastError());
    }
    if (!search) return VSR_OK;
    const int sms = sm_count();
    if (sms < 0) return VSR_ERR_CUDA;
    switch (bin_shape(T, sms)) {
    case 0:
        bin_kernel<true, VSR_BIN_CB_LARGE, VSR_BIN_TPW_LARGE>
            <<<(T + 4 * VSR_BIN_TPW_LARGE - 1) / (4 * VSR_BIN_TPW_LARGE), 128, 0, st>>>(v, T, ids, cap, status);
        break;
    case 1: bin_kernel<true, 4, 32><<<(T + 127) / 128, 128, 0, st>>>(v, T, ids, cap, status); break;
    default: bin_kernel<true, 4, 8><<<(T + 31) / 32, 128, 0, st>>>(v, T, ids, cap, status); break;
    }
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

// ---- large exclusive scan (multi-CTA) ---------------------------------------
// pass 1: per 4096-element block sums; pass 2: one CTA scans the block sums
// (partials[nb] = total); pass 3: per block, local scan plus the block's base.

__global__ void __launch_bounds__(1024) scan_block_sums(const uint32_t* __restrict__ counts,
                                                         const uint32_t* __restrict__ extra, int n,
                                                         uint32_t* __restrict__ partials)
{
    __shared__ uint32_t ws[32];
    const int b = blockIdx.x * 4096 + 4 * threadIdx.x;
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (b + q < n) v += counts[b + q] + (extra ? extra[b + q] : 0u);
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = ws[threadIdx.x];
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = w;
    }
}

__global__ void __launch_bounds__(1024) scan_blocks_apply(const uint32_t* __restrict__ counts,
                                                           const uint32_t* __restrict__ extra, int n,
                                                           const uint32_t* __restrict__ bases,
                                                           uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x * 4096 + 4 * tid;
    uint32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = b + q < n ? counts[b + q] + (extra ? extra[b + q] : 0u) : 0u;
    const uint32_t local = v[0] + v[1] + v[2] + v[3];
    uint32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t run = bases[blockIdx.x] + x - local + (warp > 0 ? warp_sums[warp - 1] : 0u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (b + q < n) offsets[b + q] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0) offsets[n] = bases[gridDim.x];
}

vsr_status launch_scan_large(const uint32_t* counts, const uint32_t* extra, int n, uint32_t* partials,
                             uint32_t* offsets, cudaStream_t st)
{
    const int nb = (n + 4095) / 4096;
    if (nb <= 1) return launch_scan(counts, extra, n, nullptr, offsets, st);
    scan_block_sums<<<nb, 1024, 0, st>>>(counts, extra, n, partials);
    // scan the nb block sums in place into partials[nb + 1 ...]: reuse the one-CTA scan
    vsr_status s = launch_scan(partials, nullptr, nb, nullptr, partials + nb + 1, st);
    if (s != VSR_OK) return s;
    scan_blocks_apply<<<nb, 1024, 0, st>>>(counts, extra, n, partials + nb + 1, offsets);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}
