// bin.cu -- tile binning: which triangles may produce a fragment in which
// 16x16 tile.
//
// A fragment of triangle t at pixel direction G needs G inside the miter
// cap enlarged by the ramp half-width (the gbpxstep test of the miter plane,
// Sec. 1.1.1 / 1.1.2): G.S-hat - cos rho > -h sin rho, h = 1/(2 delta).  The
// binner keeps (tile, t) when that enlarged cap can reach the tile's view
// cone (cap_hits_cone).  The paper's analogue is the low-resolution region
// mask widened by fwidth/2 (getPolygonRegion).
//
// The candidate tiles of a triangle come from the map's tile index (a
// latitude-longitude grid of the view sphere in which every tile is filed
// once, see TileIndexHdr): only the cells within beta + alpha_small_max of
// the cap centre are visited, so the work per triangle is a few dozen cone
// tests whatever the map's size, and no tile is found twice.
//
// Per frame: count (one thread per triangle, atomic per-tile counters) ->
// exclusive scan -> fill (atomic per-tile cursors).  The order of ids inside
// a bin is not fixed; the raster kernel's result does not depend on it.
#include <math.h>

#include "vsr_internal.cuh"

namespace {

constexpr float PI_F = 3.14159265358979f;

__device__ __forceinline__ int hist_bin(float a)
{
    // third-of-an-octave bins from 2^-17 rad
    int b = (int)floorf((log2f(fmaxf(a, 1e-30f)) + 17.0f) * 3.0f);
    return min(IDX_HIST - 1, max(0, b));
}

__device__ __forceinline__ float hist_upper(int b) { return exp2f((float)(b + 1) / 3.0f - 17.0f); }

__device__ __forceinline__ float cone_half_angle(const Cone& c) { return acosf(fmaxf(-1.0f, fminf(1.0f, c.c0.w))); }

__device__ __forceinline__ int cell_row(float lat, const TileIndexHdr& h)
{
    return min(h.nlat - 1, max(0, (int)floorf((lat + 0.5f * PI_F) / h.cell)));
}

__device__ __forceinline__ int cell_col(float lon, const TileIndexHdr& h)
{
    int c = (int)floorf((lon + PI_F) / h.cell);
    c %= h.nlon;
    return c < 0 ? c + h.nlon : c;
}

__device__ __forceinline__ int home_cell(float3 a, const TileIndexHdr& h)
{
    float lat = asinf(fmaxf(-1.0f, fminf(1.0f, a.y)));
    float lon = atan2f(a.x, a.z);
    return cell_row(lat, h) * h.nlon + cell_col(lon, h);
}

// ---- tile index -------------------------------------------------------------
//
// One CTA of IDX_THREADS threads builds the whole index: the histogram of
// tile half-angles and the grid plan, the per-cell counts (in shared
// memory), their exclusive scan, and the cell-sorted cone copies.  A tile
// index holds one entry per tile, so a single CTA keeps every phase a few
// loads per thread and saves the launch gaps of separate kernels.

constexpr int IDX_THREADS = 1024;

__device__ __forceinline__ Cone index_entry(const Cone& c, int i)
{
    Cone e;
    e.c0 = c.c0;
    e.c1 = make_float4(c.c1.x, c.c1.y, __uint_as_float((uint32_t)i), 0.0f);
    return e;
}

__global__ void __launch_bounds__(IDX_THREADS) idx_build_kernel(const Cone* __restrict__ tiles, int ntiles,
                                                                 TileIndexHdr* __restrict__ hdr,
                                                                 uint32_t* __restrict__ cell_start,
                                                                 Cone* __restrict__ sorted, Cone* __restrict__ big)
{
    extern __shared__ uint32_t s_cell[];  // IDX_CELLS_MAX counts, then cursors
    __shared__ unsigned s_hist[IDX_HIST];
    __shared__ unsigned s_nvalid, s_hmax, s_amax, s_nbig;
    __shared__ TileIndexHdr s_h;
    __shared__ uint32_t s_warp[IDX_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int q = tid; q < IDX_CELLS_MAX; q += IDX_THREADS) s_cell[q] = 0u;
    if (tid < IDX_HIST) s_hist[tid] = 0u;
    if (tid == 0) s_nvalid = s_hmax = s_amax = s_nbig = 0u;
    __syncthreads();

    // histogram of half-angles, widest ramp
    for (int i = tid; i < ntiles; i += IDX_THREADS) {
        const Cone c = tiles[i];
        if (c.c1.z == 0.0f) continue;
        atomicAdd(&s_hist[hist_bin(cone_half_angle(c))], 1u);
        atomicAdd(&s_nvalid, 1u);
        atomicMax(&s_hmax, __float_as_uint(c.c1.y));  // non-negative floats order as their bits
    }
    __syncthreads();

    // grid size and small / big threshold from the 99th percentile
    if (tid == 0) {
        unsigned target = (unsigned)ceilf(0.99f * (float)s_nvalid), run = 0;
        int b = 0;
        for (; b < IDX_HIST; ++b) {
            run += s_hist[b];
            if (run >= target) break;
        }
        const float cut = hist_upper(min(b, IDX_HIST - 1));
        const float cell = fminf(PI_F / 8.0f, fmaxf(PI_F / IDX_NLAT_MAX, cut));
        const int nlat = min(IDX_NLAT_MAX, (int)ceilf(PI_F / cell));
        s_h.nlat = nlat;
        s_h.nlon = 2 * nlat;
        s_h.ncell = 2 * nlat * nlat;
        s_h.cell = PI_F / nlat;
        s_h.alpha_cut = cut;
    }
    __syncthreads();
    const TileIndexHdr h = s_h;

    // per-cell counts of the small tiles; big tiles to their own list
    for (int i = tid; i < ntiles; i += IDX_THREADS) {
        const Cone c = tiles[i];
        if (c.c1.z == 0.0f) continue;
        const float a = cone_half_angle(c);
        if (a > h.alpha_cut) {
            big[atomicAdd(&s_nbig, 1u)] = index_entry(c, i);
        } else {
            atomicAdd(&s_cell[home_cell(make_float3(c.c0.x, c.c0.y, c.c0.z), h)], 1u);
            atomicMax(&s_amax, __float_as_uint(a));
        }
    }
    __syncthreads();

    // exclusive scan of the cell counts (contiguous segment per thread)
    const int per = (h.ncell + IDX_THREADS - 1) / IDX_THREADS;
    const int b0 = min(h.ncell, tid * per), b1 = min(h.ncell, b0 + per);
    uint32_t local = 0;
    for (int q = b0; q < b1; ++q) local += s_cell[q];
    uint32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    uint32_t run = x - local + (warp > 0 ? s_warp[warp - 1] : 0u);
    for (int q = b0; q < b1; ++q) {
        const uint32_t cnt = s_cell[q];
        cell_start[q] = run;
        s_cell[q] = run;  // becomes the fill cursor
        run += cnt;
    }
    if (tid == IDX_THREADS - 1) cell_start[h.ncell] = s_warp[31];
    __syncthreads();

    // cell-sorted copies of the small tiles' cones
    for (int i = tid; i < ntiles; i += IDX_THREADS) {
        const Cone c = tiles[i];
        if (c.c1.z == 0.0f || cone_half_angle(c) > h.alpha_cut) continue;
        sorted[atomicAdd(&s_cell[home_cell(make_float3(c.c0.x, c.c0.y, c.c0.z), h)], 1u)] = index_entry(c, i);
    }
    if (tid == 0) {
        TileIndexHdr o = h;
        o.alpha_small_max = s_amax;
        o.h_max = s_hmax;
        o.n_big = s_nbig;
        o.n_valid = s_nvalid;
        for (int q = 0; q < IDX_HIST; ++q) o.hist[q] = s_hist[q];
        *hdr = o;
    }
}

// ---- per-triangle binning ---------------------------------------------------

// One thread per triangle of the view v.
template <bool FILL>
__global__ void __launch_bounds__(128) bin_kernel(BinView v, int T, uint32_t* __restrict__ ids, uint32_t cap,
                                                   int* status)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const float4* __restrict__ rec = v.rec;
    const TileIndexHdr* __restrict__ hdr = v.hdr;
    const uint32_t* __restrict__ cell_start = v.cell_start;
    const Cone* __restrict__ sorted = v.sorted;
    const Cone* __restrict__ big = v.big;
    uint32_t* __restrict__ counts = v.counts;
    uint32_t* __restrict__ extra = v.extra;
    uint32_t* __restrict__ hits = v.hits;
    const uint32_t* __restrict__ offsets = v.offsets;
    const size_t TT = (size_t)T;
    uint32_t* my_hits = hits + (size_t)t * BIN_HIT_WORDS;
    uint32_t nhit = 0;

    auto put = [&](uint32_t tile, uint32_t pos) {
        if (pos < cap && pos < offsets[tile + 1])
            ids[pos] = (uint32_t)t;
        else
            raise_status(status, VSR_ERR_BIN_OVERFLOW);
    };

    if (FILL) {
        // the count pass recorded (tile, slot) for up to BIN_HIT_CACHE hits
        const uint32_t n = my_hits[0];
        const uint32_t nc = min(n, (uint32_t)BIN_HIT_CACHE);
        for (uint32_t q = 0; q < nc; ++q) {
            const uint32_t tile = my_hits[1 + 2 * q];
            put(tile, offsets[tile] + my_hits[2 + 2 * q]);
        }
        if (n <= BIN_HIT_CACHE) return;
    }

    // count: the first BIN_HIT_CACHE hits take a slot in `counts`, the rest
    // are counted in `extra`.  fill (only for triangles with more hits):
    // search again, skip the cached hits, place the others after the slotted
    // ones of their tile.
    auto emit = [&](uint32_t tile) {
        if (!FILL) {
            if (nhit < BIN_HIT_CACHE) {
                my_hits[1 + 2 * nhit] = tile;
                my_hits[2 + 2 * nhit] = atomicAdd(&counts[tile], 1u);
            } else {
                atomicAdd(&extra[tile], 1u);
            }
        } else if (nhit >= BIN_HIT_CACHE) {
            put(tile, offsets[tile] + counts[tile] + atomicSub(&extra[tile], 1u) - 1u);
        }
        ++nhit;
    };

    const float4 c0 = rec[RF_CAP * TT + t];
    const float4 c1 = rec[RF_CAP2 * TT + t];
    if (c1.w == 0.0f) {  // culled
        if (!FILL) my_hits[0] = 0;
        return;
    }
    const float3 S = make_float3(c0.x, c0.y, c0.z);
    const float cr = c0.w, sr = c1.x;
    const TileIndexHdr& h = *hdr;
    const int nlat = h.nlat, nlon = h.nlon;
    const float cell = h.cell;
    const float amax = __uint_as_float(h.alpha_small_max), hmax = __uint_as_float(h.h_max);

    // the cap enlarged once by the map's widest ramp (>= every tile's own):
    // cos / sin of its radius beta, so each tile test is a few FMAs
    const float cb = fmaxf(-1.0f, fminf(1.0f, cr - hmax * sr));
    const float sb = sqrtf(fmaxf(0.0f, 1.0f - cb * cb));
    auto scan_range = [&](const Cone* __restrict__ list, uint32_t k0, uint32_t k1) {
        for (uint32_t k = k0; k < k1; ++k) {
            const Cone c = list[k];
            // angle(S, axis) <= alpha + beta  (always when alpha + beta >= pi)
            const float cg = fmaf(S.x, c.c0.x, fmaf(S.y, c.c0.y, S.z * c.c0.z));
            if (cb + c.c0.w <= 2e-6f || cg >= fmaf(c.c0.w, cb, -c.c1.x * sb) - 2e-6f) emit(__float_as_uint(c.c1.z));
        }
    };

    // search radius: enlarged cap + largest small tile
    const float gamma = acosf(cb) + amax + 1e-4f;
    int r0 = 0, r1 = nlat - 1, c0i = 0, ncol = nlon;
    if (gamma < PI_F) {
        const float lat = asinf(fmaxf(-1.0f, fminf(1.0f, S.y)));
        const float lon = atan2f(S.x, S.z);
        r0 = cell_row(lat - gamma, h);
        r1 = cell_row(lat + gamma, h);
        if (fabsf(lat) + gamma < 0.5f * PI_F - 1e-3f) {
            // longitude half-width of a cap that holds no pole
            const float dl = asinf(fminf(1.0f, sinf(gamma) / cosf(lat))) + 1e-4f;
            c0i = (int)floorf((lon - dl + PI_F) / cell);
            const int c1i = (int)floorf((lon + dl + PI_F) / cell);
            ncol = min(nlon, c1i - c0i + 1);
            c0i %= nlon;
            if (c0i < 0) c0i += nlon;
        }
    }
    for (int r = r0; r <= r1; ++r) {
        const uint32_t* row = cell_start + r * nlon;
        if (c0i + ncol <= nlon) {
            scan_range(sorted, row[c0i], row[c0i + ncol]);
        } else {  // the window wraps across longitude +-pi
            scan_range(sorted, row[c0i], row[nlon]);
            scan_range(sorted, row[0], row[c0i + ncol - nlon]);
        }
    }
    scan_range(big, 0, h.n_big);
    if (!FILL) my_hits[0] = nhit;
}

// Exclusive scan of n counts (+ extra, when not NULL) into offsets[0..n] by
// one CTA of 1024 threads:
// chunks of 4096 (four consecutive elements per thread), carried across
// chunks.  n comes from n_dev when it is not NULL.
__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t* __restrict__ counts,
                                                     const uint32_t* __restrict__ extra, int n_host,
                                                     const int* __restrict__ n_dev, uint32_t* __restrict__ offsets)
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
    if (tid == 0) offsets[n] = carry_s;
}

}  // namespace

vsr_status launch_scan(const uint32_t* counts, const uint32_t* extra, int n, const int* n_dev, uint32_t* offsets,
                       cudaStream_t st)
{
    scan_kernel<<<1, 1024, 0, st>>>(counts, extra, n, n_dev, offsets);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_tile_index(const Cone* tiles, int ntiles, TileIndex idx, cudaStream_t st)
{
    const size_t smem = sizeof(uint32_t) * IDX_CELLS_MAX;  // 128 KB of per-cell counts
    VSR_CUDA_TRY(cudaFuncSetAttribute(idx_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    idx_build_kernel<<<1, IDX_THREADS, smem, st>>>(tiles, ntiles, idx.hdr, idx.cell_start, idx.sorted, idx.big);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_bin_count(const float4* rec, int T, TileIndex idx, uint32_t* counts, uint32_t* extra, uint32_t* hits,
                            cudaStream_t st)
{
    if (T == 0) return VSR_OK;
    const BinView v{idx.hdr, idx.cell_start, idx.sorted, idx.big, rec, counts, extra, hits, nullptr};
    bin_kernel<false><<<(T + 127) / 128, 128, 0, st>>>(v, T, nullptr, 0, nullptr);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_bin_fill(const float4* rec, int T, TileIndex idx, const uint32_t* hits, const uint32_t* offsets,
                           uint32_t* counts, uint32_t* extra, uint32_t* ids, uint32_t cap, int* status,
                           cudaStream_t st)
{
    if (T == 0) return VSR_OK;
    const BinView v{idx.hdr, idx.cell_start, idx.sorted, idx.big, rec, counts, extra, const_cast<uint32_t*>(hits),
                    offsets};
    bin_kernel<true><<<(T + 127) / 128, 128, 0, st>>>(v, T, ids, cap, status);
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
