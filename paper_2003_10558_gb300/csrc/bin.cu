// bin.cu -- tile binning: which triangles may produce a fragment in which
// 16x16 tile.
//
// A fragment of triangle t at pixel direction G needs G inside the miter
// cap enlarged by the ramp half-width (the gbpxstep test of the miter plane,
// Sec. 1.1.1/1.1.2): G.S-hat - cos rho > -h sin rho, h = 1/(2 delta).  The
// binner keeps (tile, t) when that enlarged cap can reach the tile's view
// cone (cap_hits_cone), first against 8x8-tile super-tiles, then against
// the tiles of each super-tile that was hit.  The paper's analogue is the
// low-resolution region mask widened by fwidth/2 (getPolygonRegion).
//
// count (one thread per triangle, atomic per-tile counters) -> exclusive
// scan -> fill (atomic per-tile cursors).  The order of ids inside a bin is
// not fixed; the raster kernel's result does not depend on it.
#include "vsr_internal.cuh"

namespace {

template <bool FILL>
__global__ void __launch_bounds__(128) bin_kernel(const float4* __restrict__ rec, int T, const Cone* __restrict__ tiles,
                                                   int tx, int ty, const Cone* __restrict__ supers, int sx, int sy,
                                                   uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets,
                                                   uint32_t* __restrict__ ids, uint32_t cap, int* status)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const size_t TT = (size_t)T;
    float4 c0 = rec[RF_CAP * TT + t];
    float4 c1 = rec[RF_CAP2 * TT + t];
    if (c1.w == 0.0f) return;  // culled
    const float3 S = make_float3(c0.x, c0.y, c0.z);
    const float cr = c0.w, sr = c1.x;
    for (int s = 0; s < sx * sy; ++s) {
        Cone sc = supers[s];
        if (sc.c1.z == 0.0f) continue;
        if (!cap_hits_cone(S, cr, sr, make_float3(sc.c0.x, sc.c0.y, sc.c0.z), sc.c0.w, sc.c1.x, sc.c1.y)) continue;
        int bx = (s % sx) * SUPER, by = (s / sx) * SUPER;
        int ex = min(bx + SUPER, tx), ey = min(by + SUPER, ty);
        for (int y = by; y < ey; ++y)
            for (int x = bx; x < ex; ++x) {
                int tile = y * tx + x;
                Cone c = tiles[tile];
                if (c.c1.z == 0.0f) continue;
                if (!cap_hits_cone(S, cr, sr, make_float3(c.c0.x, c.c0.y, c.c0.z), c.c0.w, c.c1.x, c.c1.y)) continue;
                if (!FILL) {
                    atomicAdd(&counts[tile], 1u);
                } else {
                    uint32_t slot = atomicAdd(&counts[tile], 1u);
                    uint32_t pos = offsets[tile] + slot;
                    if (pos < cap && pos < offsets[tile + 1])
                        ids[pos] = (uint32_t)t;
                    else
                        raise_status(status, VSR_ERR_BIN_OVERFLOW);
                }
            }
    }
}

// Exclusive scan of n counts into offsets[0..n] by one CTA of 1024 threads,
// each owning a contiguous segment.
__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t* __restrict__ counts, int n,
                                                     uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = min(n, tid * per), e = min(n, b + per);
    uint32_t local = 0;
    for (int q = b; q < e; ++q) local += counts[q];
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
    uint32_t run = x - local + (warp > 0 ? warp_sums[warp - 1] : 0u);
    for (int q = b; q < e; ++q) {
        offsets[q] = run;
        run += counts[q];
    }
    if (tid == blockDim.x - 1) offsets[n] = warp_sums[31];
}

}  // namespace

vsr_status launch_bin_count(const float4* rec, int T, const Cone* tiles, int tx, int ty, const Cone* supers, int sx,
                            int sy, uint32_t* counts, cudaStream_t st)
{
    if (T == 0) return VSR_OK;
    bin_kernel<false><<<(T + 127) / 128, 128, 0, st>>>(rec, T, tiles, tx, ty, supers, sx, sy, counts, nullptr, nullptr,
                                                       0, nullptr);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_scan(const uint32_t* counts, int n, uint32_t* offsets, cudaStream_t st)
{
    scan_kernel<<<1, 1024, 0, st>>>(counts, n, offsets);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}

vsr_status launch_bin_fill(const float4* rec, int T, const Cone* tiles, int tx, int ty, const Cone* supers, int sx,
                           int sy, const uint32_t* offsets, uint32_t* cursors, uint32_t* ids, uint32_t cap,
                           int* status, cudaStream_t st)
{
    if (T == 0) return VSR_OK;
    bin_kernel<true><<<(T + 127) / 128, 128, 0, st>>>(rec, T, tiles, tx, ty, supers, sx, sy, cursors, offsets, ids,
                                                      cap, status);
    VSR_CUDA_TRY(cudaGetLastError());
    return VSR_OK;
}
