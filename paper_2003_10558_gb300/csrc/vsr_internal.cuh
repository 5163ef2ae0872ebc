// vsr_internal.cuh -- layouts and helpers shared by the kernels and the host
// library of the visual-sphere rasterizer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vsr.h"

// ---------------------------------------------------------------------------
// Tiling.  The map is cut into TILE x TILE pixel tiles (one raster CTA each).
constexpr int TILE = 16;
constexpr int TILE_PIX = TILE * TILE;

// ---------------------------------------------------------------------------
// Per-triangle set-up record: REC_F float4 fields stored field-major
// (field f of triangle t at rec[f * T + t]) so that the binner reads its two
// cap fields coalesced.
enum {
    RF_CAP = 0,   // (S-hat.hi xyz, cos rho)            miter cap centre and radius
    RF_CAP2 = 1,  // (sin rho, 2(1 - cos rho), 1/(2 sin rho), valid ? 1 : 0)
    RF_N1 = 2,    // (n_AB.hi xyz, tie flags)          edge normals, FP32 high parts
    RF_N2 = 3,    // (n_BC.hi xyz, 0)
    RF_N3 = 4,    // (n_CA.hi xyz, 0)
    RF_PL = 5,    // (N-hat.hi xyz, (A'.N)/|N|)         plane for the ray-plane depth
    RF_N1L = 6,   // (n_AB.lo xyz, S-hat.lo.x)          low parts
    RF_N2L = 7,   // (n_BC.lo xyz, S-hat.lo.y)
    RF_N3L = 8,   // (n_CA.lo xyz, S-hat.lo.z)
    RF_PLL = 9,   // (N-hat.lo xyz, 0)
    REC_F = 10
};

// tie flags in RF_N1.w (as integer bits): bit i set <=> the first nonzero
// component of edge normal i is positive (simulation-of-simplicity rule for
// g_i == 0 in the centre test).

// ---------------------------------------------------------------------------
// Tile cones (per tile, 2 float4):
//   c0 = (axis xyz, cos alpha)   all valid pixel directions of the tile lie
//                                within alpha of the axis
//   c1 = (sin alpha, h, n_valid, 0) with h = max over valid pixels of
//                                1/(2 delta) (the widest ramp half-width)
// An empty tile has n_valid = 0.
struct Cone {
    float4 c0, c1;
};

// ---------------------------------------------------------------------------
// Tile index of a map: a latitude-longitude grid over the view sphere
// (latitude = asin(y), longitude = atan2(x, z), so the grid's poles are the
// camera's +-y axis).  Every tile whose cone half-angle is at most alpha_cut
// is filed once, in the cell holding its axis; larger ("big") tiles are kept
// in a separate list that every triangle scans.  A triangle whose enlarged
// cap has angular radius beta can only reach small tiles whose axis lies
// within beta + alpha_small_max of the cap centre, i.e. in a small
// latitude/longitude window of cells.  Grid size and alpha_cut are chosen on
// the device from the distribution of tile half-angles.  The index serves
// the triangle-major search of the fixed-array path and is built on its
// first use after each generation of the map; the header's first word, the
// widest ramp, is kept by the map kernels for every generation.
constexpr int IDX_NLAT_MAX = 128;
constexpr int IDX_CELLS_MAX = IDX_NLAT_MAX * 2 * IDX_NLAT_MAX;
constexpr int IDX_HIST = 64;

struct TileIndexHdr {
    // (generation << 32) | float bits of the largest ramp half-width of the
    // map's latest generation: raised by the map kernels with a 64-bit
    // maximum, so the widest ramp is known without the rest of the index
    unsigned long long h_gen;
    int nlat, nlon;             // grid: nlon = 2 nlat, square cells of `cell` radians
    int ncell;                  // nlat * nlon
    float cell;
    float alpha_cut;            // small / big tile threshold (radians)
    unsigned alpha_small_max;   // float bits: largest half-angle of a small tile
    unsigned h_max;             // float bits: largest ramp half-width 1/(2 delta)
    unsigned n_big;
    unsigned n_valid;
    // float bits: the half-angle about the camera's +z axis of a cone that
    // holds every tile cone (the map's field of view), plus a margin; 0 for a
    // map without a valid pixel
    unsigned view_angle;
    unsigned hist[IDX_HIST];    // third-of-an-octave histogram of half-angles
};

// Device-side status word (vsr_status values; 0 = OK), one int per device
// owned by the host library and passed to the kernels that can fail.
__device__ __forceinline__ void raise_status(int* status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// Conservative test: may a cap (centre S, cos/sin of radius, enlarged by the
// ramp half-width h measured on the miter's normalised distance) reach a
// direction inside the cone (axis, cos/sin alpha)?
//   fragment region of the miter:  G.S - cos rho > -h sin rho
//   i.e. a cap of cos(beta) = cos rho - h sin rho.
__device__ __forceinline__ bool cap_hits_cone(float3 S, float cos_rho, float sin_rho, float3 axis, float cos_a,
                                              float sin_a, float h)
{
    const float eps = 2e-6f;
    float cb = cos_rho - h * sin_rho;
    if (cb + cos_a <= eps) return true;  // alpha + beta >= pi
    if (cb <= -1.0f) return true;
    float sb = sqrtf(fmaxf(0.0f, 1.0f - cb * cb));
    float cg = S.x * axis.x + S.y * axis.y + S.z * axis.z;
    return cg >= cos_a * cb - sin_a * sb - eps;
}

#define VSR_CUDA_TRY(expr)                                                                                              \
    do {                                                                                                                \
        cudaError_t _e = (expr);                                                                                        \
        if (_e != cudaSuccess) return VSR_ERR_CUDA;                                                                     \
    } while (0)

// Kernel launchers (defined in the .cu files, called by the host library).
// The map kernels write the tile cones and geometry and raise the map's
// widest-ramp word h_gen (TileIndexHdr::h_gen) with generation gen, which
// must exceed every generation the word has seen.
vsr_status launch_map(int W, int H, int aov, float k, float l, float s, float omega_deg, float4* map, Cone* tiles,
                      float4* geom, unsigned long long* h_gen, uint32_t gen, cudaStream_t st);
vsr_status launch_map_cones(const float4* map, int W, int H, Cone* tiles, float4* geom, unsigned long long* h_gen,
                            uint32_t gen, cudaStream_t st);
// a map of any vsr_map_kind (param after limits for the Universal kind);
// deriv (optional): 2 float4 per pixel, (d_i G, d_j G) for the pixel step
vsr_status launch_map_spec(const vsr_map_spec& spec, float4* map, Cone* tiles, float4* geom, float4* deriv,
                           unsigned long long* h_gen, uint32_t gen, cudaStream_t st);
vsr_status launch_setup(const float* tris, int T, const float cam[12], float4* rec, cudaStream_t st);

// Device memory of a tile index (sized for IDX_CELLS_MAX cells, ntiles tiles).
// The cones of the small tiles are stored sorted by home cell, so the cells
// of one grid row form one contiguous range: (axis xyz, cos alpha),
// (sin alpha, h, tile index bits, 0).  Big tiles are stored the same way.
struct TileIndex {
    TileIndexHdr* hdr;
    uint32_t* cell_start;  // IDX_CELLS_MAX + 1
    Cone* sorted;          // ntiles
    Cone* big;             // ntiles
    float4* geom;          // ntiles: (alpha, latitude, longitude of the axis, h), h = -1 if the tile is empty;
                           // written with the cones by the map kernels
    uint32_t ntiles;       // tiles of the map (the length of sorted, big and geom)
};
// The whole index from the tile cones and geometry (any generation).
vsr_status launch_tile_index(const Cone* tiles, int ntiles, TileIndex idx, cudaStream_t st);

// Grid arithmetic of the tile index (bin.cu).
constexpr float IDX_PI = 3.14159265358979f;

__device__ __forceinline__ int hist_bin(float a)
{
    // third-of-an-octave bins from 2^-17 rad
    int b = (int)floorf((log2f(fmaxf(a, 1e-30f)) + 17.0f) * 3.0f);
    return min(IDX_HIST - 1, max(0, b));
}

__device__ __forceinline__ int cell_row(float lat, const TileIndexHdr& h)
{
    return min(h.nlat - 1, max(0, (int)floorf((lat + 0.5f * IDX_PI) / h.cell)));
}

__device__ __forceinline__ int cell_col(float lon, const TileIndexHdr& h)
{
    int c = (int)floorf((lon + IDX_PI) / h.cell);
    c %= h.nlon;
    return c < 0 ? c + h.nlon : c;
}

__device__ __forceinline__ int home_cell_geom(const float4& g, const TileIndexHdr& h)
{
    return cell_row(g.y, h) * h.nlon + cell_col(g.z, h);
}

// A tile's reach from the camera's +z axis, as float bits (non-negative, so
// they order as the floats): the angle of its axis from +z plus its
// half-angle and a margin for the FP32 rounding.
__device__ __forceinline__ unsigned view_angle_bits(const Cone& c, float alpha)
{
    return __float_as_uint(acosf(fmaxf(-1.0f, fminf(1.0f, c.c0.z))) + alpha + 1e-5f);
}

// The index's copy of tile i's cone: (axis xyz, cos alpha), (sin alpha, h,
// tile index bits, 0).
__device__ __forceinline__ Cone index_entry(const Cone& c, int i)
{
    Cone e;
    e.c0 = c.c0;
    e.c1 = make_float4(c.c1.x, c.c1.y, __uint_as_float((uint32_t)i), 0.0f);
    return e;
}
// binning of one frame: counts and cursor zeroed by the caller ->
// launch_bin_count (records (tile, triangle) into pairs[0, pair_cap)
// and counts them in *cursor; pairs may be NULL) -> launch_scan(counts,
// NULL) -> launch_bin_fill (a map over the pairs when *cursor <= pair_cap,
// else a second search; pass the count pass's pairs / pair_cap, or NULL)
vsr_status launch_bin_count(const float4* rec, int T, TileIndex idx, uint32_t* counts, uint32_t* cursor,
                            uint2* pairs, uint32_t pair_cap, cudaStream_t st, int pstep = 0);
// total_host (optional): the device address of a pinned host word that
// also receives the total
vsr_status launch_scan(const uint32_t* counts, const uint32_t* extra, int n, const int* n_dev, uint32_t* offsets,
                       cudaStream_t st, uint32_t* total_host = nullptr);
vsr_status launch_bin_fill(const float4* rec, int T, TileIndex idx, const uint32_t* offsets, uint32_t* counts,
                           const uint32_t* cursor, const uint2* pairs, uint32_t pair_cap, uint32_t* ids, uint32_t cap,
                           int* status, cudaStream_t st, int pstep = 0);

// ---------------------------------------------------------------------------
// Tile-major binning.  The frame's triangles are filed by the cell of their
// cap centre on one of two latitude-longitude grids of the view sphere (the
// same latitude / longitude as the tile index): caps of enlarged radius up to
// two cells of the fine grid (pi / TRI_NLAT0) in its cells, TRI_K0 per cell,
// a triangle that does not fit (a larger cap or a full cell) in the coarse
// grid (pi / TRI_NLAT1, TRI_K1 per cell) if its cap is at most two of its
// cells, and the rest in one list.  Every tile then tests only the triangles
// of the cells within its half-angle plus each grid's largest cap radius of
// its axis, and the list: one warp per tile, the same cap / cone test as the
// triangle-major search.  One pass: the warp stages its hits in shared
// memory, takes its range of the bins with one atomic, and writes them, so
// the bins of tile u are ids[starts[u] .. ends[u]) (not ordered by tile);
// starts[ntiles] receives the total.
constexpr int TRI_NLAT0 = 128, TRI_NLON0 = 2 * TRI_NLAT0, TRI_K0 = 64;
constexpr int TRI_NLAT1 = 16, TRI_NLON1 = 2 * TRI_NLAT1, TRI_K1 = 512;
constexpr int TRI_CELLS0 = TRI_NLAT0 * TRI_NLON0;
constexpr int TRI_CELLS1 = TRI_NLAT1 * TRI_NLON1;
constexpr int TRI_LARGE = TRI_CELLS0 + TRI_CELLS1;  // the counter of the list
constexpr int TRI_CELLS = TRI_LARGE + 1;
// entry numbers: fine cells, coarse cells, then the list
constexpr uint32_t TRI_E1 = (uint32_t)TRI_CELLS0 * TRI_K0;
constexpr uint32_t TRI_E2 = TRI_E1 + (uint32_t)TRI_CELLS1 * TRI_K1;

// Device memory of a triangle index (per scene, up to T triangles and
// ntiles tiles).  The counters and the header are zero between binnings:
// the last kernel of a binning clears them for the next one, so the
// launches are the same every time and can be captured in a graph (after a
// failed launch the next binning clears them first).
constexpr int TRI_HDR = TRI_CELLS;  // header words after the cell counters:
constexpr int TRI_H_CURSOR = 2;     //   [0..1] largest enlarged cap radius of the fine / coarse grid (float bits),
constexpr int TRI_H_DONE = 3;       //   bin cursor, finished CTAs of the tile pass,
constexpr int TRI_H_HEAVY = 4;      //   heavy tiles listed,
constexpr int TRI_H_NEXT = 5;       //   heavy tiles taken,
constexpr int TRI_H_DONE2 = 6;      //   finished CTAs of the heavy-tile pass
constexpr int TRI_WORDS = TRI_CELLS + 7;
struct TriIndex {
    // TRI_WORDS: triangles filed per cell (may exceed the cell's capacity)
    // and the list length, then the header
    uint32_t* counts;
    uint32_t* heavy;  // ntiles: tiles binned by a whole CTA (more than BIN_STAGE_HITS entries)
    float4* cap;      // TRI_E2 + T entries: (S-hat xyz, cos beta)
    float2* cs;       // TRI_E2 + T entries: (sin beta, triangle bits)
    int64_t T;        // capacity of the list
    int ntiles;       // capacity of the heavy list
    bool dirty;       // host side: a binning may have left the counters behind
};
vsr_status tri_index_alloc(TriIndex* ti, int64_t T, int ntiles);
void tri_index_free(TriIndex* ti);
size_t tri_index_bytes(int64_t T, int ntiles);
// binning of one frame, tile-major: the triangle index of rec, then every
// tile of the map.  idx: the map's tile index (its header's
// widest ramp and each tile's geometry); tiles: the map's ntiles cones;
// starts / ends: ntiles + 1 / ntiles words; T <= ti->T.  With more pairs
// than cap the bins are cut at cap and VSR_ERR_BIN_OVERFLOW is raised;
// total_host (optional): the device address of a pinned host word that
// also receives the total.
vsr_status launch_bin_tiles(const float4* rec, int T, const TileIndex& idx, const Cone* tiles, int ntiles,
                            TriIndex& ti, uint32_t* starts, uint32_t* ends, uint32_t* ids, uint32_t cap, int* status,
                            uint32_t* total_host, cudaStream_t st, int pstep = 0);
// One view as the raster kernel sees it: its map, tile cones, set-up
// records, bin offsets (indexed by the view's own tile number), bin ids and
// outputs.
struct RasterView {
    const float4* map;
    int W, H;
    const Cone* tiles;
    int tiles_x;
    const float4* rec;
    int T;
    const uint32_t* offsets;
    const uint32_t* ids;
    uint32_t cap;
    uint32_t* out_id;
    float* out_depth;
    float* out_cov;
    // bins of the tile-major binner: tile u's bin ends at ends[u] (NULL:
    // bins in tile order, tile u's ending at offsets[u + 1])
    const uint32_t* ends = nullptr;
};

// One view as the binner sees it (tile index of the view's map, the view's
// set-up records, its per-tile counters and offsets).
struct BinView {
    const TileIndexHdr* hdr;
    const uint32_t* cell_start;
    const Cone* sorted;
    const Cone* big;
    const float4* rec;
    uint32_t* counts;
    const uint32_t* offsets;
    uint2* pairs;       // (tile, triangle) of every hit, or NULL
    uint32_t pair_cap;
    uint32_t* cursor;   // hits recorded (may exceed pair_cap: the list is then incomplete)
    int pstep;          // bins for the per-fragment pixel step (wider caps, see pstep_cap)
    uint32_t ntiles;    // tiles of the map: every index read from the tile index is clamped to it
};

// The cap that holds every fragment of the per-fragment pixel step
// (pstep.cu): its miter test G.S - cos rho > -(|S.d_i G| + |S.d_j G|)/2 is
// not scaled by sin rho like the global step's, and |S.d G| <= sin(theta)
// |d G| at angle theta from S, so with h >= the widest ramp half-width
// (|d_i G| + |d_j G|)/2 every fragment lies within the angle rho + 4h of S.
// Returns (cos, sin) of that radius.
__device__ __forceinline__ float2 pstep_cap(float cos_rho, float sin_rho, float h)
{
    const float e = 4.0f * h;
    if (e >= 3.14159265f) return make_float2(-1.0f, 0.0f);
    float se, ce;
    sincosf(e, &se, &ce);
    const float c = fmaf(cos_rho, ce, -sin_rho * se);
    const float s = fmaf(sin_rho, ce, cos_rho * se);
    // past the antipode the cap is the whole sphere
    return (s < 0.0f && c < 0.0f) ? make_float2(-1.0f, 0.0f) : make_float2(c, fmaxf(s, 0.0f));
}

// Work items of the raster: a tile whose bin is longer than split_max
// triangles is processed by several CTAs whose results merge order-free
// (see SplitAcc in raster.cu).
constexpr uint32_t SPLIT_SLOTS = 4096;    // split tiles per launch (others run unsplit)
constexpr uint32_t EXTRA_ITEMS = 1u << 16;  // extra items per launch
constexpr int SPLIT_MAX_DEFAULT = 512;    // triangles per item of a split tile
struct RasterWork {
    uint32_t* nsplit_of;      // n_tiles: items of each tile
    int32_t* split_slot;      // n_tiles: accumulator slot of a split tile, -1 if not split
    uint32_t* counters;       // 2: split tiles, extra items
    uint2* extra;             // extra_cap: (tile, k) of the further items
    uint32_t split_cap, extra_cap;
    unsigned long long* acc;  // split_cap x TILE_PIX, zero between frames
    unsigned long long* key;  // split_cap x TILE_PIX, all ones between frames
    uint32_t* done;           // split_cap, zero between frames
};
// SMs of the current device (looked up once per device), or -1.
int sm_count();

// A view's raster work for the pooled launch: the view, its item assignment
// (from launch_raster_assign) and its split accumulators.
struct PoolView {
    RasterView view;
    uint32_t n_tiles;
    const uint32_t* nsplit_of;
    const int32_t* split_slot;
    const uint2* extra;
    const uint32_t* n_extra;  // the work's counters + 1
    unsigned long long* acc;
    unsigned long long* key;
    uint32_t* done;
};
// items of a tile's split (a multiple of the staging chunk) and the room for
// extra items a view's work gets for bins of capacity cap
int raster_split_items(int split_max);
uint32_t raster_extra_cap(uint32_t cap, const RasterWork& w, int split_max);
// the work items of one view (split tiles, extra items), for the pooled
// launch; ends: as RasterView::ends
vsr_status launch_raster_assign(const uint32_t* offsets, uint32_t n_tiles, uint32_t cap, RasterWork w, int split_max,
                                cudaStream_t st, const uint32_t* ends = nullptr);
// one persistent raster launch over the items of several views: view v owns
// items item_start[v] .. item_start[v + 1] - 1 (its tiles, then its extra
// items); queue: a device counter (zeroed here)
vsr_status launch_raster_pool(const PoolView* views_dev, const uint32_t* item_start_dev, int nviews,
                              uint32_t* queue, int split_max, int* status, cudaStream_t st);
// items + raster over all tiles of a view; offsets: its bin offsets
// (n_tiles + 1 entries, or the bins' starts with view.ends); cap: the bins' capacity (bounds the extra items);
// host_out: the outputs are pinned host memory (written in whole tile rows)
vsr_status launch_raster_items(const RasterView& view, const uint32_t* offsets, uint32_t n_tiles, uint32_t cap,
                               RasterWork w, int split_max, int* status, cudaStream_t st, bool host_out = false);
// the dense reference: every pixel against every triangle, no bins
vsr_status launch_raster_dense(const RasterView& view, int* status, cudaStream_t st);
// allocate / free a RasterWork for up to n_tiles tiles (accumulators
// initialised)
vsr_status raster_work_alloc(RasterWork* w, uint32_t n_tiles);
void raster_work_free(RasterWork* w);
int raster_threads_per_cta();
// set-up of nviews views (grid.y = view) with the cameras in device memory
// (12 floats each: O xyz, M 3x3 row-major); view v's records at
// rec + v * REC_F * T
vsr_status launch_setup_views(const float* tris, int T, const float* cams_dev, int nviews, float4* rec,
                              cudaStream_t st);
// exclusive scan of counts (+ extra) for large n (multi-CTA); `partials`
// needs 2 * ceil(n / 4096) + 2 words
vsr_status launch_scan_large(const uint32_t* counts, const uint32_t* extra, int n, uint32_t* partials,
                             uint32_t* offsets, cudaStream_t st);

vsr_status launch_raster(const float4* map, int W, int H, const Cone* tiles, const float4* rec, int T,
                         const uint32_t* offsets, const uint32_t* ids, uint32_t cap, uint32_t* id, float* depth,
                         float* cov, unsigned long long* n_alg, unsigned long long* n_exec, int32_t* n_inside,
                         int* status, cudaStream_t st, const uint32_t* ends = nullptr);

// ---------------------------------------------------------------------------
// Differentiable path (grad.cu, map.cu).
// Gradient of the set-up records, field-major [GF_COUNT][T] float4:
enum {
    GF_N1 = 0,   // d/d n_AB (xyz), 0
    GF_N2 = 1,   // d/d n_BC
    GF_N3 = 2,   // d/d n_CA
    GF_CAP = 3,  // d/d S-hat (xyz), d/d cos rho
    GF_PL = 4,   // d/d N-hat (xyz), d/d colour
    GF_D = 5,    // d/d (A'.N-hat), 0, 0, 0
    GF_COUNT = 6
};
struct FragArgs {
    const float4* map;
    int W, H;
    const Cone* tiles;
    const float4* rec;
    int T;
    const uint32_t* offsets;  // tile bins
    const uint32_t* ids;
    uint32_t cap;
    const float* colors;      // per triangle, NULL = 1
    uint32_t* counts;         // W*H fragments per pixel (count pass)
    const uint32_t* foff;     // W*H + 1 exclusive scan of counts
    float4* frags;            // fragment records (r, t, m^f, shade)
    uint32_t fcap;
    float* image;
    float* cov;
    uint32_t* out_id;
    float* out_depth;
    int* status;
    const uint32_t* ends = nullptr;  // as RasterView::ends
};
vsr_status launch_frag_count(const FragArgs& a, cudaStream_t st);
vsr_status launch_frag_fill(const FragArgs& a, cudaStream_t st);
vsr_status launch_frag_backward(const FragArgs& a, const uint32_t* id, const float* dimage, const float* dcov,
                                const float* ddepth, float4* grad, float4* dmap, cudaStream_t st);
vsr_status launch_setup_backward(const float* tris, int T, const float cam[12], const float4* rec, const float4* grad,
                                 float* dtris, float* dcolors, cudaStream_t st);
size_t map_backward_partials(int W, int H);
vsr_status launch_map_backward(int W, int H, int aov, float k, float l, float s, float omega_deg,
                               const float4* dmap, float* partials, double* dlens, cudaStream_t st);

// rasterization with the per-fragment pixel step (pstep.cu): one CTA per
// tile over whole bins; deriv: 2 float4 per pixel from launch_map_spec
vsr_status launch_raster_pstep(const RasterView& view, const float4* deriv, int* status, cudaStream_t st);
