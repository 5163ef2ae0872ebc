/*
 * vsr.h -- C ABI of the GB300 visual-sphere rasterizer.
 *
 * The library rasterizes triangles directly into a per-pixel direction map
 * ("perspective map") as described in J. M. Fober, "Perspective picture from
 * Visual Sphere: a new approach to image rasterization" (arXiv 2003.10558):
 * every pixel carries a unit view direction G from the Universal perspective
 * model (Sec. 2), a triangle ABC seen from the eye O is bounded by the three
 * great-circle planes OAB, OBC, OCA (Sec. 1.1) plus the miter cap of its
 * smallest enclosing circle (Sec. 1.1.2), coverage uses the analytic
 * global-delta step (Sec. 1.1.1), depth is the ray-plane distance (Sec.
 * 1.1.4) and fragments merge front to back (Sec. 1.4).
 *
 * Conventions shared by every entry point:
 *   - All device pointers are CUDA global-memory pointers on the current
 *     device; host pointers are ordinary (pageable or pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is asynchronous on that stream unless stated.
 *   - Handles (vsr_map, vsr_scene) are owned by the library; free them with
 *     their *_free function.  Output buffers are owned by the caller.
 *   - No call aborts or exits.  Every error is a vsr_status.  Errors raised
 *     by device code (e.g. bin overflow) are recorded in a per-device status
 *     word and returned by vsr_last_device_status(), which synchronises.
 *   - Inputs are never modified.
 *   - Images are row-major [H][W]; pixel (i, j) is column i, row j, row 0
 *     first in memory.
 */
#ifndef VSR_H
#define VSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VSR_OK = 0,
    VSR_ERR_INVALID_ARG = -1,  /* bad size, NULL pointer, non-finite parameter */
    VSR_ERR_OOM = -2,          /* device or host allocation failed */
    VSR_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    VSR_ERR_BIN_OVERFLOW = -4, /* a tile bin exceeded its capacity (device-side) */
    VSR_ERR_FRAG_OVERFLOW = -5,/* differentiable path: fragment lists of another frame (device status) */
    VSR_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
    VSR_ERR_BUDGET = -7,       /* a request does not fit the memory budget */
    VSR_ERR_CANCELLED = -8
} vsr_status;

/* Angle-of-view types of the view-coordinate normalisation (Sec. 2, remark
 * on AOV types): x = 2 f_s - 1, y = 2 f_t - 1, then
 *   HORIZONTAL  y /= a              (a = W/H)
 *   DIAGONAL    (x a, y) / sqrt(1 + a^2)
 *   VERTICAL    x *= a
 *   H4X3        (x a, y) / (4/3)                                         */
typedef enum { VSR_AOV_HORIZONTAL = 0, VSR_AOV_DIAGONAL = 1, VSR_AOV_VERTICAL = 2, VSR_AOV_H4X3 = 3 } vsr_aov;

typedef struct vsr_map_s* vsr_map;
typedef struct vsr_scene_s* vsr_scene;

/* Universal perspective parameters (Sec. 2, "Universal perspective
 * parameters and limits").  k in [-1, 1] picks the azimuthal projection
 * (1 gnomonic, 0.5 stereographic, 0 equidistant, -0.5 equisolid,
 * -1 orthographic); l in [0, 1] cylindricity; s anamorphic correction;
 * omega_deg the angle of view in degrees.  The limits of the paper are
 * applied on creation: k, l clamped; omega clamped to
 * [1, (k > 0 ? 179 : 180) / max(|k|, 1/2)]; s clamped to [0.8, 1] when
 * strict_limits != 0, else to [0.5, 1]. */
typedef struct {
    float k, l, s, omega_deg;
    int W, H;
    int aov;           /* vsr_aov */
    int strict_limits; /* 0 or 1 */
} vsr_map_params;

/* ---- perspective map ------------------------------------------------------
 * vsr_make_map: build the direction map of a W x H picture on `stream`
 * (Universal perspective 2D->3D transform, Sec. 2): for pixel centre
 * f = ((i + 1/2)/W, (j + 1/2)/H) with view coordinates (x, y),
 *   R = sqrt(x^2 + l y^2),
 *   theta = atan(tan(k Omega/2) R)/k | Omega/2 R | asin(sin(k Omega/2) R)/k
 *           for k > 0 | k = 0 | k < 0,
 *   G = normalize(x sin(theta)/R, y sin(theta)/R / (l(1-s)+s), cos(theta)),
 * and the global delta delta = 1 / max_c fwidth(G_c) (Sec. 1.1.1) from
 * central differences of the map function at the neighbouring pixel
 * centres.  Stored as float4 (G_x, G_y, G_z, delta) per pixel; pixels where
 * asin is undefined are (0, 0, 0, 0) and are never covered.  Also builds the
 * per-tile view cones used by the binner.
 * Horizontal AOV, non-strict limits.  1 <= W, H <= 32768.
 * Returns VSR_ERR_INVALID_ARG for bad sizes or non-finite parameters. */
vsr_status vsr_make_map(float k, float l, float s, float omega_deg, int W, int H, void* stream, vsr_map* out);
vsr_status vsr_make_map_ex(const vsr_map_params* p, void* stream, vsr_map* out);

/* Build a map from a caller-supplied float4 [H][W] (G_x, G_y, G_z, delta)
 * array in DEVICE memory (copied; the caller keeps ownership).  Directions
 * must be unit length where delta > 0; delta <= 0 marks an invalid pixel.
 * Tile cones are computed from the data.  Lets a user rasterize into a map
 * made elsewhere (the paper's "perspective pixel-shader pass", Sec. 1.1.5). */
vsr_status vsr_map_from_device(const float* xyzd_dev, int W, int H, void* stream, vsr_map* out);

/* Maps of other projections (Sec. 2.2) and lens distortion (Sec. 2.3).
 * The rasterizer takes any direction map, so these feed the same raster,
 * binning and differentiable path.  Pixel centres, AOV types and the
 * global delta as for vsr_make_map; the delta uses neighbours on the same
 * chart only (one-sided at a cube map's face borders).
 *   VSR_MAP_UNIVERSAL    param = (k, l, s, omega_deg), limits applied
 *   VSR_MAP_RECTILINEAR  param = (omega_deg): G = normalize(x, y, cot(Omega/2))
 *                        (Sec. 2.2.1; omega < 180)
 *   VSR_MAP_PANORAMA     param = (omega_h_deg, height): with
 *                        f' = (Omega_h (f_s - 1/2), height (f_t - 1/2)),
 *                        G = normalize(sin f'_x, f'_y, cos f'_x) (Sec. 2.2.2)
 *   VSR_MAP_DOME         param = (compression_deg, tilt_deg, offset): with
 *                        f' = (2 f_s - 1, 1 - 2 f_t), R = |f'|,
 *                        theta = R (compression + 90 deg),
 *                        G = normalize(f'_x sin(theta)/R, cos(theta),
 *                        f'_y sin(theta)/R + offset) tilted about x; pixels
 *                        with R > 1 are invalid (Sec. 2.2.3)
 *   VSR_MAP_EQUIRECT     no param: f' = pi (2 f_s - 1, f_t),
 *                        G = (sin f'_x sin f'_y, -cos f'_y, cos f'_x sin f'_y)
 *                        (Sec. 2.2.4)
 *   VSR_MAP_CUBE         no param: W = 6 H for square faces; face
 *                        floor(6 f_s) rotates normalize(fract(6 f_s) - 1/2,
 *                        f_t - 1/2, 1/2) to look along +x, -x, -z, +z, +y,
 *                        -y (Sec. 2.2.7; face 3, absent from the paper's
 *                        case list, is the front face along +z)
 * distortion = (k1, k2, p1, p2, q1, q2), Brown-Conrady on the view
 * coordinates of the Universal and rectilinear kinds (Sec. 2.3):
 * r2 = x^2 + y^2, (x, y) <- (x, y)(1 + k1 r2 + k2 r2^2) + (x, y)(p1 x + p2 y)
 * + (q1, q2) r2; zeros leave the map unchanged.
 * vsr_raster_backward's lens gradient exists only for undistorted
 * Universal maps. */
typedef enum {
    VSR_MAP_UNIVERSAL = 0,
    VSR_MAP_RECTILINEAR = 1,
    VSR_MAP_PANORAMA = 2,
    VSR_MAP_DOME = 3,
    VSR_MAP_EQUIRECT = 4,
    VSR_MAP_CUBE = 5
} vsr_map_kind;
typedef struct {
    int kind;  /* vsr_map_kind */
    int W, H;
    int aov;   /* vsr_aov: Universal and rectilinear */
    float param[4];
    float distortion[6];
    int flags; /* VSR_MAP_DERIVATIVES: keep (d_i G, d_j G) for vsr_raster_pstep */
} vsr_map_spec;
#define VSR_MAP_DERIVATIVES 1
vsr_status vsr_make_map_spec(const vsr_map_spec* spec, void* stream, vsr_map* out);

/* (d_i G, d_j G) of a map made with VSR_MAP_DERIVATIVES, synchronous copy
 * into host memory: W*H*8 floats, (d_i G xyz, 0, d_j G xyz, 0) per pixel --
 * the central (one-sided next to an unusable neighbour) differences of the
 * map function that the global delta is formed from. */
vsr_status vsr_map_download_derivatives(vsr_map m, float* host);

/* Regenerate an existing map in place for new parameters (reallocates
 * only when W or H change).  Same semantics as vsr_make_map_ex. */
vsr_status vsr_map_update(vsr_map m, const vsr_map_params* p, void* stream);

/* Effective parameters after the limits (omega in degrees). */
vsr_status vsr_map_params_effective(vsr_map m, vsr_map_params* out);

/* Device pointer of the map's float4 [H][W] array (owned by the map). */
vsr_status vsr_map_data(vsr_map m, const float** xyzd_dev, int* W, int* H);

/* Synchronous copy of the map into host memory (W*H*4 floats). */
vsr_status vsr_map_download(vsr_map m, float* host_xyzd);

void vsr_map_free(vsr_map m);

/* ---- triangle set-up --------------------------------------------------------
 * vsr_setup: per-triangle set-up (Sec. 1.1, 1.1.2, 1.1.4) of T world-space
 * triangles `tris_dev` (device, FP32, [T][3 vertices][xyz]) seen by the
 * camera `cam` (host, 12 floats: eye O xyz, then the 3x3 world->camera
 * rotation M row-major; X' = M (X - O)).  Computes in FP32-pair arithmetic
 * the edge-plane normals ||A' x B'||, ||B' x C'||, ||C' x A'|| oriented by
 * sign(A'.(B' x C')), the miter cap (smallest circle centre S-hat, cos and
 * sin of its radius), and the plane (unit normal of (A'-B') x (C'-B'),
 * offset).  Triangles with a vertex at the eye or with A'.(B' x C') = 0 are
 * culled.  The scene keeps a pointer-free copy of the records; `tris_dev`
 * may be freed once the call has completed on `stream`.
 * 0 <= T < 2^31 - 1. */
vsr_status vsr_setup(const float* tris_dev, int64_t T, const float cam[12], void* stream, vsr_scene* out);

/* An empty scene (T = 0) to be filled by vsr_scene_update or
 * vsr_render_host. */
vsr_status vsr_scene_create(vsr_scene* out);

/* Re-run the set-up of an existing scene for new triangles and/or camera,
 * reusing its device memory when T does not grow. */
vsr_status vsr_scene_update(vsr_scene s, const float* tris_dev, int64_t T, const float cam[12], void* stream);

void vsr_scene_free(vsr_scene s);
int64_t vsr_scene_size(vsr_scene s);

/* ---- rasterization ---------------------------------------------------------
 * vsr_raster: rasterize the scene into the map (Sec. 1.1.2 eq.
 * "rasterization", Sec. 1.1.1 gpstep/gbpxstep, Sec. 1.1.4 depth, Sec. 1.4
 * merge).  For pixel direction G with global delta delta and triangle t:
 *   g_1..3 = G.n_i, g_4 = miter distance (G.S-hat - cos rho)/sin rho,
 *   fragment iff every g_i > -1/(2 delta) and depth r = (A'.N)/(G.N) > 0,
 *   m^f = min_i clamp(delta g_i + 1/2, 0, 1),
 *   centre-inside iff g_1..3 >= 0 (ties: inside iff the first nonzero
 *   component of the edge normal is positive).
 * Outputs (caller-owned DEVICE buffers of W*H elements, any may be NULL):
 *   id    uint32: the nearest centre-inside triangle (ties: lower index),
 *         0xFFFFFFFF if none;
 *   depth float: its r, +inf if none;
 *   cov   float: the front-to-back merged mask m^b = min(1, sum of m^f).
 * The merge of Sec. 1.4 (m^fc = min(m^f, 1 - m^b), m^b += m^fc) telescopes
 * to min(1, sum m^f), so the result does not depend on fragment order; it is
 * accumulated in 2^-22 fixed point and is bit-reproducible.
 * Binning (which triangles may cover which 16x16 tile: the enlarged cap of
 * each triangle against the tile's view cone, the region mask of Sec.
 * 1.1.3): with at most 64 triangles per tile, tile-major (the triangles
 * filed by cap cell, then each tile over the cells in its reach), else
 * triangle-major over the map's tile index (built on the first such
 * binning after each update of the map); both give the same outputs.
 * Scratch (tile bins, the triangle index of the tile-major binning: about
 * 57 MB plus 24 B per triangle) is held by the scene handle.  It is sized
 * with one synchronisation of `stream` the first time and whenever the
 * map's tile count or the scene's T changes; otherwise no call
 * synchronises: the bins
 * grow ahead of need from the pair count of an earlier frame, and a frame
 * that still outgrows them (e.g. after the camera moved) raises
 * VSR_ERR_BIN_OVERFLOW in the device status (vsr_last_device_status) with
 * that frame's outputs incomplete, the next call growing the bins.  A scene
 * must not be rasterized on two streams at the same time. */
vsr_status vsr_raster(vsr_map m, vsr_scene s, uint32_t* id_dev, float* depth_dev, float* cov_dev, void* stream);

/* vsr_raster_pstep: vsr_raster with the per-fragment pixel step of Sec.
 * 1.1.1 instead of the global delta: every plane distance g ramps over its
 * own fwidth w = |d_i g| + |d_j g|, d g = n . d G for the edges and
 * (S-hat . d G)/sin(rho) for the miter, from the map's differences:
 *   fragment iff every g > -w/2 (bpxstep), m^f = min clamp(g/w + 1/2, 0, 1).
 * The map must be made with VSR_MAP_DERIVATIVES (else VSR_ERR_INVALID_ARG).
 * Bins the scene for the wider caps of this step (bins that vsr_raster_tiles
 * may reuse).  Outputs as vsr_raster. */
vsr_status vsr_raster_pstep(vsr_map m, vsr_scene s, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                            void* stream);

/* The two halves of vsr_raster, for callers that reuse one binning:
 * vsr_bin builds the tile bins of (m, s) (as described for vsr_raster);
 * vsr_raster_tiles runs the tile coverage/depth kernel on the current bins
 * and returns VSR_ERR_INVALID_ARG if they were built for another map or an
 * older set-up of the scene. */
vsr_status vsr_bin(vsr_map m, vsr_scene s, void* stream);

/* Diagnostics of one rasterization (all optional, NULL to skip). */
typedef struct {
    uint64_t* n_alg_dev;     /* device: += pairs with G inside the enlarged cap */
    uint64_t* n_exec_dev;    /* device: += pixel x triangle pairs evaluated */
    int32_t* n_inside_dev;   /* device [H][W]: count of centre-inside triangles */
} vsr_raster_stats;

vsr_status vsr_raster_ex(vsr_map m, vsr_scene s, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                         const vsr_raster_stats* stats, void* stream);
vsr_status vsr_raster_tiles(vsr_map m, vsr_scene s, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                            const vsr_raster_stats* stats, void* stream);

/* vsr_raster_dense: the same outputs as vsr_raster, computed without tile
 * binning: every pixel of the map against every triangle of the scene --
 * the rasterization equation (Sec. 1.1.2; the four plane distances, gpstep /
 * gbpxstep / bstep of Sec. 1.1.1, the depth of Sec. 1.1.4, the merge of Sec.
 * 1.4) with no region mask (Sec. 1.1.3) at all.  The miter distance is taken
 * first and a triangle whose enlarged cap misses a warp's 64 pixels is
 * skipped after it, as the FP64 reference skips it per pixel.  Costs W*H*T
 * pair tests: a baseline that shows what the binning saves, not a fast path.
 * The scene must hold set-up records (vsr_setup / vsr_scene_update).
 * Outputs as vsr_raster (caller-owned device memory, W*H each, any may be
 * NULL), bit for bit equal to vsr_raster's.  Asynchronous on `stream`;
 * device errors go to the scene's status word as for vsr_raster. */
vsr_status vsr_raster_dense(vsr_map m, vsr_scene s, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                            void* stream);

/* vsr_raster_noalloc: the same rasterization as vsr_raster, for callers that
 * cannot allocate device memory while they render (a host framework that
 * owns all device memory and forbids side allocations, or a real-time loop
 * that must not wait on cudaMalloc or on the synchronisation with which
 * vsr_raster sizes the bins of a new map/scene pair).  The paper has no
 * counterpart; this is a service of the library.
 * The tile bins live in one fixed device array inside the library (about
 * 4.3 MB, held on every device that loads the library until the process
 * exits) instead of the scene's workspace: the call allocates nothing and
 * never synchronises.  Maps and scenes are made beforehand as usual.
 * Limits: at most 16384 tiles of 16x16 pixels (e.g. 2048 x 2048; else
 * VSR_ERR_INVALID_ARG), at most 2^20 (tile, triangle) pairs (known only on
 * the device: exceeding it writes VSR_ERR_BIN_OVERFLOW to the status and
 * leaves the outputs incomplete).
 * status_dev: optional caller-owned device int32 that receives VSR_OK or the
 * device-side error of this call (cleared by the call).  With NULL the
 * status goes to a private word of the library's array that no call reads
 * (vsr_last_device_status does not see it), so a bin overflow -- outputs
 * incomplete -- cannot be observed: pass status_dev to learn of it.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make it before any stream capture.  Every call
 * shares the one array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller. */
vsr_status vsr_raster_noalloc(vsr_map m, vsr_scene s, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                              int32_t* status_dev, void* stream);

/* Number of (tile, triangle) pairs in the last binning of this scene
 * (synchronises `stream`). */
vsr_status vsr_scene_bin_pairs(vsr_scene s, void* stream, int64_t* pairs);

/* ---- end to end from host memory ------------------------------------------
 * vsr_render_host: one call from host buffers -- the operations of
 * vsr_setup (Sec. 1.1, 1.1.2, 1.1.4) and vsr_raster (Sec. 1.1.1-1.1.4,
 * 1.4): re-runs the set-up of the
 * work scene `s` (a handle from vsr_scene_create, whose device buffers are
 * reused across calls) on `tris_host` ([T][3][3] FP32, host), rasterizes
 * into the map and returns id/depth/cov (W*H each, host; any may be NULL),
 * then synchronises `stream`.  Same outputs as vsr_raster, but always
 * complete: since the call waits for the frame, a frame that outgrew the
 * scene's bins (see vsr_raster) is rendered again with grown bins before it
 * returns, and a bin overflow that persists is returned by the call
 * (VSR_ERR_BIN_OVERFLOW) instead of being raised in the per-device status.
 * Buffers in pinned host memory mapped into the device's address space
 * (cudaHostAlloc, cudaMallocHost, torch pin_memory) are read and written in
 * place by the kernels over the host link, so the transfers overlap the
 * set-up and raster kernels; other host memory is staged through device
 * buffers with copies before and after them.
 * The set-up (and the triangles' copy) runs on a stream of the scene's own
 * that waits only for the last queued use of `s` (by any call, on any
 * stream, from the first vsr_render_host on `s` on; at that first call,
 * for all work queued on `stream`).  Work queued on `stream` before the
 * call that does not use `s` -- a vsr_map_update of `m` -- therefore runs
 * beside the set-up; binning and raster follow on `stream` after both.
 * Uses of `s` inside a stream capture are not tracked: their graph
 * launches must complete before this call. */
vsr_status vsr_render_host(vsr_map m, vsr_scene s, const float* tris_host, int64_t T, const float cam[12],
                           uint32_t* id_host, float* depth_host, float* cov_host, void* stream);

/* vsr_render_host_async: vsr_render_host (the same operations and
 * passages) without the wait -- the frame is
 * queued on `stream` (the set-up on the scene's own stream as above) and the
 * call returns; vsr_render_host_wait(s) waits for it.  Frames of different
 * (map, scene) pairs queued on different streams run at the same time on the
 * device, so one frame's host transfers and raster overlap the next frame's
 * map, set-up and binning (two maps and two scenes used in turn pipeline a
 * stream of frames).  Until the wait returns, the scene, the map, the
 * triangles and the output buffers must not be touched, and a second
 * vsr_render_host(_async) on `s` returns VSR_ERR_INVALID_ARG.  Overlap needs
 * pinned buffers (in place); pageable ones are staged with copies.
 * vsr_render_host_wait returns VSR_OK (outputs complete),
 * VSR_ERR_BIN_OVERFLOW (the frame outgrew the scene's bins: its outputs are
 * incomplete; the next render of the scene grows them -- render it again),
 * or VSR_ERR_CUDA; VSR_OK also when no frame of `s` is queued. */
vsr_status vsr_render_host_async(vsr_map m, vsr_scene s, const float* tris_host, int64_t T, const float cam[12],
                                 uint32_t* id_host, float* depth_host, float* cov_host, void* stream);
vsr_status vsr_render_host_wait(vsr_scene s);

/* ---- batched multi-view rendering -------------------------------------------
 * A batch renders V views of one scene as one CUDA graph.  Each view is the
 * chain of vsr_setup (with the view's camera, Sec. 1.1, 1.1.2, 1.1.4), vsr_bin
 * and vsr_raster_tiles on a workspace of its own; the chains are spread over
 * S parallel streams inside the graph, so every view keeps its working set
 * in L2 while independent views overlap on the GPU, and no launch pays host
 * overhead.  Outputs per view are those of vsr_raster.
 *
 * vsr_batch_render: maps[V] (built with vsr_make_map*), tris_dev [T][3][3]
 * (device, shared by all views), cams (host, V x 12 floats, one camera per
 * view as in vsr_setup), id_dev / depth_dev / cov_dev (host arrays of V
 * caller-owned device pointers, [H_v][W_v] each; the arrays themselves or
 * any entry may be NULL).  The first call for a configuration (the same
 * maps, map contents, scene buffer and T, output pointers) renders the
 * views eagerly, synchronises `stream` once to size every view's bins, then
 * captures graphs of two kinds for each S in {1, 2, 4, 8}: each view's chain
 * ending in its own raster launch, and chains that end after binning and
 * work-item assignment, the views rasterized in G in {1, 4, 16} pooled
 * launches -- persistent CTAs (resident CTAs per SM x SMs) that take the
 * (view, item) work of a group of views from a shared queue (an atomic
 * counter; no CTA waits for another), each group's launch on a stream of its
 * own as soon as its views are binned, beside the next groups' chains.
 * It times their replays, keeps the fastest, then tries 256 and 1024
 * triangles per work item of a long bin at that S and kind (the autotuner;
 * vsr_batch_set_mode can restrict the kinds); later calls with the same configuration
 * copy only the cameras (into pinned staging of the batch) and replay the
 * graph on `stream`.  Each call waits for the previous frame of the batch to
 * finish; a replay leaves every view's (tile, triangle) pair total in pinned
 * memory, and a call that finds a view within 1/8 of its bin capacity
 * re-sizes the bins and captures again (as for a new configuration).  A
 * frame whose cameras outgrow the bins before that raises
 * VSR_ERR_BIN_OVERFLOW in the device status with its outputs incomplete; the
 * next call grows the bins.  Device memory per view: T x 228 B of set-up
 * records and bin caches plus its bins.  A batch must not render on two
 * streams at once. */
typedef struct vsr_batch_s* vsr_batch;
vsr_status vsr_batch_create(vsr_batch* out);
vsr_status vsr_batch_render(vsr_batch b, int nviews, const vsr_map* maps, const float* tris_dev, int64_t T,
                            const float* cams, uint32_t* const* id_dev, float* const* depth_dev,
                            float* const* cov_dev, void* stream);
/* The autotuned configuration (any pointer may be NULL): parallel streams
 * S, whether a graph is ready, and the triangles per work item of a long
 * bin (a tile whose bin holds more is rasterized by several CTAs). */
vsr_status vsr_batch_config(vsr_batch b, int* streams, int* graphed, int* split_max);
/* vsr_batch_config plus `pooled`: the number of pooled raster launches
 * (groups of views) of the kept graph, 0 if each view has its own. */
vsr_status vsr_batch_config_ex(vsr_batch b, int* streams, int* graphed, int* split_max, int* pooled);
/* Graph kinds the autotuner may keep: VSR_BATCH_AUTO (both; the default),
 * VSR_BATCH_CHAINS (per-view raster launches only) or VSR_BATCH_POOLED (the
 * pooled raster launch only).  A change takes effect at the next render,
 * which tunes again.  VSR_ERR_INVALID_ARG for another value. */
enum { VSR_BATCH_AUTO = 0, VSR_BATCH_CHAINS = 1, VSR_BATCH_POOLED = 2 };
vsr_status vsr_batch_set_mode(vsr_batch b, int mode);
void vsr_batch_free(vsr_batch b);

/* ---- serving ------------------------------------------------------------------
 * A rendering server with continuous batching.  A worker thread owns `slots`
 * CUDA streams; submitted requests wait in a FIFO queue and are admitted into
 * free slots as soon as a slot and device memory allow, while earlier
 * requests still run, so their launches overlap on the GPU.  Each request is
 * rendered exactly as vsr_raster renders it alone (its map, its camera's
 * set-up, its bins), on a workspace of its slot.  Maps come from an LRU cache
 * keyed by the exact lens parameters and size; entries in use are never
 * evicted.  Device memory of cached maps and slot workspaces is held under
 * `budget_bytes`: a request needing more evicts idle maps, waits while other
 * requests run, and fails with VSR_ERR_BUDGET if it cannot fit alone.  A
 * request whose bins outgrew their capacity is rendered again with grown
 * bins (counted in `reruns`; the server's workspaces report to status words
 * of their own, so vsr_last_device_status does not see them).  Completion is polled on the host; no device
 * code waits.  Timestamps are seconds of one steady clock (vsr_serve_now). */
typedef struct vsr_server_s* vsr_server;
typedef struct {
    int64_t budget_bytes; /* device memory for maps and workspaces */
    int slots;            /* requests in flight at once (one stream each), 1..32 */
    int max_maps;         /* map-cache entries, 0 = limited by the budget only */
} vsr_serve_cfg;
typedef struct {
    int scene;            /* index from vsr_serve_add_scene */
    vsr_map_params lens;  /* the request's map (W, H included) */
    float cam[12];        /* camera as in vsr_setup */
    uint32_t* id_dev;     /* caller-owned device outputs [lens.H][lens.W]; */
    float* depth_dev;     /* any may be NULL; must stay valid until the */
    float* cov_dev;       /* request is done */
} vsr_request;
typedef struct {
    vsr_status status;    /* VSR_OK, VSR_ERR_CANCELLED, VSR_ERR_BUDGET, ... */
    int done;             /* 1 once final (then the ticket is released) */
    int map_cache_hit;
    double t_submit, t_start, t_done;
} vsr_result;
typedef struct {
    int64_t submitted, completed, failed, cancelled;
    int64_t map_hits, map_misses, map_evictions, reruns;
    int64_t bytes_in_use, maps_cached, queued;
} vsr_serve_stats;

vsr_status vsr_serve_create(const vsr_serve_cfg* cfg, vsr_server* out);
/* Register resident triangles (device [T][3][3], caller-owned, kept alive by
 * the caller while the server lives); returns its scene index. */
vsr_status vsr_serve_add_scene(vsr_server s, const float* tris_dev, int64_t T, int* scene);
/* Queue a request (non-blocking).  VSR_ERR_INVALID_ARG for bad parameters
 * or scene, VSR_ERR_BUDGET if its map alone exceeds the budget. */
vsr_status vsr_serve_submit(vsr_server s, const vsr_request* r, uint64_t* ticket);
/* Non-blocking: out->done = 0 while pending. */
vsr_status vsr_serve_poll(vsr_server s, uint64_t ticket, vsr_result* out);
/* Blocks until the request is final. */
vsr_status vsr_serve_wait(vsr_server s, uint64_t ticket, vsr_result* out);
/* Cancels a request still in the queue (VSR_ERR_INVALID_ARG once running). */
vsr_status vsr_serve_cancel(vsr_server s, uint64_t ticket);
vsr_status vsr_serve_stats_get(vsr_server s, vsr_serve_stats* out);
double vsr_serve_now(void);
/* Finishes the queued and running requests, then frees everything. */
vsr_status vsr_serve_destroy(vsr_server s);

/* ---- differentiable rendering ----------------------------------------------
 * A shaded image and its hand-written adjoint.  The image is the
 * front-to-back mask merge of Sec. 1.4 applied to a shade pass
 *   I = sum over the fragments of a pixel in ascending (r, t) of
 *       m^fc shade,  m^fc = min(m^f, 1 - m^b),  m^b += m^fc,
 *   shade_t = c_t |N-hat_t . G|   (N-hat the hard normal of Sec. 1.1.4),
 * with the fragments, m^f (gpstep on the four plane distances, Sec. 1.1.1
 * and 1.1.2) and depth of vsr_raster.  The merge depends on the order, so
 * the forward keeps every fragment of every pixel in a fragment-list handle
 * that the backward reads.
 *
 * vsr_frags: library-owned fragment lists and backward workspace; grows to
 * the largest frame it has seen.  One frame at a time: a forward replaces
 * the lists of the previous one. */
typedef struct vsr_frags_s* vsr_frags;
vsr_status vsr_frags_create(vsr_frags* out);
void vsr_frags_free(vsr_frags f);

/* vsr_raster_shaded: bins (as vsr_raster), counts the fragments of every
 * pixel, sizes the lists (one synchronisation of `stream` per call: the
 * fragment total is read back), fills, sorts and merges them.
 * colors_dev: device [T] colour c_t per triangle (NULL: all 1).
 * Outputs (caller-owned device [H][W], any may be NULL): image_dev (I),
 * cov_dev (final m^b of the merge: the coverage of vsr_raster within
 * rounding), id_dev and depth_dev (as vsr_raster).  At most 2^32 - 1
 * fragments per frame.  Errors: VSR_ERR_INVALID_ARG, VSR_ERR_OOM,
 * VSR_ERR_CUDA; device-side VSR_ERR_BIN_OVERFLOW / VSR_ERR_FRAG_OVERFLOW in
 * the status word. */
vsr_status vsr_raster_shaded(vsr_map m, vsr_scene s, const float* colors_dev, vsr_frags f, float* image_dev,
                             float* cov_dev, uint32_t* id_dev, float* depth_dev, void* stream);

/* vsr_raster_backward: the adjoint of the last vsr_raster_shaded of (m, s)
 * into f.  Upstream gradients (device [H][W], NULL = 0): dimage_dev = dL/dI,
 * dcov_dev = dL/dcov, ddepth_dev = dL/ddepth (through r = (A'.N)/(G.N) of
 * the visible triangle, Sec. 1.1.4; the visibility switch itself has no
 * gradient).  id_dev: that forward's id output (needed with ddepth_dev).
 * tris_dev: the world triangles [T][3][3] of the scene's current set-up
 * (the camera is the scene's).  Outputs (device, overwritten, NULL to
 * skip): dtris_dev [T][3][3] = dL/d(world vertices), dcolors_dev [T] =
 * dL/dc_t, dlens_dev (double [4]) = dL/d(k, l, s, Omega in degrees) of the
 * map at its effective parameters (after the limits; a map made by
 * vsr_map_from_device, a distorted map or another kind of vsr_make_map_spec
 * has none: VSR_ERR_INVALID_ARG).
 * The adjoint follows the forward exactly: the merge (saturation at the
 * first fragment with m^f > 1 - m^b), gpstep / min (the gradient goes to
 * the minimising plane distance while its clamp is open), the plane
 * distances g_1..3 = G.n_i and g_4 = (G.S-hat - cos rho)/sin rho, the
 * set-up (edge normals, smallest circle, plane, camera transform) and the
 * map (2D->3D transform and global delta).  Per-triangle sums use float
 * atomics (their order, hence the last bits, varies between runs).
 * VSR_ERR_INVALID_ARG if f holds no forward of this map and set-up. */
vsr_status vsr_raster_backward(vsr_map m, vsr_scene s, const float* tris_dev, const float* colors_dev, vsr_frags f,
                               const uint32_t* id_dev, const float* dimage_dev, const float* dcov_dev,
                               const float* ddepth_dev, float* dtris_dev, float* dcolors_dev, double* dlens_dev,
                               void* stream);

/* ---- status ---------------------------------------------------------------- */
const char* vsr_status_str(vsr_status s);
/* Synchronises the device, returns and clears the device-side status word
 * (VSR_OK when nothing was raised). */
vsr_status vsr_last_device_status(void);
/* Library version string. */
const char* vsr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VSR_H */
