// handles.cuh -- the library's handle structures and host helpers, shared
// by the host files of the library (api.cu, serve.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vsr_internal.cuh"

// The device-side status word of the current device (allocated and zeroed
// on first use).
int* status_word();

template <class Tp>
inline vsr_status dalloc(Tp** p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc((void**)p, n * sizeof(Tp)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return VSR_ERR_OOM;
    }
    return VSR_OK;
}

struct vsr_map_s {
    vsr_map_params p;  // effective parameters
    vsr_map_spec spec = {};  // the projection (kind VSR_MAP_UNIVERSAL with no distortion for vsr_make_map*)
    bool lens_grad = true;   // the lens gradient of vsr_raster_backward applies (undistorted Universal)
    float4* deriv = nullptr; // 2 float4 per pixel with VSR_MAP_DERIVATIVES
    float4* map = nullptr;
    Cone* tiles = nullptr;
    // tile geometry and widest ramp (every generation), and the tile index
    // of the triangle-major search, built for the current generation on
    // first use (vsr_raster_noalloc)
    TileIndex idx = {};
    bool idx_built = false;
    uint32_t hgen = 0;  // generation of the widest-ramp word (idx.hdr->h_gen)
    int tx = 0, ty = 0;
    uint64_t gen = 0;
};

struct vsr_scene_s {
    int64_t T = 0;
    float cam[12] = {};  // camera of the current set-up
    int64_t T_alloc = 0;
    float4* rec = nullptr;
    uint64_t gen = 0;
    // bin workspace
    int ws_tiles = 0;
    // bins: tile-major, tile u's at ids[offsets[u] .. ends[u]) (offsets[ntiles]:
    // the total); triangle-major, in tile order at ids[offsets[u] ..
    // offsets[u + 1]), `ends` holding the count pass's counters and cursor
    bool tile_major = false;
    uint32_t* offsets = nullptr;  // ntiles + 1
    uint32_t* ends = nullptr;     // ntiles + 1
    uint32_t* ids = nullptr;
    uint2* pairs = nullptr;  // (tile, triangle) of every hit of the triangle-major count pass, cap entries
    uint32_t cap = 0;
    TriIndex tri = {};  // the frame's triangles by cap cell (tile-major binning)
    uint64_t sized_shape = 0;           // (tiles, T) the bins were last sized for
    uint32_t* h_total = nullptr;        // pinned: pair total of a recent binning
    uint32_t* h_total_dev = nullptr;    // its device address (the scan kernel stores the total there)
    cudaEvent_t total_event = nullptr;  // completion of that copy
    bool total_pending = false;
    uint64_t total_map = 0, total_scene = 0;  // generations of the binning whose total it is
    int last_ntiles = 0;
    uint64_t binned_map = 0, binned_scene = 0;  // generations the current bins belong to
    RasterWork work = {};
    uint32_t work_tiles = 0;
    // host-path buffers (vsr_render_host)
    float* tris_dev = nullptr;
    int64_t tris_alloc = 0;
    void* out_dev = nullptr;  // id | depth | cov staging, 12 B per pixel
    size_t out_alloc = 0;
    // device status word of this scene's kernels: NULL = the per-device word
    // of vsr_last_device_status; the server gives its workspaces their own
    int* status = nullptr;
    // bins sized without waiting for the device when the map's shape changes
    // (the capacity of earlier binnings is kept and only grows): an owner
    // that renders a request again after a bin overflow (the server) needs
    // no synchronisation per new shape; everyone else gets exact bins on
    // every call
    bool async_sizing = false;
    // vsr_render_host runs the set-up on a stream of the scene's own, beside
    // work the caller queued before the call that does not touch the scene
    // (a map update).  From its first call on, use_event is recorded after
    // every queued use of the scene's buffers, so that stream waits for
    // exactly those.
    cudaStream_t side = nullptr;
    cudaEvent_t use_event = nullptr;
    cudaEvent_t setup_event = nullptr;
    // its device status word: a frame that outgrew its bins is rendered
    // again, so the overflow it raised goes here, not to the per-device word
    int* host_status = nullptr;
    // vsr_render_host_async: the frame's completion, whether one is queued
    // and not yet waited for, and the map generation it was binned against
    cudaEvent_t host_done = nullptr;
    bool host_pending = false;
    uint64_t host_map_gen = 0;
};

inline int* scene_status(const vsr_scene_s* s) { return s->status ? s->status : status_word(); }

// the bins' end array for the raster views (NULL: bins in tile order)
inline const uint32_t* scene_ends(const vsr_scene_s* s) { return s->tile_major ? s->ends : nullptr; }

// triangles per tile up to which a scene is binned tile-major: 27 on the
// 1080p single-view frame (220k triangles, bin stage 65.8 -> ~40 us against
// the triangle-major search); 122-977 on the batched views' 1M triangles,
// where the tile-major walk was slower (tiles few and wide)
constexpr int64_t TILE_MAJOR_TRIS_PER_TILE = 64;

// Note a use of the scene's buffers queued on st (see use_event).
inline vsr_status scene_used(vsr_scene_s* s, cudaStream_t st)
{
    if (!s->use_event) return VSR_OK;
    // uses inside a stream capture run when their graph is launched: the
    // caller orders those launches
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return VSR_ERR_CUDA;
    }
    if (cs == cudaStreamCaptureStatusNone && cudaEventRecord(s->use_event, st) != cudaSuccess) {
        cudaGetLastError();
        return VSR_ERR_CUDA;
    }
    return VSR_OK;
}
