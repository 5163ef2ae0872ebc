// api.cu -- host side of the C ABI declared in include/vsr.h: handles,
// device memory, argument checks and the launch sequence of one frame
//   map (once per lens) -> set-up (once per scene/camera) -> bin count ->
//   scan -> bin fill -> tile raster.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <vector>
#include <mutex>

#include "handles.cuh"

namespace {

std::atomic<uint64_t> g_gen{1};
std::mutex g_status_mu;
int* g_status[256] = {};

}  // namespace

int* status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status[dev]) {
        int* p = nullptr;
        if (cudaMalloc((void**)&p, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        g_status[dev] = p;
    }
    return g_status[dev];
}

namespace {

bool finite4(float a, float b, float c, float d) { return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d); }

void apply_limits(vsr_map_params* p)
{
    // Sec. 2, "Universal perspective parameters and limits"
    float k = fminf(1.0f, fmaxf(-1.0f, p->k));
    float l = fminf(1.0f, fmaxf(0.0f, p->l));
    float s = fminf(1.0f, fmaxf(p->strict_limits ? 0.8f : 0.5f, p->s));
    float kmag = fabsf(k) > 0.5f ? fabsf(k) : 0.5f;
    float omax = (k > 0.0f ? 179.0f : 180.0f) / kmag;
    float om = fminf(omax, fmaxf(1.0f, p->omega_deg));
    p->k = k;
    p->l = l;
    p->s = s;
    p->omega_deg = om;
}

vsr_status map_alloc(vsr_map m, int W, int H)
{
    m->tx = (W + TILE - 1) / TILE;
    m->ty = (H + TILE - 1) / TILE;
    const size_t nt = (size_t)m->tx * m->ty;
    vsr_status st;
    if ((st = dalloc(&m->map, (size_t)W * H)) != VSR_OK) return st;
    if ((st = dalloc(&m->tiles, nt)) != VSR_OK) return st;
    if ((st = dalloc(&m->idx.hdr, 1)) != VSR_OK) return st;
    if ((st = dalloc(&m->idx.cell_start, (size_t)IDX_CELLS_MAX + 1)) != VSR_OK) return st;
    if ((st = dalloc(&m->idx.sorted, nt)) != VSR_OK) return st;
    if ((st = dalloc(&m->idx.big, nt)) != VSR_OK) return st;
    if ((st = dalloc(&m->idx.geom, nt)) != VSR_OK) return st;
    m->idx.ntiles = (uint32_t)nt;
    m->idx_built = false;
    m->hgen = 0;  // the first generation clears the widest-ramp word
    if ((m->spec.flags & VSR_MAP_DERIVATIVES) && (st = dalloc(&m->deriv, 2 * (size_t)W * H)) != VSR_OK) return st;
    return VSR_OK;
}

void map_release(vsr_map m)
{
    if (!m) return;
    cudaFree(m->map);
    cudaFree(m->tiles);
    cudaFree(m->idx.hdr);
    cudaFree(m->idx.cell_start);
    cudaFree(m->idx.sorted);
    cudaFree(m->idx.big);
    cudaFree(m->idx.geom);
    cudaFree(m->deriv);
    m->deriv = nullptr;
    m->map = nullptr;
    m->idx_built = false;
    m->tiles = nullptr;
    m->idx = TileIndex{};
}

// Device address of host memory that kernels can read and write in place
// (pinned and mapped into the current device's address space), else NULL.
void* mapped_host(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

bool size_ok(int W, int H) { return W >= 1 && H >= 1 && W <= 32768 && H <= 32768; }

vsr_status check_params(const vsr_map_params* p)
{
    if (!p) return VSR_ERR_INVALID_ARG;
    if (!size_ok(p->W, p->H)) return VSR_ERR_INVALID_ARG;
    if (!finite4(p->k, p->l, p->s, p->omega_deg)) return VSR_ERR_INVALID_ARG;
    if (p->aov < 0 || p->aov > 3) return VSR_ERR_INVALID_ARG;
    return VSR_OK;
}

// the spec of a plain Universal map with m->p's (effective) parameters
void set_universal_spec(vsr_map m)
{
    const int flags = m->spec.flags;
    m->spec = vsr_map_spec{};
    m->spec.flags = flags;
    m->spec.kind = VSR_MAP_UNIVERSAL;
    m->spec.W = m->p.W;
    m->spec.H = m->p.H;
    m->spec.aov = m->p.aov;
    m->spec.param[0] = m->p.k;
    m->spec.param[1] = m->p.l;
    m->spec.param[2] = m->p.s;
    m->spec.param[3] = m->p.omega_deg;
    m->lens_grad = true;
}

// the next generation of the map's widest-ramp word: the first one (of
// new memory, or after 2^32 - 1 of them) clears the word on st first
vsr_status next_hgen(vsr_map m, cudaStream_t st)
{
    if (m->hgen == 0 || m->hgen == 0xffffffffu) {
        VSR_CUDA_TRY(cudaMemsetAsync(&m->idx.hdr->h_gen, 0, sizeof(unsigned long long), st));
        m->hgen = 0;
    }
    ++m->hgen;
    return VSR_OK;
}

// One generation of the map: the map kernel writes the map, the tile cones
// and geometry and the widest ramp, all the tile-major binner needs; the
// tile index of the triangle-major search is left to its first use.
vsr_status map_generate(vsr_map m, cudaStream_t st)
{
    bool plain = m->spec.kind == VSR_MAP_UNIVERSAL && !m->deriv;
    for (int q = 0; q < 6; ++q) plain = plain && m->spec.distortion[q] == 0.0f;
    m->idx_built = false;
    vsr_status s = next_hgen(m, st);
    if (s != VSR_OK) return s;
    s = plain ? launch_map(m->p.W, m->p.H, m->p.aov, m->p.k, m->p.l, m->p.s, m->p.omega_deg, m->map, m->tiles,
                           m->idx.geom, &m->idx.hdr->h_gen, m->hgen, st)
              : launch_map_spec(m->spec, m->map, m->tiles, m->idx.geom, m->deriv, &m->idx.hdr->h_gen, m->hgen, st);
    m->gen = g_gen.fetch_add(1);
    return s;
}

// the tile index of the map's current generation (built on first use)
vsr_status ensure_tile_index(vsr_map m, cudaStream_t st)
{
    if (m->idx_built) return VSR_OK;
    vsr_status s = launch_tile_index(m->tiles, m->tx * m->ty, m->idx, st);
    if (s == VSR_OK) m->idx_built = true;
    return s;
}

vsr_status scene_setup(vsr_scene sc, const float* tris_dev, int64_t T, const float cam[12], cudaStream_t st)
{
    if (T > sc->T_alloc) {
        cudaFree(sc->rec);
        sc->rec = nullptr;
        sc->T_alloc = 0;
        vsr_status s = dalloc(&sc->rec, (size_t)REC_F * (size_t)T);
        if (s != VSR_OK) return s;
        sc->T_alloc = T;
    }
    sc->T = T;
    for (int q = 0; q < 12; ++q) sc->cam[q] = cam[q];
    // the record layout is field-major with stride T: keep it dense
    vsr_status s = launch_setup(tris_dev, (int)T, cam, sc->rec, st);
    sc->gen = g_gen.fetch_add(1);
    return s == VSR_OK ? scene_used(sc, st) : s;
}

// bin ids and the triangle-major count pass's pair list, both of `want`
// entries (frees the old ones, which waits for the launches still using
// them)
vsr_status bins_realloc(vsr_scene sc, uint32_t want)
{
    cudaFree(sc->ids);
    cudaFree(sc->pairs);
    sc->ids = nullptr;
    sc->pairs = nullptr;
    sc->cap = 0;
    vsr_status s;
    if ((s = dalloc(&sc->ids, (size_t)want)) != VSR_OK) return s;
    if ((s = dalloc(&sc->pairs, (size_t)want)) != VSR_OK) {
        cudaFree(sc->ids);
        sc->ids = nullptr;
        return s;
    }
    sc->cap = want;
    return VSR_OK;
}

vsr_status ensure_ws(vsr_scene sc, int ntiles)
{
    if (ntiles <= sc->ws_tiles) return VSR_OK;
    cudaFree(sc->ends);
    cudaFree(sc->offsets);
    sc->ends = sc->offsets = nullptr;
    sc->ws_tiles = 0;
    vsr_status s;
    if ((s = dalloc(&sc->ends, (size_t)ntiles + 1)) != VSR_OK) return s;  // (+1: the triangle-major pair cursor)
    if ((s = dalloc(&sc->offsets, (size_t)ntiles + 1)) != VSR_OK) return s;
    sc->ws_tiles = ntiles;
    sc->sized_shape = 0;
    return VSR_OK;
}

}  // namespace

extern "C" {

const char* vsr_version(void) { return "vsr 0.1 (sm_103a)"; }

const char* vsr_status_str(vsr_status s)
{
    switch (s) {
    case VSR_OK: return "ok";
    case VSR_ERR_INVALID_ARG: return "invalid argument";
    case VSR_ERR_OOM: return "out of memory";
    case VSR_ERR_CUDA: return "CUDA error";
    case VSR_ERR_BIN_OVERFLOW: return "tile bin overflow";
    case VSR_ERR_FRAG_OVERFLOW: return "fragment list overflow";
    case VSR_ERR_TIMEOUT: return "device wait timed out";
    case VSR_ERR_BUDGET: return "memory budget exceeded";
    case VSR_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

vsr_status vsr_last_device_status(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return VSR_ERR_CUDA;
    int* w = status_word();
    if (!w) return VSR_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return VSR_ERR_CUDA;
    if (cudaMemset(w, 0, sizeof(int)) != cudaSuccess) return VSR_ERR_CUDA;
    return (vsr_status)v;
}

vsr_status vsr_make_map_ex(const vsr_map_params* p, void* stream, vsr_map* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    vsr_status s = check_params(p);
    if (s != VSR_OK) return s;
    vsr_map m = new (std::nothrow) vsr_map_s;
    if (!m) return VSR_ERR_OOM;
    m->p = *p;
    apply_limits(&m->p);
    set_universal_spec(m);
    if ((s = map_alloc(m, p->W, p->H)) != VSR_OK || (s = map_generate(m, (cudaStream_t)stream)) != VSR_OK) {
        map_release(m);
        delete m;
        return s;
    }
    *out = m;
    return VSR_OK;
}

vsr_status vsr_make_map(float k, float l, float s, float omega_deg, int W, int H, void* stream, vsr_map* out)
{
    vsr_map_params p;
    p.k = k;
    p.l = l;
    p.s = s;
    p.omega_deg = omega_deg;
    p.W = W;
    p.H = H;
    p.aov = VSR_AOV_HORIZONTAL;
    p.strict_limits = 0;
    return vsr_make_map_ex(&p, stream, out);
}

vsr_status vsr_make_map_spec(const vsr_map_spec* sp, void* stream, vsr_map* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!sp || !size_ok(sp->W, sp->H) || sp->kind < VSR_MAP_UNIVERSAL || sp->kind > VSR_MAP_CUBE || sp->aov < 0 ||
        sp->aov > 3)
        return VSR_ERR_INVALID_ARG;
    for (int q = 0; q < 4; ++q)
        if (!isfinite(sp->param[q])) return VSR_ERR_INVALID_ARG;
    bool undistorted = true;
    for (int q = 0; q < 6; ++q) {
        if (!isfinite(sp->distortion[q])) return VSR_ERR_INVALID_ARG;
        undistorted = undistorted && sp->distortion[q] == 0.0f;
    }
    if (sp->kind == VSR_MAP_RECTILINEAR && !(sp->param[0] > 0.0f && sp->param[0] < 180.0f)) return VSR_ERR_INVALID_ARG;
    if (sp->flags & ~VSR_MAP_DERIVATIVES) return VSR_ERR_INVALID_ARG;
    if (sp->kind == VSR_MAP_PANORAMA && !(sp->param[0] > 0.0f && sp->param[1] >= 0.0f)) return VSR_ERR_INVALID_ARG;
    vsr_map m = new (std::nothrow) vsr_map_s;
    if (!m) return VSR_ERR_OOM;
    memset(&m->p, 0, sizeof(m->p));
    m->p.W = sp->W;
    m->p.H = sp->H;
    m->p.aov = sp->aov;
    m->spec = *sp;
    if (sp->kind == VSR_MAP_UNIVERSAL) {
        m->p.k = sp->param[0];
        m->p.l = sp->param[1];
        m->p.s = sp->param[2];
        m->p.omega_deg = sp->param[3];
        apply_limits(&m->p);
        m->spec.param[0] = m->p.k;
        m->spec.param[1] = m->p.l;
        m->spec.param[2] = m->p.s;
        m->spec.param[3] = m->p.omega_deg;
        m->lens_grad = undistorted;
    } else {
        m->p.k = m->p.l = m->p.s = m->p.omega_deg = NAN;
        m->lens_grad = false;
    }
    vsr_status s;
    if ((s = map_alloc(m, sp->W, sp->H)) != VSR_OK || (s = map_generate(m, (cudaStream_t)stream)) != VSR_OK) {
        map_release(m);
        delete m;
        return s;
    }
    *out = m;
    return VSR_OK;
}

vsr_status vsr_map_update(vsr_map m, const vsr_map_params* p, void* stream)
{
    if (!m) return VSR_ERR_INVALID_ARG;
    vsr_status s = check_params(p);
    if (s != VSR_OK) return s;
    if (p->W != m->p.W || p->H != m->p.H) {
        map_release(m);
        if ((s = map_alloc(m, p->W, p->H)) != VSR_OK) return s;
    }
    m->p = *p;
    apply_limits(&m->p);
    set_universal_spec(m);
    return map_generate(m, (cudaStream_t)stream);
}

vsr_status vsr_map_from_device(const float* xyzd_dev, int W, int H, void* stream, vsr_map* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!xyzd_dev || !size_ok(W, H)) return VSR_ERR_INVALID_ARG;
    vsr_map m = new (std::nothrow) vsr_map_s;
    if (!m) return VSR_ERR_OOM;
    memset(&m->p, 0, sizeof(m->p));
    m->p.W = W;
    m->p.H = H;
    m->p.k = m->p.l = m->p.s = m->p.omega_deg = NAN;
    m->lens_grad = false;
    vsr_status s = map_alloc(m, W, H);
    cudaStream_t st = (cudaStream_t)stream;
    if (s == VSR_OK && cudaMemcpyAsync(m->map, xyzd_dev, sizeof(float4) * (size_t)W * H, cudaMemcpyDeviceToDevice,
                                       st) != cudaSuccess)
        s = VSR_ERR_CUDA;
    if (s == VSR_OK) s = next_hgen(m, st);
    if (s == VSR_OK) s = launch_map_cones(m->map, W, H, m->tiles, m->idx.geom, &m->idx.hdr->h_gen, m->hgen, st);
    if (s != VSR_OK) {
        map_release(m);
        delete m;
        return s;
    }
    m->gen = g_gen.fetch_add(1);
    *out = m;
    return VSR_OK;
}

vsr_status vsr_map_params_effective(vsr_map m, vsr_map_params* out)
{
    if (!m || !out) return VSR_ERR_INVALID_ARG;
    *out = m->p;
    return VSR_OK;
}

vsr_status vsr_map_data(vsr_map m, const float** xyzd_dev, int* W, int* H)
{
    if (!m) return VSR_ERR_INVALID_ARG;
    if (xyzd_dev) *xyzd_dev = (const float*)m->map;
    if (W) *W = m->p.W;
    if (H) *H = m->p.H;
    return VSR_OK;
}

vsr_status vsr_map_download(vsr_map m, float* host_xyzd)
{
    if (!m || !host_xyzd) return VSR_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return VSR_ERR_CUDA;
    if (cudaMemcpy(host_xyzd, m->map, sizeof(float4) * (size_t)m->p.W * m->p.H, cudaMemcpyDeviceToHost) != cudaSuccess)
        return VSR_ERR_CUDA;
    return VSR_OK;
}

vsr_status vsr_map_download_derivatives(vsr_map m, float* host)
{
    if (!m || !host || !m->deriv) return VSR_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return VSR_ERR_CUDA;
    if (cudaMemcpy(host, m->deriv, 2 * sizeof(float4) * (size_t)m->p.W * m->p.H, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return VSR_ERR_CUDA;
    return VSR_OK;
}

void vsr_map_free(vsr_map m)
{
    if (!m) return;
    map_release(m);
    delete m;
}

vsr_status vsr_scene_create(vsr_scene* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    vsr_scene sc = new (std::nothrow) vsr_scene_s;
    if (!sc) return VSR_ERR_OOM;
    if (cudaMallocHost((void**)&sc->h_total, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete sc;
        return VSR_ERR_OOM;
    }
    *sc->h_total = 0;
    sc->h_total_dev = (uint32_t*)mapped_host(sc->h_total);
    if (!sc->h_total_dev || cudaEventCreateWithFlags(&sc->total_event, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(sc->h_total);
        delete sc;
        return VSR_ERR_CUDA;
    }
    *out = sc;
    return VSR_OK;
}

static bool setup_args_ok(const float* tris, int64_t T, const float* cam)
{
    if (T < 0 || T >= 0x7fffffffLL || (T > 0 && !tris) || !cam) return false;
    for (int q = 0; q < 12; ++q)
        if (!isfinite(cam[q])) return false;
    return true;
}

vsr_status vsr_setup(const float* tris_dev, int64_t T, const float cam[12], void* stream, vsr_scene* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!setup_args_ok(tris_dev, T, cam)) return VSR_ERR_INVALID_ARG;
    vsr_scene sc;
    vsr_status s = vsr_scene_create(&sc);
    if (s != VSR_OK) return s;
    s = scene_setup(sc, tris_dev, T, cam, (cudaStream_t)stream);
    if (s != VSR_OK) {
        vsr_scene_free(sc);
        return s;
    }
    *out = sc;
    return VSR_OK;
}

vsr_status vsr_scene_update(vsr_scene sc, const float* tris_dev, int64_t T, const float cam[12], void* stream)
{
    if (!sc || !setup_args_ok(tris_dev, T, cam)) return VSR_ERR_INVALID_ARG;
    return scene_setup(sc, tris_dev, T, cam, (cudaStream_t)stream);
}

void vsr_scene_free(vsr_scene sc)
{
    if (!sc) return;
    cudaFree(sc->rec);
    cudaFree(sc->ends);
    cudaFree(sc->offsets);
    cudaFree(sc->ids);
    cudaFree(sc->pairs);
    tri_index_free(&sc->tri);
    raster_work_free(&sc->work);
    cudaFree(sc->tris_dev);
    cudaFree(sc->out_dev);
    if (sc->total_event) {
        cudaEventSynchronize(sc->total_event);
        cudaEventDestroy(sc->total_event);
    }
    if (sc->h_total) cudaFreeHost(sc->h_total);
    if (sc->host_done) {
        cudaEventSynchronize(sc->host_done);
        cudaEventDestroy(sc->host_done);
    }
    if (sc->side) cudaStreamDestroy(sc->side);
    if (sc->use_event) cudaEventDestroy(sc->use_event);
    if (sc->setup_event) cudaEventDestroy(sc->setup_event);
    cudaFree(sc->host_status);
    delete sc;
}

int64_t vsr_scene_size(vsr_scene sc) { return sc ? sc->T : -1; }

static vsr_status bin_scene(vsr_map m, vsr_scene sc, int pstep, cudaStream_t st);

vsr_status vsr_bin(vsr_map m, vsr_scene sc, void* stream)
{
    if (!m || !sc) return VSR_ERR_INVALID_ARG;
    return bin_scene(m, sc, 0, (cudaStream_t)stream);
}

vsr_status vsr_raster_pstep(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev, void* stream)
{
    if (!m || !sc || !m->deriv) return VSR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    vsr_status s = bin_scene(m, sc, 1, st);
    if (s != VSR_OK) return s;
    const RasterView v{m->map,  m->p.W, m->p.H, m->tiles, m->tx,     sc->rec,   (int)sc->T, sc->offsets,
                       sc->ids, sc->cap, id_dev, depth_dev, cov_dev, scene_ends(sc)};
    s = launch_raster_pstep(v, m->deriv, scene_status(sc), st);
    return s == VSR_OK ? scene_used(sc, st) : s;
}

}  // extern "C"

static vsr_status bin_scene(vsr_map m, vsr_scene sc, int pstep, cudaStream_t st)
{
    const int ntiles = m->tx * m->ty;
    vsr_status s = ensure_ws(sc, ntiles);
    if (s != VSR_OK) return s;
    const int T = (int)sc->T;
    sc->last_ntiles = ntiles;
    // The binner: tile-major while the triangles are few per tile (each
    // tile's warp then walks a short window), else the triangle-major search
    // over the map's tile index (its work spread over the triangles).
    sc->tile_major = (int64_t)T <= TILE_MAJOR_TRIS_PER_TILE * (int64_t)ntiles;
    if (sc->tile_major) {
        if ((s = tri_index_alloc(&sc->tri, T, ntiles)) != VSR_OK) return s;
    } else if ((s = ensure_tile_index(m, st)) != VSR_OK) {
        return s;
    }
    // Bin capacity.  Sized synchronously the first time and whenever the
    // number of tiles or triangles changes (the first time only, for a scene
    // with async_sizing); otherwise the pair total of the previous binning
    // (copied to pinned memory, read only once its event has completed, never
    // waited for) grows the capacity ahead of need, and the binning kernels
    // report any overflow in the status word.
    // the bins' sizes depend on the map, the scene and the step's cap width
    const uint64_t shape = ((uint64_t)ntiles << 32) ^ (uint64_t)sc->T ^ ((uint64_t)(pstep != 0) << 63);
    const bool resize = sc->cap == 0 || (!sc->async_sizing && sc->sized_shape != shape);
    if (!resize && sc->total_pending && cudaEventQuery(sc->total_event) == cudaSuccess) {
        sc->total_pending = false;
        const uint64_t last = *sc->h_total;
        if (last + last / 8 > sc->cap) {
            uint64_t want = last + last / 4 + 4096;
            if (want > 0xffffffffull) want = 0xffffffffull;
            if ((s = bins_realloc(sc, (uint32_t)want)) != VSR_OK) return s;
        }
    }
    // the pair total also goes to the pinned host word (its device address)
    // unless an earlier total has not been read yet -- and always when this
    // binning sizes the bins, which reads this total
    const bool record = resize || !sc->total_pending;
    uint32_t* total_host = record ? sc->h_total_dev : nullptr;
    // triangle-major: per-tile counters and the pair cursor in the end array
    uint32_t* counts = sc->ends;
    uint32_t* cursor = counts + ntiles;
    uint2* pairs = sc->pairs;
    const uint32_t pair_cap = sc->cap;
    if (sc->tile_major) {
        // one pass (a sizing pass reports no overflow: its bins are grown and
        // binned again)
        if ((s = launch_bin_tiles(sc->rec, T, m->idx, m->tiles, ntiles, sc->tri, sc->offsets, sc->ends, sc->ids,
                                  sc->cap, resize ? nullptr : scene_status(sc), total_host, st, pstep)) != VSR_OK)
            return s;
    } else {
        VSR_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ((size_t)ntiles + 1), st));
        if ((s = launch_bin_count(sc->rec, T, m->idx, counts, cursor, pairs, pair_cap, st, pstep)) != VSR_OK)
            return s;
        if ((s = launch_scan(counts, nullptr, ntiles, nullptr, sc->offsets, st, total_host)) != VSR_OK) return s;
    }
    if (record) {
        VSR_CUDA_TRY(cudaEventRecord(sc->total_event, st));
        sc->total_pending = true;
        sc->total_map = m->gen;
        sc->total_scene = sc->gen;
    }
    bool grown = false;
    if (resize) {
        VSR_CUDA_TRY(cudaEventSynchronize(sc->total_event));
        sc->total_pending = false;
        const uint32_t total = *sc->h_total;
        if (total > sc->cap || sc->cap == 0) {
            uint64_t want = (uint64_t)total + total / 4 + 4096;
            if (want > 0xffffffffull) want = 0xffffffffull;
            if ((s = bins_realloc(sc, (uint32_t)want)) != VSR_OK) return s;
            pairs = nullptr;  // this frame's pair list went with the old buffer: search again
            grown = true;
        }
        sc->sized_shape = shape;
    }
    if (sc->tile_major) {
        if (grown && (s = launch_bin_tiles(sc->rec, T, m->idx, m->tiles, ntiles, sc->tri, sc->offsets, sc->ends,
                                           sc->ids, sc->cap, scene_status(sc), nullptr, st, pstep)) != VSR_OK)
            return s;
    } else if ((s = launch_bin_fill(sc->rec, T, m->idx, sc->offsets, counts, cursor, pairs, pair_cap, sc->ids,
                                    sc->cap, scene_status(sc), st, pstep)) != VSR_OK) {
        return s;
    }
    sc->binned_map = m->gen;
    sc->binned_scene = sc->gen;
    return scene_used(sc, st);
}

// host_out: the outputs are pinned host memory written in place
static vsr_status raster_tiles(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                               const vsr_raster_stats* stats, void* stream, bool host_out)
{
    if (!m || !sc) return VSR_ERR_INVALID_ARG;
    if (sc->binned_map != m->gen || sc->binned_scene != sc->gen) return VSR_ERR_INVALID_ARG;
    const uint32_t ntiles = (uint32_t)(m->tx * m->ty);
    if (!stats || (!stats->n_alg_dev && !stats->n_exec_dev && !stats->n_inside_dev)) {
        // timed path: work items, large bins split over several CTAs
        if (ntiles > sc->work_tiles) {
            raster_work_free(&sc->work);
            sc->work_tiles = 0;
            vsr_status s = raster_work_alloc(&sc->work, ntiles);
            if (s != VSR_OK) return s;
            sc->work_tiles = ntiles;
        }
        const RasterView v{m->map,  m->p.W, m->p.H, m->tiles, m->tx,     sc->rec,   (int)sc->T, sc->offsets,
                           sc->ids, sc->cap, id_dev, depth_dev, cov_dev, scene_ends(sc)};
        const vsr_status s = launch_raster_items(v, sc->offsets, ntiles, sc->cap, sc->work, SPLIT_MAX_DEFAULT,
                                                 scene_status(sc), (cudaStream_t)stream, host_out);
        return s == VSR_OK ? scene_used(sc, (cudaStream_t)stream) : s;
    }
    // diagnostics: one CTA per tile, whole bins, counters
    const vsr_status s =
        launch_raster(m->map, m->p.W, m->p.H, m->tiles, sc->rec, (int)sc->T, sc->offsets, sc->ids, sc->cap, id_dev,
                      depth_dev, cov_dev, stats ? (unsigned long long*)stats->n_alg_dev : nullptr,
                      stats ? (unsigned long long*)stats->n_exec_dev : nullptr, stats ? stats->n_inside_dev : nullptr,
                      scene_status(sc), (cudaStream_t)stream, scene_ends(sc));
    return s == VSR_OK ? scene_used(sc, (cudaStream_t)stream) : s;
}

extern "C" {

vsr_status vsr_raster_tiles(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                            const vsr_raster_stats* stats, void* stream)
{
    return raster_tiles(m, sc, id_dev, depth_dev, cov_dev, stats, stream, false);
}

vsr_status vsr_raster_dense(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                            void* stream)
{
    if (!m || !sc || sc->T < 0) return VSR_ERR_INVALID_ARG;
    const RasterView v{m->map, m->p.W, m->p.H, m->tiles, m->tx, sc->rec, (int)sc->T, nullptr,
                       nullptr, 0u, id_dev, depth_dev, cov_dev};
    const vsr_status s = launch_raster_dense(v, scene_status(sc), (cudaStream_t)stream);
    return s == VSR_OK ? scene_used(sc, (cudaStream_t)stream) : s;
}

vsr_status vsr_raster_ex(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                         const vsr_raster_stats* stats, void* stream)
{
    vsr_status s = vsr_bin(m, sc, stream);
    if (s != VSR_OK) return s;
    return vsr_raster_tiles(m, sc, id_dev, depth_dev, cov_dev, stats, stream);
}

vsr_status vsr_raster(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev, void* stream)
{
    return vsr_raster_ex(m, sc, id_dev, depth_dev, cov_dev, nullptr, stream);
}

vsr_status vsr_scene_bin_pairs(vsr_scene sc, void* stream, int64_t* pairs)
{
    if (!sc || !pairs || sc->last_ntiles == 0) return VSR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    VSR_CUDA_TRY(cudaStreamSynchronize(st));
    const size_t n = (size_t)sc->last_ntiles;
    if (!sc->tile_major) {  // bins in tile order: the scan's total
        uint32_t v = 0;
        VSR_CUDA_TRY(cudaMemcpy(&v, sc->offsets + n, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        *pairs = v;
        return VSR_OK;
    }
    std::vector<uint32_t> b0(n), b1(n);
    VSR_CUDA_TRY(cudaMemcpy(b0.data(), sc->offsets, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    VSR_CUDA_TRY(cudaMemcpy(b1.data(), sc->ends, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    int64_t v = 0;
    for (size_t u = 0; u < n; ++u) v += (int64_t)(b1[u] - b0[u]);
    *pairs = v;
    return VSR_OK;
}

}  // extern "C"

namespace {

// One frame of the host path: the device addresses of the host buffers (or
// of their staging), and whether the raster writes them in place.
struct HostFrame {
    uint32_t* id_d = nullptr;
    float* depth_d = nullptr;
    float* cov_d = nullptr;
    bool stage_id = false, stage_depth = false, stage_cov = false, in_place = false;
    size_t npix = 0;
};

// Queue the front of a host frame: the scene's own stream and events (made
// at the first call), the triangles' copy when they are not addressable in
// place, and the set-up on that stream; `st` then waits for the set-up.
vsr_status host_frame_front(vsr_map m, vsr_scene sc, const float* tris_host, int64_t T, const float cam[12],
                            uint32_t* id_host, float* depth_host, float* cov_host, cudaStream_t st, HostFrame* f)
{
    vsr_status s;
    f->npix = (size_t)m->p.W * m->p.H;
    // Host buffers the GPU can address in place (pinned memory mapped into
    // its address space) are read by the set-up kernel and written by the
    // raster kernel directly over the host link, so the transfers overlap
    // the kernels; other host memory is staged through device buffers.
    const float* tris_src = T > 0 ? (const float*)mapped_host(tris_host) : nullptr;
    f->id_d = (uint32_t*)mapped_host(id_host);
    f->depth_d = (float*)mapped_host(depth_host);
    f->cov_d = (float*)mapped_host(cov_host);
    // The set-up (and the triangles' copy) runs on the scene's own stream and
    // waits only for the scene's last queued use, so it overlaps work queued
    // on `stream` before this call that leaves the scene alone -- a map
    // update; the binning, on `stream`, waits for both.
    if (!sc->side) {
        if (cudaStreamCreateWithFlags(&sc->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sc->use_event, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sc->setup_event, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sc->host_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc((void**)&sc->host_status, sizeof(int)) != cudaSuccess ||
            cudaMemset(sc->host_status, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            if (sc->side) cudaStreamDestroy(sc->side);
            if (sc->use_event) cudaEventDestroy(sc->use_event);
            if (sc->setup_event) cudaEventDestroy(sc->setup_event);
            if (sc->host_done) cudaEventDestroy(sc->host_done);
            cudaFree(sc->host_status);
            sc->side = nullptr;
            sc->use_event = sc->setup_event = sc->host_done = nullptr;
            sc->host_status = nullptr;
            return VSR_ERR_CUDA;
        }
        // uses queued before the tracking began are unknown: this once, the
        // set-up waits for all the work queued on `stream`
        VSR_CUDA_TRY(cudaEventRecord(sc->use_event, st));
    }
    VSR_CUDA_TRY(cudaStreamWaitEvent(sc->side, sc->use_event, 0));
    if (T > 0 && !tris_src) {
        if (T > sc->tris_alloc) {
            cudaFree(sc->tris_dev);
            sc->tris_dev = nullptr;
            sc->tris_alloc = 0;
            if ((s = dalloc(&sc->tris_dev, (size_t)T * 9)) != VSR_OK) return s;
            sc->tris_alloc = T;
        }
        VSR_CUDA_TRY(cudaMemcpyAsync(sc->tris_dev, tris_host, sizeof(float) * 9 * (size_t)T, cudaMemcpyHostToDevice,
                                     sc->side));
        tris_src = sc->tris_dev;
    }
    f->stage_id = id_host && !f->id_d;
    f->stage_depth = depth_host && !f->depth_d;
    f->stage_cov = cov_host && !f->cov_d;
    if (f->stage_id || f->stage_depth || f->stage_cov) {
        if (12 * f->npix > sc->out_alloc) {
            cudaFree(sc->out_dev);
            sc->out_dev = nullptr;
            sc->out_alloc = 0;
            if (cudaMalloc(&sc->out_dev, 12 * f->npix) != cudaSuccess) {
                cudaGetLastError();
                return VSR_ERR_OOM;
            }
            sc->out_alloc = 12 * f->npix;
        }
        if (f->stage_id) f->id_d = (uint32_t*)sc->out_dev;
        if (f->stage_depth) f->depth_d = (float*)((char*)sc->out_dev + 4 * f->npix);
        if (f->stage_cov) f->cov_d = (float*)((char*)sc->out_dev + 8 * f->npix);
    }
    f->in_place = (id_host && !f->stage_id) || (depth_host && !f->stage_depth) || (cov_host && !f->stage_cov);
    if ((s = scene_setup(sc, tris_src, T, cam, sc->side)) != VSR_OK) return s;
    VSR_CUDA_TRY(cudaEventRecord(sc->setup_event, sc->side));
    VSR_CUDA_TRY(cudaStreamWaitEvent(st, sc->setup_event, 0));
    return VSR_OK;
}

// Queue the back of a host frame on `st`: binning and raster, reporting to
// the scene's own status word, then the copies of staged outputs.
vsr_status host_frame_back(vsr_map m, vsr_scene sc, const HostFrame& f, uint32_t* id_host, float* depth_host,
                           float* cov_host, cudaStream_t st)
{
    int* const saved_status = sc->status;
    sc->status = sc->host_status;
    vsr_status s = vsr_bin(m, sc, st);
    if (s == VSR_OK) s = raster_tiles(m, sc, f.id_d, f.depth_d, f.cov_d, nullptr, st, f.in_place);
    sc->status = saved_status;
    if (s == VSR_OK && f.stage_id && cudaMemcpyAsync(id_host, f.id_d, 4 * f.npix, cudaMemcpyDeviceToHost, st))
        s = VSR_ERR_CUDA;
    if (s == VSR_OK && f.stage_depth &&
        cudaMemcpyAsync(depth_host, f.depth_d, 4 * f.npix, cudaMemcpyDeviceToHost, st))
        s = VSR_ERR_CUDA;
    if (s == VSR_OK && f.stage_cov && cudaMemcpyAsync(cov_host, f.cov_d, 4 * f.npix, cudaMemcpyDeviceToHost, st))
        s = VSR_ERR_CUDA;
    if (s != VSR_OK) cudaGetLastError();
    return s;
}

// After the frame completed: did it outgrow its bins (the pair total, stored
// into pinned memory by the scan, above the capacity)?
bool host_frame_outgrew(vsr_scene sc, uint64_t map_gen)
{
    return sc->total_pending && sc->total_map == map_gen && sc->total_scene == sc->gen && *sc->h_total > sc->cap;
}

}  // namespace

extern "C" {

vsr_status vsr_render_host(vsr_map m, vsr_scene sc, const float* tris_host, int64_t T, const float cam[12],
                           uint32_t* id_host, float* depth_host, float* cov_host, void* stream)
{
    if (!m || !sc || !setup_args_ok(tris_host, T, cam)) return VSR_ERR_INVALID_ARG;
    if (sc->host_pending) return VSR_ERR_INVALID_ARG;  // an asynchronous frame of this scene is not waited for
    cudaStream_t st = (cudaStream_t)stream;
    HostFrame f;
    vsr_status s = host_frame_front(m, sc, tris_host, T, cam, id_host, depth_host, cov_host, st, &f);
    if (s != VSR_OK) return s;
    // The call waits for the frame anyway, so a frame that outgrew its bins
    // is rendered again: the next binning grows the bins from its total.
    for (int attempt = 0;; ++attempt) {
        s = host_frame_back(m, sc, f, id_host, depth_host, cov_host, st);
        if (s == VSR_OK && cudaStreamSynchronize(st) != cudaSuccess) s = VSR_ERR_CUDA;
        if (s != VSR_OK || !host_frame_outgrew(sc, m->gen)) break;
        if (attempt == 2) return VSR_ERR_BIN_OVERFLOW;
    }
    if (s != VSR_OK) cudaGetLastError();
    return s;
}

vsr_status vsr_render_host_async(vsr_map m, vsr_scene sc, const float* tris_host, int64_t T, const float cam[12],
                                 uint32_t* id_host, float* depth_host, float* cov_host, void* stream)
{
    if (!m || !sc || !setup_args_ok(tris_host, T, cam)) return VSR_ERR_INVALID_ARG;
    if (sc->host_pending) return VSR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HostFrame f;
    vsr_status s = host_frame_front(m, sc, tris_host, T, cam, id_host, depth_host, cov_host, st, &f);
    if (s == VSR_OK) s = host_frame_back(m, sc, f, id_host, depth_host, cov_host, st);
    if (s != VSR_OK) return s;
    VSR_CUDA_TRY(cudaEventRecord(sc->host_done, st));
    sc->host_pending = true;
    sc->host_map_gen = m->gen;
    return VSR_OK;
}

vsr_status vsr_render_host_wait(vsr_scene sc)
{
    if (!sc) return VSR_ERR_INVALID_ARG;
    if (!sc->host_pending) return VSR_OK;
    sc->host_pending = false;
    if (cudaEventSynchronize(sc->host_done) != cudaSuccess) {
        cudaGetLastError();
        return VSR_ERR_CUDA;
    }
    return host_frame_outgrew(sc, sc->host_map_gen) ? VSR_ERR_BIN_OVERFLOW : VSR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Rasterization without allocation (vsr_raster_noalloc).
//
// Some callers cannot allocate device memory while they render: a host
// framework that owns every byte of device memory and forbids side
// allocations, or a real-time loop that must never wait on cudaMalloc and the
// synchronisation the first vsr_raster of a new (map, scene) pair performs
// to size its bins.  For them the tile bins live in one file-scope device
// array of fixed size instead of the scene's workspace.  The maps and scenes
// are prepared beforehand; the call itself allocates nothing and never
// synchronises.
//
// Limits: map of at most NA_TILES_MAX 16x16 tiles (e.g. 2048 x 2048), at
// most NA_PAIRS_MAX (tile, triangle) bin pairs.  The array takes about
// 4.3 MB on every device that loads the library, until the process exits.
namespace {

constexpr uint32_t NA_TILES_MAX = 16384;
constexpr uint32_t NA_PAIRS_MAX = 1u << 20;
constexpr size_t NA_STATUS_WORDS = 64;  // word 0: status when the caller passes none
constexpr size_t NA_COUNTS = NA_STATUS_WORDS;
constexpr size_t NA_OFFSETS = NA_COUNTS + NA_TILES_MAX;
constexpr size_t NA_IDS = NA_OFFSETS + NA_TILES_MAX + 64;
constexpr size_t NA_WORDS = NA_IDS + NA_PAIRS_MAX;

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

std::mutex g_noalloc_mu;
uint32_t* g_noalloc_addr[256] = {};

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress allocates nothing).
uint32_t* noalloc_scratch(vsr_status* err)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        *err = VSR_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            *err = VSR_ERR_CUDA;
            return nullptr;
        }
        g_noalloc_addr[dev] = (uint32_t*)p;
    }
    return g_noalloc_addr[dev];
}

}  // namespace

extern "C" vsr_status vsr_raster_noalloc(vsr_map m, vsr_scene sc, uint32_t* id_dev, float* depth_dev, float* cov_dev,
                                         int32_t* status_dev, void* stream)
{
    if (!m || !sc) return VSR_ERR_INVALID_ARG;
    const int ntiles = m->tx * m->ty;
    if ((uint32_t)ntiles > NA_TILES_MAX || sc->T < 0) return VSR_ERR_INVALID_ARG;
    vsr_status err = VSR_OK;
    uint32_t* base = noalloc_scratch(&err);
    if (!base) return err;
    cudaStream_t st = (cudaStream_t)stream;
    const int T = (int)sc->T;
    int* status = status_dev ? (int*)status_dev : (int*)base;
    uint32_t* counts = base + NA_COUNTS;
    uint32_t* offsets = base + NA_OFFSETS;
    uint32_t* ids = base + NA_IDS;
    vsr_status s;
    // the array keeps the previous call's contents: clear what starts at zero
    VSR_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    VSR_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)ntiles, st));
    // the triangle-major search over the map's tile index (no pair list: the
    // fill searches again)
    if ((s = ensure_tile_index(m, st)) != VSR_OK) return s;
    if ((s = launch_bin_count(sc->rec, T, m->idx, counts, nullptr, nullptr, 0, st)) != VSR_OK) return s;
    if ((s = launch_scan(counts, nullptr, ntiles, nullptr, offsets, st)) != VSR_OK) return s;
    if ((s = launch_bin_fill(sc->rec, T, m->idx, offsets, counts, nullptr, nullptr, 0, ids, NA_PAIRS_MAX, status,
                             st)) != VSR_OK)
        return s;
    if ((s = launch_raster(m->map, m->p.W, m->p.H, m->tiles, sc->rec, T, offsets, ids, NA_PAIRS_MAX, id_dev,
                           depth_dev, cov_dev, nullptr, nullptr, nullptr, status, st)) != VSR_OK)
        return s;
    return scene_used(sc, st);
}

// ---------------------------------------------------------------------------
// Batched multi-view rendering (vsr_batch_*).
//
// V views of one scene as one CUDA graph: each view is a chain of the
// single-view launches (set-up with the view's camera read from device
// memory, bin count, scan, bin fill, raster work items) on its own
// workspace, and the chains are spread over S parallel streams inside the
// graph, so each view keeps its working set in L2 while independent views
// overlap on the GPU and no launch pays host overhead.  The first call for a
// configuration runs the views eagerly (sizing every view's bins with one
// synchronisation), then captures one graph per candidate (S in {1, 2, 4, 8}
// streams; the views' own raster launches or 1, 4 or 16 pooled ones; then the
// work-item size), times their replays and keeps the fastest (the
// autotuner).  Later calls
// with the same configuration copy the cameras into pinned staging and
// replay.
namespace {

constexpr int BATCH_STREAMS_MAX = 8;

struct BatchView {
    float4* rec = nullptr;
    uint32_t* counts = nullptr;
    uint32_t* offsets = nullptr;
    uint32_t* partials = nullptr;
    uint32_t* ids = nullptr;
    uint2* pairs = nullptr;  // the count pass's hits, cap entries
    uint32_t cap = 0;
    int tiles = 0;
    int64_t T = 0;
    RasterWork work = {};
};

void batch_view_free(BatchView& v)
{
    cudaFree(v.rec);
    cudaFree(v.counts);
    cudaFree(v.offsets);
    cudaFree(v.partials);
    cudaFree(v.ids);
    cudaFree(v.pairs);
    raster_work_free(&v.work);
    v = BatchView{};
}

}  // namespace

struct vsr_batch_s {
    cudaStream_t streams[BATCH_STREAMS_MAX] = {};
    cudaEvent_t fork = nullptr, join[BATCH_STREAMS_MAX] = {};
    cudaEvent_t cams_done = nullptr;
    std::vector<BatchView> views;
    float* cams_dev = nullptr;
    float* cams_host = nullptr;  // pinned
    int cams_alloc = 0;
    uint32_t* h_total = nullptr;  // pinned, one per view
    int totals_alloc = 0;
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    int nstreams = 0;
    int split_max = SPLIT_MAX_DEFAULT;
    int mode = VSR_BATCH_AUTO;
    // the kept graph rasterizes its views in pool_groups pooled launches (0:
    // one raster launch per view)
    int pool_groups = 0;
    // the pooled launches' views, item ranges (per group: its views' starts,
    // then its total) and queue counters (device), and their stream
    PoolView* pool_views = nullptr;
    uint32_t* pool_start = nullptr;
    uint32_t* pool_queue = nullptr;
    int pool_alloc = 0;
    cudaStream_t pool_stream = nullptr;
    cudaEvent_t pool_join = nullptr;
};

namespace {

vsr_status batch_view_alloc(BatchView& v, int64_t T, int tiles)
{
    vsr_status s;
    if (T > v.T) {
        cudaFree(v.rec);
        v.rec = nullptr;
        v.T = 0;
        if ((s = dalloc(&v.rec, (size_t)REC_F * (size_t)T)) != VSR_OK) return s;
        v.T = T;
    }
    if (tiles > v.tiles) {
        cudaFree(v.counts);
        cudaFree(v.offsets);
        cudaFree(v.partials);
        raster_work_free(&v.work);
        v.counts = v.offsets = v.partials = nullptr;
        v.tiles = 0;
        if ((s = dalloc(&v.counts, (size_t)tiles + 1)) != VSR_OK) return s;  // counts | pair cursor
        if ((s = dalloc(&v.offsets, (size_t)tiles + 1)) != VSR_OK) return s;
        if ((s = dalloc(&v.partials, 2 * (size_t)((tiles + 4095) / 4096) + 2)) != VSR_OK) return s;
        if ((s = raster_work_alloc(&v.work, (uint32_t)tiles)) != VSR_OK) return s;
        v.tiles = tiles;
    }
    return VSR_OK;
}

// set-up, count and scan of view v (before its bins are sized); with
// use_pairs the count records its hits for the fill (not while the bins may
// still be re-sized)
vsr_status batch_view_front(vsr_batch b, int v, vsr_map m, const float* tris, int64_t T, bool use_pairs,
                            cudaStream_t st)
{
    BatchView& bv = b->views[v];
    const int tiles = m->tx * m->ty;
    vsr_status s;
    if ((s = launch_setup_views(tris, (int)T, b->cams_dev + 12 * v, 1, bv.rec, st)) != VSR_OK) return s;
    VSR_CUDA_TRY(cudaMemsetAsync(bv.counts, 0, sizeof(uint32_t) * ((size_t)tiles + 1), st));
    if ((s = launch_bin_count(bv.rec, (int)T, m->idx, bv.counts, bv.counts + tiles, use_pairs ? bv.pairs : nullptr,
                              use_pairs ? bv.cap : 0u, st)) != VSR_OK)
        return s;
    return tiles <= 65536 ? launch_scan(bv.counts, nullptr, tiles, nullptr, bv.offsets, st)
                          : launch_scan_large(bv.counts, nullptr, tiles, bv.partials, bv.offsets, st);
}

// fill and raster of view v (pooled: fill and item assignment only; the
// pooled launch rasterizes the view)
vsr_status batch_view_back(vsr_batch b, int v, vsr_map m, int64_t T, bool use_pairs, uint32_t* id, float* depth,
                           float* cov, cudaStream_t st, int split_max = SPLIT_MAX_DEFAULT, bool pooled = false)
{
    BatchView& bv = b->views[v];
    const int tiles = m->tx * m->ty;
    vsr_status s;
    if ((s = launch_bin_fill(bv.rec, (int)T, m->idx, bv.offsets, bv.counts, bv.counts + tiles,
                             use_pairs ? bv.pairs : nullptr, use_pairs ? bv.cap : 0u, bv.ids, bv.cap, status_word(),
                             st)) != VSR_OK)
        return s;
    if (pooled) return launch_raster_assign(bv.offsets, (uint32_t)tiles, bv.cap, bv.work, split_max, st);
    const RasterView rv{m->map, m->p.W, m->p.H, m->tiles, m->tx, bv.rec, (int)T, bv.offsets,
                        bv.ids, bv.cap, id, depth, cov};
    return launch_raster_items(rv, bv.offsets, (uint32_t)tiles, bv.cap, bv.work, split_max, status_word(),
                               st);
}

constexpr int POOL_GROUPS_MAX = 16;

// Views [first, last) of pool group g of `groups` (contiguous, as even as
// possible).
inline int pool_first(int g, int groups, int nviews) { return (int)((int64_t)g * nviews / groups); }

// The pooled launches' per-view work and item ranges for this configuration,
// split and number of groups, uploaded once (outside any capture).  Group g's
// item starts sit at pool_start + first(g) + g: its views' starts relative to
// the group, then the group's total.
vsr_status batch_pool_upload(vsr_batch b, int nviews, const vsr_map* maps, int64_t T, uint32_t* const* id,
                             float* const* depth, float* const* cov, int split_max, int groups)
{
    if (nviews > b->pool_alloc) {
        cudaFree(b->pool_views);
        cudaFree(b->pool_start);
        cudaFree(b->pool_queue);
        b->pool_views = nullptr;
        b->pool_start = nullptr;
        b->pool_queue = nullptr;
        b->pool_alloc = 0;
        if (cudaMalloc((void**)&b->pool_views, sizeof(PoolView) * (size_t)nviews) != cudaSuccess ||
            cudaMalloc((void**)&b->pool_start, sizeof(uint32_t) * ((size_t)nviews + POOL_GROUPS_MAX)) != cudaSuccess ||
            cudaMalloc((void**)&b->pool_queue, sizeof(uint32_t) * POOL_GROUPS_MAX) != cudaSuccess) {
            cudaGetLastError();
            return VSR_ERR_OOM;
        }
        b->pool_alloc = nviews;
    }
    if (groups < 1 || groups > POOL_GROUPS_MAX || groups > nviews) return VSR_ERR_INVALID_ARG;
    std::vector<PoolView> pv((size_t)nviews);
    std::vector<uint32_t> start((size_t)nviews + POOL_GROUPS_MAX, 0u);
    uint64_t items = 0;
    int g = 0;
    for (int v = 0; v < nviews; ++v) {
        if (v == pool_first(g, groups, nviews)) items = 0;  // a group's items count from 0
        const BatchView& bv = b->views[v];
        const vsr_map m = maps[v];
        const uint32_t tiles = (uint32_t)(m->tx * m->ty);
        pv[v].view = RasterView{m->map, m->p.W, m->p.H, m->tiles, m->tx, bv.rec, (int)T, bv.offsets,
                                bv.ids, bv.cap, id ? id[v] : nullptr, depth ? depth[v] : nullptr,
                                cov ? cov[v] : nullptr};
        pv[v].n_tiles = tiles;
        pv[v].nsplit_of = bv.work.nsplit_of;
        pv[v].split_slot = bv.work.split_slot;
        pv[v].extra = bv.work.extra;
        pv[v].n_extra = bv.work.counters + 1;
        pv[v].acc = bv.work.acc;
        pv[v].key = bv.work.key;
        pv[v].done = bv.work.done;
        start[(size_t)v + g] = (uint32_t)items;
        items += tiles + raster_extra_cap(bv.cap, bv.work, split_max);
        if (items > 0xffffffffull) return VSR_ERR_INVALID_ARG;
        if (v + 1 == pool_first(g + 1, groups, nviews)) {
            start[(size_t)v + 1 + g] = (uint32_t)items;  // the group's total
            ++g;
        }
    }
    VSR_CUDA_TRY(cudaMemcpy(b->pool_views, pv.data(), sizeof(PoolView) * (size_t)nviews, cudaMemcpyHostToDevice));
    VSR_CUDA_TRY(cudaMemcpy(b->pool_start, start.data(), sizeof(uint32_t) * ((size_t)nviews + groups),
                            cudaMemcpyHostToDevice));
    return VSR_OK;
}

}  // namespace

extern "C" {

vsr_status vsr_batch_create(vsr_batch* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    vsr_batch b = new (std::nothrow) vsr_batch_s;
    if (!b) return VSR_ERR_OOM;
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->cams_done, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->pool_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->pool_join, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < BATCH_STREAMS_MAX; ++i)
        ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        vsr_batch_free(b);
        return VSR_ERR_CUDA;
    }
    *out = b;
    return VSR_OK;
}

void vsr_batch_free(vsr_batch b)
{
    if (!b) return;
    if (b->cams_done) cudaEventSynchronize(b->cams_done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& v : b->views) batch_view_free(v);
    cudaFree(b->cams_dev);
    if (b->cams_host) cudaFreeHost(b->cams_host);
    if (b->h_total) cudaFreeHost(b->h_total);
    for (int i = 0; i < BATCH_STREAMS_MAX; ++i) {
        if (b->streams[i]) cudaStreamDestroy(b->streams[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cams_done) cudaEventDestroy(b->cams_done);
    cudaFree(b->pool_views);
    cudaFree(b->pool_start);
    cudaFree(b->pool_queue);
    if (b->pool_stream) cudaStreamDestroy(b->pool_stream);
    if (b->pool_join) cudaEventDestroy(b->pool_join);
    delete b;
}

vsr_status vsr_batch_render(vsr_batch b, int nviews, const vsr_map* maps, const float* tris_dev, int64_t T,
                            const float* cams, uint32_t* const* id_dev, float* const* depth_dev,
                            float* const* cov_dev, void* stream)
{
    if (!b || nviews <= 0 || !maps || !cams || !setup_args_ok(tris_dev, T, cams)) return VSR_ERR_INVALID_ARG;
    for (int v = 0; v < nviews; ++v) {
        if (!maps[v]) return VSR_ERR_INVALID_ARG;
        for (int q = 0; q < 12; ++q)
            if (!isfinite(cams[12 * v + q])) return VSR_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    auto out_ptr = [](auto* const* arr, int v) { return arr ? arr[v] : nullptr; };

    std::vector<uint64_t> key = {(uint64_t)nviews, (uint64_t)T, (uint64_t)(uintptr_t)tris_dev};
    for (int v = 0; v < nviews; ++v) {
        key.push_back((uint64_t)(uintptr_t)maps[v]);
        key.push_back(maps[v]->gen);
        key.push_back((uint64_t)(uintptr_t)out_ptr(id_dev, v));
        key.push_back((uint64_t)(uintptr_t)out_ptr(depth_dev, v));
        key.push_back((uint64_t)(uintptr_t)out_ptr(cov_dev, v));
    }
    const size_t cam_bytes = sizeof(float) * 12 * (size_t)nviews;

    if (b->exec && key == b->key) {
        // replay: new cameras only.  The previous replay (complete once its
        // event has) left each view's pair total in pinned memory: a view
        // within 1/8 of its bin capacity rebuilds the configuration with
        // larger bins before this frame instead of overflowing in a later one.
        VSR_CUDA_TRY(cudaEventSynchronize(b->cams_done));
        bool grow = false;
        for (int v = 0; v < nviews && !grow; ++v) {
            const uint64_t last = b->h_total[v];
            grow = last + last / 8 > b->views[v].cap;
        }
        if (!grow) {
            memcpy(b->cams_host, cams, cam_bytes);
            VSR_CUDA_TRY(cudaGraphLaunch(b->exec, st));
            VSR_CUDA_TRY(cudaEventRecord(b->cams_done, st));
            return VSR_OK;
        }
    }

    // new configuration
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->key.clear();
    VSR_CUDA_TRY(cudaEventSynchronize(b->cams_done));
    vsr_status s;
    if (nviews > b->cams_alloc) {
        cudaFree(b->cams_dev);
        if (b->cams_host) cudaFreeHost(b->cams_host);
        if (b->h_total) cudaFreeHost(b->h_total);
        b->cams_dev = nullptr;
        b->cams_host = nullptr;
        b->h_total = nullptr;
        b->cams_alloc = 0;
        if ((s = dalloc(&b->cams_dev, 12 * (size_t)nviews)) != VSR_OK) return s;
        if (cudaMallocHost((void**)&b->cams_host, cam_bytes) != cudaSuccess ||
            cudaMallocHost((void**)&b->h_total, sizeof(uint32_t) * (size_t)nviews) != cudaSuccess) {
            cudaGetLastError();
            return VSR_ERR_OOM;
        }
        b->cams_alloc = nviews;
    }
    if ((int)b->views.size() < nviews) b->views.resize(nviews);
    for (int v = 0; v < nviews; ++v)
        if ((s = batch_view_alloc(b->views[v], T, maps[v]->tx * maps[v]->ty)) != VSR_OK) return s;
    memcpy(b->cams_host, cams, cam_bytes);
    VSR_CUDA_TRY(cudaMemcpyAsync(b->cams_dev, b->cams_host, cam_bytes, cudaMemcpyHostToDevice, st));

    // the views' binning searches their maps' tile indexes (built once per
    // generation of a map; the key holds the generations)
    for (int v = 0; v < nviews; ++v)
        if ((s = ensure_tile_index(maps[v], st)) != VSR_OK) return s;
    // eager frame: fronts, one synchronisation to size every view's bins, backs
    for (int v = 0; v < nviews; ++v) {
        if ((s = batch_view_front(b, v, maps[v], tris_dev, T, false, st)) != VSR_OK) return s;
        const int tiles = maps[v]->tx * maps[v]->ty;
        VSR_CUDA_TRY(cudaMemcpyAsync(b->h_total + v, b->views[v].offsets + tiles, sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost, st));
    }
    VSR_CUDA_TRY(cudaStreamSynchronize(st));
    for (int v = 0; v < nviews; ++v) {
        BatchView& bv = b->views[v];
        const uint32_t total = b->h_total[v];
        if (total + total / 8 > bv.cap || !bv.ids) {
            cudaFree(bv.ids);
            cudaFree(bv.pairs);
            bv.ids = nullptr;
            bv.pairs = nullptr;
            bv.cap = 0;
            uint64_t want = (uint64_t)total + total / 4 + 4096;
            if (want > 0xffffffffull) want = 0xffffffffull;
            if ((s = dalloc(&bv.ids, (size_t)want)) != VSR_OK) return s;
            if ((s = dalloc(&bv.pairs, (size_t)want)) != VSR_OK) return s;
            bv.cap = (uint32_t)want;
        }
    }
    for (int v = 0; v < nviews; ++v)
        if ((s = batch_view_back(b, v, maps[v], T, false, out_ptr(id_dev, v), out_ptr(depth_dev, v),
                                 out_ptr(cov_dev, v), st)) != VSR_OK)
            return s;
    VSR_CUDA_TRY(cudaEventRecord(b->cams_done, st));

    // autotune: capture one graph per candidate (parallel streams S, raster
    // kind, triangles per work item of a long bin), time three replays, keep
    // the fastest; first the stream counts and kinds at the default split,
    // then the splits at the best of them
    float best = 1e30f;
    cudaEvent_t e0, e1;
    VSR_CUDA_TRY(cudaEventCreate(&e0));
    VSR_CUDA_TRY(cudaEventCreate(&e1));
    // groups > 0: the views' chains end after binning and item assignment,
    // and each group of views is rasterized by one pooled launch on the pool
    // stream as soon as its views are binned, beside the next groups' chains
    auto candidate = [&](int S, int split, int groups) -> vsr_status {
        S = S < nviews ? S : nviews;
        if (groups > nviews) return VSR_OK;
        const bool pooled = groups > 0;
        if (pooled) {
            const vsr_status us = batch_pool_upload(b, nviews, maps, T, id_dev, depth_dev, cov_dev, split, groups);
            if (us != VSR_OK) return us;
        }
        cudaStream_t cs = b->streams[0];
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VSR_ERR_CUDA;
        vsr_status cst = VSR_OK;
        if (cudaMemcpyAsync(b->cams_dev, b->cams_host, cam_bytes, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
            cudaEventRecord(b->fork, cs) != cudaSuccess)
            cst = VSR_ERR_CUDA;
        for (int i = 1; cst == VSR_OK && i < S; ++i)
            if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) cst = VSR_ERR_CUDA;
        if (cst == VSR_OK && pooled && cudaStreamWaitEvent(b->pool_stream, b->fork, 0) != cudaSuccess)
            cst = VSR_ERR_CUDA;
        int group = 0;
        for (int v = 0; cst == VSR_OK && v < nviews; ++v) {
            cudaStream_t vs = b->streams[v % S];
            cst = batch_view_front(b, v, maps[v], tris_dev, T, true, vs);
            const int tiles = maps[v]->tx * maps[v]->ty;
            if (cst == VSR_OK && cudaMemcpyAsync(b->h_total + v, b->views[v].offsets + tiles, sizeof(uint32_t),
                                                 cudaMemcpyDeviceToHost, vs) != cudaSuccess)
                cst = VSR_ERR_CUDA;
            if (cst == VSR_OK)
                cst = batch_view_back(b, v, maps[v], T, true, out_ptr(id_dev, v), out_ptr(depth_dev, v),
                                      out_ptr(cov_dev, v), vs, split, pooled);
            if (cst == VSR_OK && pooled && v + 1 == pool_first(group + 1, groups, nviews)) {
                // the group's views are binned once every stream reaches this point
                for (int i = 0; cst == VSR_OK && i < S; ++i)
                    if (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess ||
                        cudaStreamWaitEvent(b->pool_stream, b->join[i], 0) != cudaSuccess)
                        cst = VSR_ERR_CUDA;
                const int first = pool_first(group, groups, nviews);
                if (cst == VSR_OK)
                    cst = launch_raster_pool(b->pool_views + first, b->pool_start + first + group, v + 1 - first,
                                             b->pool_queue + group, split, status_word(), b->pool_stream);
                ++group;
            }
        }
        for (int i = 1; cst == VSR_OK && i < S; ++i)
            if (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess ||
                cudaStreamWaitEvent(cs, b->join[i], 0) != cudaSuccess)
                cst = VSR_ERR_CUDA;
        if (cst == VSR_OK && pooled &&
            (cudaEventRecord(b->pool_join, b->pool_stream) != cudaSuccess ||
             cudaStreamWaitEvent(cs, b->pool_join, 0) != cudaSuccess))
            cst = VSR_ERR_CUDA;
        const cudaError_t ee = cudaStreamEndCapture(cs, &g);
        if (cst != VSR_OK || ee != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return cst != VSR_OK ? cst : VSR_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            return VSR_OK;  // not this candidate
        }
        // one warm replay, then three timed one at a time: frames of a batch
        // run alone (each render waits for the previous frame), so a graph
        // is measured by its own span, not by overlap with the next replay
        float ms = 0.0f;
        bool timed = cudaGraphLaunch(ex, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
        for (int r = 0; timed && r < 3; ++r) {
            float one = 0.0f;
            timed = cudaEventRecord(e0, st) == cudaSuccess && cudaGraphLaunch(ex, st) == cudaSuccess &&
                    cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&one, e0, e1) == cudaSuccess;
            ms += one;
        }
        if (timed && ms < best) {
            best = ms;
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = ex;
            b->nstreams = S;
            b->split_max = split;
            b->pool_groups = groups;
        } else {
            cudaGraphExecDestroy(ex);
        }
        return VSR_OK;
    };
    // the per-view raster launches and the pooled one: each at every stream
    // count and the default split, then the splits at the best of them
    vsr_status ts = VSR_OK;
    const bool try_chains = b->mode != VSR_BATCH_POOLED, try_pool = b->mode != VSR_BATCH_CHAINS;
    for (int S : {1, 2, 4, 8}) {
        if (ts == VSR_OK && try_chains) ts = candidate(S, SPLIT_MAX_DEFAULT, 0);
        for (int groups : {1, 4, 16})
            if (ts == VSR_OK && try_pool) ts = candidate(S, SPLIT_MAX_DEFAULT, groups);
    }
    const int bestS = b->nstreams;
    const int best_groups = b->pool_groups;
    for (int split : {256, 1024})
        if (ts == VSR_OK && b->exec) ts = candidate(bestS, split, best_groups);
    // the kept graph's pooled views must carry its split and grouping
    if (ts == VSR_OK && b->exec && b->pool_groups > 0)
        ts = batch_pool_upload(b, nviews, maps, T, id_dev, depth_dev, cov_dev, b->split_max, b->pool_groups);
    if (ts != VSR_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return ts;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!b->exec) return VSR_ERR_CUDA;
    b->key = key;
    VSR_CUDA_TRY(cudaEventRecord(b->cams_done, st));
    return VSR_OK;
}

vsr_status vsr_batch_config(vsr_batch b, int* streams, int* graphed, int* split_max)
{
    return vsr_batch_config_ex(b, streams, graphed, split_max, nullptr);
}

vsr_status vsr_batch_config_ex(vsr_batch b, int* streams, int* graphed, int* split_max, int* pooled)
{
    if (!b) return VSR_ERR_INVALID_ARG;
    if (streams) *streams = b->nstreams;
    if (graphed) *graphed = b->exec != nullptr;
    if (split_max) *split_max = b->split_max;
    if (pooled) *pooled = b->exec != nullptr ? b->pool_groups : 0;
    return VSR_OK;
}

vsr_status vsr_batch_set_mode(vsr_batch b, int mode)
{
    if (!b || mode < VSR_BATCH_AUTO || mode > VSR_BATCH_POOLED) return VSR_ERR_INVALID_ARG;
    if (mode != b->mode) {
        b->mode = mode;
        b->key.clear();  // the next render tunes again
    }
    return VSR_OK;
}

}  // extern "C"
