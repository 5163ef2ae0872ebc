// grad_api.cu -- C ABI of the differentiable path: vsr_frags,
// vsr_raster_shaded and vsr_raster_backward (kernels in grad.cu, map.cu).
#include <math.h>
#include <new>

#include "handles.cuh"

struct vsr_frags_s {
    size_t npix = 0;            // per-pixel buffers sized for this many pixels
    uint32_t* counts = nullptr;  // npix
    uint32_t* foff = nullptr;    // npix + 1
    uint32_t* scan_part = nullptr;
    float4* frags = nullptr;
    uint32_t fcap = 0;
    uint32_t* h_total = nullptr;  // pinned
    float4* dmap = nullptr;       // npix
    float* lens_part = nullptr;
    float4* grad = nullptr;       // GF_COUNT x grad_T
    int64_t grad_T = 0;
    // the forward the lists belong to
    uint64_t map_gen = 0, scene_gen = 0;
    int W = 0, H = 0;
    bool valid = false;
};

namespace {

void frags_release_pixels(vsr_frags f)
{
    cudaFree(f->counts);
    cudaFree(f->foff);
    cudaFree(f->scan_part);
    cudaFree(f->dmap);
    cudaFree(f->lens_part);
    f->counts = f->foff = f->scan_part = nullptr;
    f->dmap = nullptr;
    f->lens_part = nullptr;
    f->npix = 0;
}

vsr_status frags_ensure_pixels(vsr_frags f, int W, int H)
{
    const size_t n = (size_t)W * H;
    if (n <= f->npix) return VSR_OK;
    frags_release_pixels(f);
    vsr_status s;
    const size_t nb = (n + 4095) / 4096;
    if ((s = dalloc(&f->counts, n)) != VSR_OK || (s = dalloc(&f->foff, n + 1)) != VSR_OK ||
        (s = dalloc(&f->scan_part, 2 * nb + 2)) != VSR_OK || (s = dalloc(&f->dmap, n)) != VSR_OK ||
        (s = dalloc(&f->lens_part, map_backward_partials(W, H) + (size_t)W * 4)) != VSR_OK) {
        frags_release_pixels(f);
        return s;
    }
    f->npix = n;
    return VSR_OK;
}

FragArgs frag_args(vsr_map m, vsr_scene sc, const float* colors, vsr_frags f)
{
    FragArgs a{};
    a.map = m->map;
    a.W = m->p.W;
    a.H = m->p.H;
    a.tiles = m->tiles;
    a.rec = sc->rec;
    a.T = (int)sc->T;
    a.offsets = sc->offsets;
    a.ends = scene_ends(sc);
    a.ids = sc->ids;
    a.cap = sc->cap;
    a.colors = colors;
    a.counts = f->counts;
    a.foff = f->foff;
    a.frags = f->frags;
    a.fcap = f->fcap;
    a.status = scene_status(sc);
    return a;
}

}  // namespace

extern "C" {

vsr_status vsr_frags_create(vsr_frags* out)
{
    if (!out) return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    vsr_frags f = new (std::nothrow) vsr_frags_s;
    if (!f) return VSR_ERR_OOM;
    if (cudaMallocHost((void**)&f->h_total, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete f;
        return VSR_ERR_OOM;
    }
    *out = f;
    return VSR_OK;
}

void vsr_frags_free(vsr_frags f)
{
    if (!f) return;
    frags_release_pixels(f);
    cudaFree(f->frags);
    cudaFree(f->grad);
    if (f->h_total) cudaFreeHost(f->h_total);
    delete f;
}

vsr_status vsr_raster_shaded(vsr_map m, vsr_scene sc, const float* colors_dev, vsr_frags f, float* image_dev,
                             float* cov_dev, uint32_t* id_dev, float* depth_dev, void* stream)
{
    if (!m || !sc || !f) return VSR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    f->valid = false;
    vsr_status s = vsr_bin(m, sc, stream);
    if (s != VSR_OK) return s;
    const int W = m->p.W, H = m->p.H;
    if ((s = frags_ensure_pixels(f, W, H)) != VSR_OK) return s;
    FragArgs a = frag_args(m, sc, colors_dev, f);
    if ((s = launch_frag_count(a, st)) != VSR_OK) return s;
    const int npix = W * H;
    if ((s = launch_scan_large(f->counts, nullptr, npix, f->scan_part, f->foff, st)) != VSR_OK) return s;
    VSR_CUDA_TRY(cudaMemcpyAsync(f->h_total, f->foff + npix, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    VSR_CUDA_TRY(cudaStreamSynchronize(st));
    const uint32_t total = *f->h_total;
    if (total > f->fcap) {
        cudaFree(f->frags);
        f->frags = nullptr;
        f->fcap = 0;
        uint64_t want = (uint64_t)total + total / 4 + 1024;
        if (want > 0xffffffffull) want = 0xffffffffull;
        if ((s = dalloc(&f->frags, (size_t)want)) != VSR_OK) return s;
        f->fcap = (uint32_t)want;
    }
    a.frags = f->frags;
    a.fcap = f->fcap;
    a.image = image_dev;
    a.cov = cov_dev;
    a.out_id = id_dev;
    a.out_depth = depth_dev;
    if ((s = launch_frag_fill(a, st)) != VSR_OK) return s;
    f->map_gen = m->gen;
    f->scene_gen = sc->gen;
    f->W = W;
    f->H = H;
    f->valid = true;
    return scene_used(sc, st);
}

vsr_status vsr_raster_backward(vsr_map m, vsr_scene sc, const float* tris_dev, const float* colors_dev, vsr_frags f,
                               const uint32_t* id_dev, const float* dimage_dev, const float* dcov_dev,
                               const float* ddepth_dev, float* dtris_dev, float* dcolors_dev, double* dlens_dev,
                               void* stream)
{
    if (!m || !sc || !f || !f->valid) return VSR_ERR_INVALID_ARG;
    if (f->map_gen != m->gen || f->scene_gen != sc->gen || f->W != m->p.W || f->H != m->p.H)
        return VSR_ERR_INVALID_ARG;
    if (ddepth_dev && !id_dev) return VSR_ERR_INVALID_ARG;
    if (dtris_dev && sc->T > 0 && !tris_dev) return VSR_ERR_INVALID_ARG;
    if (dlens_dev && !m->lens_grad) return VSR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t T = sc->T;
    vsr_status s;
    if (T > f->grad_T) {
        cudaFree(f->grad);
        f->grad = nullptr;
        f->grad_T = 0;
        if ((s = dalloc(&f->grad, (size_t)GF_COUNT * (size_t)T)) != VSR_OK) return s;
        f->grad_T = T;
    }
    if (T > 0) VSR_CUDA_TRY(cudaMemsetAsync(f->grad, 0, sizeof(float4) * GF_COUNT * (size_t)T, st));
    FragArgs a = frag_args(m, sc, colors_dev, f);
    if ((s = launch_frag_backward(a, id_dev, dimage_dev, dcov_dev, ddepth_dev, f->grad, f->dmap, st)) != VSR_OK)
        return s;
    if (dtris_dev || dcolors_dev) {
        if ((s = launch_setup_backward(tris_dev, (int)T, sc->cam, sc->rec, f->grad, dtris_dev, dcolors_dev, st)) !=
            VSR_OK)
            return s;
    }
    if (dlens_dev) {
        if ((s = launch_map_backward(m->p.W, m->p.H, m->p.aov, m->p.k, m->p.l, m->p.s, m->p.omega_deg, f->dmap,
                                     f->lens_part, dlens_dev, st)) != VSR_OK)
            return s;
    }
    return scene_used(sc, st);
}

}  // extern "C"
