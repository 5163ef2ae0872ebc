// serve.cu -- a rendering server with continuous batching (vsr_serve_*).
//
// A worker thread owns `slots` CUDA streams.  Requests (a resident scene,
// lens parameters, a camera, caller-owned outputs) wait in a FIFO queue and
// are admitted into free slots as soon as a slot and device memory allow,
// while earlier requests are still running on the GPU: their launches
// overlap on the device, each on its own stream and workspace.  The
// perspective maps of the requests come from an LRU cache keyed by the
// exact lens parameters and picture size; entries used by requests in
// flight are never evicted.  Memory held by maps and per-(slot, scene)
// workspaces is accounted against a budget: a request that needs a new map
// evicts idle cache entries until it fits, waits while other requests hold
// memory, and fails with VSR_ERR_BUDGET when it cannot fit even alone.
// Completion is detected by polling CUDA events from the worker thread (no
// device-side waits).  The workspaces size their bins without waiting for
// the device when a request's map shape differs from the previous one's
// (the capacity only grows), so admitting a request never blocks the worker;
// a request whose bins outgrew their capacity (known from the pair count
// once it has finished) is rendered again with grown bins; the slots' workspaces report to status words of their own, so such
// handled overflows do not reach vsr_last_device_status.  Every request's
// output equals that of rendering it alone: the arithmetic is per request and
// order-free.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handles.cuh"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

struct MapKey {
    float k, l, s, omega;
    int W, H, aov, strict;
    bool operator==(const MapKey& o) const { return memcmp(this, &o, sizeof(MapKey)) == 0; }
};

struct MapKeyHash {
    size_t operator()(const MapKey& k) const
    {
        const unsigned char* p = (const unsigned char*)&k;
        size_t h = 1469598103934665603ull;  // FNV-1a over the key's bytes
        for (size_t i = 0; i < sizeof(MapKey); ++i) h = (h ^ p[i]) * 1099511628211ull;
        return h;
    }
};

struct MapEntry {
    MapKey key;
    vsr_map map = nullptr;
    size_t bytes = 0;
    int refs = 0;
    // recorded after the map's generation on the stream of the slot that
    // made it; a slot on another stream that takes the cached map waits for
    // it on its own stream before reading the map, cones or tile index
    cudaEvent_t ready = nullptr;
};

struct Request {
    uint64_t ticket;
    vsr_request r;
    double t_submit;
    int reruns = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int* status = nullptr;  // device status word of this slot's workspaces
    bool busy = false;
    Request req;
    std::list<MapEntry>::iterator map;
    vsr_scene work = nullptr;  // workspace of the request's scene on this slot
    double t_start = 0;
    bool hit = false;
};

struct Scene {
    const float* tris = nullptr;
    int64_t T = 0;
};

size_t map_bytes(int W, int H)
{
    const size_t tiles = (size_t)((W + TILE - 1) / TILE) * ((H + TILE - 1) / TILE);
    // map, cones (tiles, sorted, big), per-tile geometry, cell starts, header
    return (size_t)W * H * sizeof(float4) + tiles * (3 * sizeof(Cone) + sizeof(float4)) +
           sizeof(uint32_t) * (IDX_CELLS_MAX + 1) + sizeof(TileIndexHdr);
}

// device memory a (slot, scene) workspace will take once used: records,
// triangle index (tile-major binning), bins and their pair list (estimated
// at 4 pairs per triangle) and split accumulators
size_t work_estimate(int64_t T, int W, int H)
{
    const size_t tiles = (size_t)((W + TILE - 1) / TILE) * ((H + TILE - 1) / TILE);
    const size_t split = tiles < SPLIT_SLOTS ? tiles : SPLIT_SLOTS;
    const size_t tri = T <= TILE_MAJOR_TRIS_PER_TILE * (int64_t)tiles ? tri_index_bytes(T, (int)tiles) : 0;
    return (size_t)T * (REC_F * sizeof(float4) + 4 * (sizeof(uint32_t) + sizeof(uint2))) + tri +
           tiles * 4 * sizeof(uint32_t) + split * TILE_PIX * 2 * sizeof(uint64_t) + EXTRA_ITEMS * sizeof(uint2);
}

size_t scene_bytes(const vsr_scene_s* s)
{
    size_t b = (size_t)s->T_alloc * REC_F * sizeof(float4) + (size_t)s->ws_tiles * 2 * sizeof(uint32_t) +
               (size_t)s->cap * (sizeof(uint32_t) + sizeof(uint2));
    if (s->tri.counts) b += tri_index_bytes(s->tri.T, s->tri.ntiles);
    if (s->work_tiles)
        b += (size_t)s->work.split_cap * TILE_PIX * (sizeof(uint64_t) * 2) + (size_t)s->work.extra_cap * sizeof(uint2) +
             (size_t)s->work_tiles * 2 * sizeof(uint32_t);
    return b;
}

}  // namespace

struct vsr_server_s {
    vsr_serve_cfg cfg;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, vsr_result> results;
    std::vector<Scene> scenes;
    std::vector<Slot> slots;
    std::vector<std::vector<vsr_scene>> work;  // [slot][scene]
    std::list<MapEntry> cache;                 // most recently used first
    std::unordered_map<MapKey, std::list<MapEntry>::iterator, MapKeyHash> index;
    size_t map_bytes_used = 0;
    vsr_serve_stats stats = {};
    uint64_t next_ticket = 1;
    bool stop = false;
    int device = 0;
    std::thread worker;

    size_t used() const
    {
        size_t b = map_bytes_used;
        for (const auto& per_slot : work)
            for (vsr_scene w : per_slot)
                if (w) b += scene_bytes(w);
        return b;
    }

    void finish(const Request& q, vsr_status st, double t_start, bool hit)
    {
        vsr_result res;
        res.status = st;
        res.done = 1;
        res.map_cache_hit = hit ? 1 : 0;
        res.t_submit = q.t_submit;
        res.t_start = t_start;
        res.t_done = now_s();
        results[q.ticket] = res;
        if (st == VSR_OK)
            ++stats.completed;
        else if (st == VSR_ERR_CANCELLED)
            ++stats.cancelled;
        else
            ++stats.failed;
        cv.notify_all();
    }

    // find or make the map of a request; false when the budget does not
    // allow it now
    bool get_map(const vsr_map_params& p, size_t extra_need, cudaStream_t st, std::list<MapEntry>::iterator* out,
                 bool* hit, vsr_status* err)
    {
        MapKey key{p.k, p.l, p.s, p.omega_deg, p.W, p.H, p.aov, p.strict_limits};
        auto it = index.find(key);
        if (it != index.end() && used() + extra_need <= (size_t)cfg.budget_bytes) {
            if (cudaStreamWaitEvent(st, it->second->ready, 0) != cudaSuccess) {
                cudaGetLastError();
                *err = VSR_ERR_CUDA;
                return false;
            }
            cache.splice(cache.begin(), cache, it->second);
            *out = cache.begin();
            *hit = true;
            ++stats.map_hits;
            return true;
        }
        const size_t need = (it != index.end() ? 0 : map_bytes(p.W, p.H)) + extra_need;
        // a new map over the budget first takes the place of the least
        // recently used idle map of its own size: that handle is regenerated
        // in place (vsr_map_update), which needs no cudaFree -- a
        // device-wide synchronisation -- and no cudaMalloc
        vsr_map reuse = nullptr;
        if (it == index.end() && used() + need > (size_t)cfg.budget_bytes) {
            for (auto e = cache.end(); e != cache.begin();) {
                --e;
                if (e->refs == 0 && e->key.W == p.W && e->key.H == p.H) {
                    map_bytes_used -= e->bytes;
                    index.erase(e->key);
                    reuse = e->map;
                    if (e->ready) cudaEventDestroy(e->ready);
                    cache.erase(e);
                    ++stats.map_evictions;
                    break;
                }
            }
        }
        // evict idle entries, least recently used first
        for (auto e = cache.end(); e != cache.begin();) {
            --e;
            const bool over_count = cfg.max_maps > 0 && (int)cache.size() >= cfg.max_maps;
            if (used() + need <= (size_t)cfg.budget_bytes && !over_count) break;
            if (e->refs == 0 && !(it != index.end() && e == it->second)) {
                map_bytes_used -= e->bytes;
                index.erase(e->key);
                vsr_map_free(e->map);
                if (e->ready) cudaEventDestroy(e->ready);
                e = cache.erase(e);
                ++stats.map_evictions;
            }
        }
        if (used() + need > (size_t)cfg.budget_bytes) {
            if (reuse) vsr_map_free(reuse);
            *err = VSR_ERR_BUDGET;
            return false;
        }
        if (it != index.end()) {  // a hit that needed room for its workspace
            if (cudaStreamWaitEvent(st, it->second->ready, 0) != cudaSuccess) {
                cudaGetLastError();
                *err = VSR_ERR_CUDA;
                return false;
            }
            cache.splice(cache.begin(), cache, it->second);
            *out = cache.begin();
            *hit = true;
            ++stats.map_hits;
            return true;
        }
        vsr_map m = reuse;
        vsr_status s = reuse ? vsr_map_update(reuse, &p, st) : vsr_make_map_ex(&p, st, &m);
        if (s != VSR_OK) {
            if (reuse) vsr_map_free(reuse);
            *err = s;
            return false;
        }
        cudaEvent_t ready = nullptr;
        if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ready, st) != cudaSuccess) {
            cudaGetLastError();
            if (ready) cudaEventDestroy(ready);
            vsr_map_free(m);
            *err = VSR_ERR_CUDA;
            return false;
        }
        const size_t mb = map_bytes(p.W, p.H);
        cache.push_front(MapEntry{key, m, mb, 0, ready});
        index[key] = cache.begin();
        map_bytes_used += mb;
        *out = cache.begin();
        *hit = false;
        ++stats.map_misses;
        return true;
    }

    vsr_status launch(Slot& sl)
    {
        const vsr_request& r = sl.req.r;
        const Scene& sc = scenes[r.scene];
        vsr_status s = vsr_scene_update(sl.work, sc.tris, sc.T, r.cam, sl.stream);
        if (s == VSR_OK) s = vsr_raster(sl.map->map, sl.work, r.id_dev, r.depth_dev, r.cov_dev, sl.stream);
        if (s == VSR_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) s = VSR_ERR_CUDA;
        return s;
    }

    void loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progressed = false;
            // completions
            for (Slot& sl : slots) {
                if (!sl.busy) continue;
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) {
                    // the slot's work failed on the device: report it instead
                    // of waiting for an event that will not complete
                    cudaGetLastError();
                    sl.map->refs--;
                    finish(sl.req, VSR_ERR_CUDA, sl.t_start, sl.hit);
                    sl.busy = false;
                    progressed = true;
                    continue;
                }
                vsr_scene_s* w = sl.work;
                const bool overflow = *w->h_total > w->cap;
                if (overflow && sl.req.reruns < 3) {
                    // the bins overflowed: vsr_bin grows them from this count; render again
                    ++sl.req.reruns;
                    ++stats.reruns;
                    if (launch(sl) == VSR_OK) continue;
                }
                sl.map->refs--;
                // outputs of bins that still overflow are incomplete: say so
                finish(sl.req, overflow ? VSR_ERR_BIN_OVERFLOW : VSR_OK, sl.t_start, sl.hit);
                sl.busy = false;
                progressed = true;
            }
            // admissions: continuous batching into free slots
            for (Slot& sl : slots) {
                if (sl.busy || queue.empty()) continue;
                Request q = queue.front();
                std::list<MapEntry>::iterator me;
                bool hit = false;
                vsr_status err = VSR_OK;
                const int si = (int)(&sl - slots.data());
                const size_t wneed =
                    work[si][q.r.scene] ? 0 : work_estimate(scenes[q.r.scene].T, q.r.lens.W, q.r.lens.H);
                if (!get_map(q.r.lens, wneed, sl.stream, &me, &hit, &err)) {
                    bool any_busy = false;
                    for (const Slot& o : slots) any_busy |= o.busy;
                    if (err == VSR_ERR_BUDGET && any_busy) break;  // wait for memory to free up
                    queue.pop_front();
                    finish(q, err, now_s(), false);
                    progressed = true;
                    continue;
                }
                queue.pop_front();
                vsr_scene& w = work[si][q.r.scene];
                if (!w) {
                    if (vsr_scene_create(&w) != VSR_OK) {
                        finish(q, VSR_ERR_OOM, now_s(), hit);
                        continue;
                    }
                    w->status = sl.status;  // overflows are handled here, not reported globally
                    w->async_sizing = true;  // a bin overflow renders the request again (below)
                }
                sl.req = q;
                sl.map = me;
                sl.work = w;
                sl.hit = hit;
                sl.t_start = now_s();
                me->refs++;
                lk.unlock();
                const vsr_status s = launch(sl);
                lk.lock();
                if (s != VSR_OK) {
                    me->refs--;
                    finish(q, s, sl.t_start, hit);
                } else {
                    sl.busy = true;
                }
                progressed = true;
            }
            bool any_busy = false;
            for (const Slot& sl : slots) any_busy |= sl.busy;
            if (stop && queue.empty() && !any_busy) break;
            if (!progressed) {
                if (any_busy)
                    cv.wait_for(lk, std::chrono::microseconds(20));
                else
                    cv.wait_for(lk, std::chrono::milliseconds(5), [&] { return stop || !queue.empty(); });
            }
        }
    }
};

extern "C" {

vsr_status vsr_serve_create(const vsr_serve_cfg* cfg, vsr_server* out)
{
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 32 || cfg->budget_bytes <= 0 || cfg->max_maps < 0)
        return VSR_ERR_INVALID_ARG;
    *out = nullptr;
    vsr_server s = new (std::nothrow) vsr_server_s;
    if (!s) return VSR_ERR_OOM;
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return VSR_ERR_CUDA;
    }
    s->slots.resize(cfg->slots);
    s->work.resize(cfg->slots);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc((void**)&sl.status, sizeof(int)) != cudaSuccess || cudaMemset(sl.status, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            vsr_serve_destroy(s);
            return VSR_ERR_CUDA;
        }
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return VSR_OK;
}

vsr_status vsr_serve_add_scene(vsr_server s, const float* tris_dev, int64_t T, int* scene)
{
    if (!s || !scene || T < 0 || T >= 0x7fffffffLL || (T > 0 && !tris_dev)) return VSR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->scenes.push_back(Scene{tris_dev, T});
    for (auto& per_slot : s->work) per_slot.resize(s->scenes.size(), nullptr);
    *scene = (int)s->scenes.size() - 1;
    return VSR_OK;
}

vsr_status vsr_serve_submit(vsr_server s, const vsr_request* r, uint64_t* ticket)
{
    if (!s || !r || !ticket) return VSR_ERR_INVALID_ARG;
    const vsr_map_params& p = r->lens;
    if (!isfinite(p.k) || !isfinite(p.l) || !isfinite(p.s) || !isfinite(p.omega_deg) || p.W < 1 || p.H < 1 ||
        p.W > 32768 || p.H > 32768 || p.aov < 0 || p.aov > 3)
        return VSR_ERR_INVALID_ARG;
    for (int q = 0; q < 12; ++q)
        if (!isfinite(r->cam[q])) return VSR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->scene < 0 || r->scene >= (int)s->scenes.size() || s->stop) return VSR_ERR_INVALID_ARG;
    if (map_bytes(p.W, p.H) > (size_t)s->cfg.budget_bytes) return VSR_ERR_BUDGET;
    Request q;
    q.ticket = s->next_ticket++;
    q.r = *r;
    q.t_submit = now_s();
    vsr_result pending = {};
    pending.status = VSR_OK;
    pending.t_submit = q.t_submit;
    s->results[q.ticket] = pending;
    s->queue.push_back(q);
    ++s->stats.submitted;
    *ticket = q.ticket;
    s->cv.notify_all();
    return VSR_OK;
}

vsr_status vsr_serve_poll(vsr_server s, uint64_t ticket, vsr_result* out)
{
    if (!s || !out) return VSR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return VSR_ERR_INVALID_ARG;
    *out = it->second;
    if (out->done) s->results.erase(it);
    return VSR_OK;
}

vsr_status vsr_serve_wait(vsr_server s, uint64_t ticket, vsr_result* out)
{
    if (!s || !out) return VSR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        auto it = s->results.find(ticket);
        if (it == s->results.end()) return VSR_ERR_INVALID_ARG;
        if (it->second.done) {
            *out = it->second;
            s->results.erase(it);
            return VSR_OK;
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
}

vsr_status vsr_serve_cancel(vsr_server s, uint64_t ticket)
{
    if (!s) return VSR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (it->ticket == ticket) {
            const Request q = *it;
            s->queue.erase(it);
            s->finish(q, VSR_ERR_CANCELLED, now_s(), false);
            return VSR_OK;
        }
    return VSR_ERR_INVALID_ARG;  // unknown, running or finished
}

vsr_status vsr_serve_stats_get(vsr_server s, vsr_serve_stats* out)
{
    if (!s || !out) return VSR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->bytes_in_use = (int64_t)s->used();
    out->maps_cached = (int64_t)s->cache.size();
    out->queued = (int64_t)s->queue.size();
    return VSR_OK;
}

double vsr_serve_now(void) { return now_s(); }

vsr_status vsr_serve_destroy(vsr_server s)
{
    if (!s) return VSR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto& per_slot : s->work)
        for (vsr_scene w : per_slot) vsr_scene_free(w);
    for (Slot& sl : s->slots) cudaFree(sl.status);
    for (MapEntry& e : s->cache) {
        vsr_map_free(e.map);
        if (e.ready) cudaEventDestroy(e.ready);
    }
    delete s;
    return VSR_OK;
}

}  // extern "C"
