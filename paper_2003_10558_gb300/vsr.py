"""Python binding of libvsr.so (the C ABI in include/vsr.h).

Argument marshalling only: every step of the rasterizer runs in the CUDA
kernels of libvsr.so.  PyTorch provides device memory (tensors) and streams.
There is no CPU fallback: if the library is missing or a call fails, an
exception is raised.

Low-level functions carry the C names (vsr_make_map, vsr_setup, vsr_raster,
...) and take raw pointers; the classes Map and Scene and the function
raster() wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvsr.so")

VSR_OK = 0
VSR_ERR_INVALID_ARG, VSR_ERR_OOM, VSR_ERR_CUDA, VSR_ERR_BIN_OVERFLOW = -1, -2, -3, -4
VSR_ERR_FRAG_OVERFLOW, VSR_ERR_TIMEOUT, VSR_ERR_BUDGET, VSR_ERR_CANCELLED = -5, -6, -7, -8
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "tile bin overflow",
          -5: "fragment list overflow", -6: "device wait timed out", -7: "memory budget exceeded", -8: "cancelled"}
NO_ID = 0xFFFFFFFF
AOV_HORIZONTAL, AOV_DIAGONAL, AOV_VERTICAL, AOV_H4X3 = 0, 1, 2, 3
MAP_UNIVERSAL, MAP_RECTILINEAR, MAP_PANORAMA, MAP_DOME, MAP_EQUIRECT, MAP_CUBE = range(6)

# every symbol include/vsr.h declares
EXPORTS = ("vsr_make_map", "vsr_make_map_ex", "vsr_make_map_spec", "vsr_map_download_derivatives", "vsr_raster_pstep",
           "vsr_map_from_device", "vsr_map_update", "vsr_map_params_effective",
           "vsr_map_data", "vsr_map_download", "vsr_map_free", "vsr_setup", "vsr_scene_create", "vsr_scene_update",
           "vsr_scene_free", "vsr_scene_size", "vsr_raster", "vsr_raster_ex", "vsr_bin", "vsr_raster_tiles",
           "vsr_scene_bin_pairs", "vsr_raster_noalloc", "vsr_raster_dense", "vsr_batch_create", "vsr_batch_render",
           "vsr_batch_config", "vsr_batch_config_ex", "vsr_batch_set_mode", "vsr_batch_free", "vsr_serve_create", "vsr_serve_add_scene", "vsr_serve_submit",
           "vsr_serve_poll", "vsr_serve_wait", "vsr_serve_cancel", "vsr_serve_stats_get", "vsr_serve_now",
           "vsr_serve_destroy",
           "vsr_frags_create", "vsr_frags_free", "vsr_raster_shaded", "vsr_raster_backward",
           "vsr_render_host", "vsr_render_host_async", "vsr_render_host_wait", "vsr_status_str",
           "vsr_last_device_status", "vsr_version")


class VsrError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")


class MapParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_float), ("l", ctypes.c_float), ("s", ctypes.c_float), ("omega_deg", ctypes.c_float),
                ("W", ctypes.c_int), ("H", ctypes.c_int), ("aov", ctypes.c_int), ("strict_limits", ctypes.c_int)]


class MapSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("W", ctypes.c_int), ("H", ctypes.c_int), ("aov", ctypes.c_int),
                ("param", ctypes.c_float * 4), ("distortion", ctypes.c_float * 6), ("flags", ctypes.c_int)]


MAP_DERIVATIVES = 1


class ServeCfg(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int), ("max_maps", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_int), ("lens", MapParams), ("cam", ctypes.c_float * 12),
                ("id_dev", ctypes.c_void_p), ("depth_dev", ctypes.c_void_p), ("cov_dev", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("done", ctypes.c_int), ("map_cache_hit", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "cancelled", "map_hits",
                                              "map_misses", "map_evictions", "reruns", "bytes_in_use",
                                              "maps_cached", "queued")]


class RasterStats(ctypes.Structure):
    _fields_ = [("n_alg_dev", ctypes.c_void_p), ("n_exec_dev", ctypes.c_void_p), ("n_inside_dev", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libvsr.so (built by paper_2003_10558_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run `python -m paper_2003_10558_gb300.build` "
                               "(the rasterizer has no CPU fallback)")
        L = ctypes.CDLL(path)
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
        P = ctypes.POINTER
        sig = {
            "vsr_make_map": ([f32, f32, f32, f32, i32, i32, vp, P(vp)], i32),
            "vsr_make_map_ex": ([P(MapParams), vp, P(vp)], i32),
            "vsr_make_map_spec": ([P(MapSpec), vp, P(vp)], i32),
            "vsr_map_download_derivatives": ([vp, vp], i32),
            "vsr_raster_pstep": ([vp, vp, vp, vp, vp, vp], i32),
            "vsr_map_from_device": ([vp, i32, i32, vp, P(vp)], i32),
            "vsr_map_update": ([vp, P(MapParams), vp], i32),
            "vsr_map_params_effective": ([vp, P(MapParams)], i32),
            "vsr_map_data": ([vp, P(vp), P(i32), P(i32)], i32),
            "vsr_map_download": ([vp, vp], i32),
            "vsr_map_free": ([vp], None),
            "vsr_setup": ([vp, i64, vp, vp, P(vp)], i32),
            "vsr_scene_create": ([P(vp)], i32),
            "vsr_scene_update": ([vp, vp, i64, vp, vp], i32),
            "vsr_scene_free": ([vp], None),
            "vsr_scene_size": ([vp], i64),
            "vsr_raster": ([vp, vp, vp, vp, vp, vp], i32),
            "vsr_raster_ex": ([vp, vp, vp, vp, vp, P(RasterStats), vp], i32),
            "vsr_bin": ([vp, vp, vp], i32),
            "vsr_raster_tiles": ([vp, vp, vp, vp, vp, P(RasterStats), vp], i32),
            "vsr_scene_bin_pairs": ([vp, vp, P(i64)], i32),
            "vsr_raster_noalloc": ([vp, vp, vp, vp, vp, vp, vp], i32),
            "vsr_raster_dense": ([vp, vp, vp, vp, vp, vp], i32),
            "vsr_batch_create": ([P(vp)], i32),
            "vsr_batch_render": ([vp, i32, vp, vp, i64, vp, vp, vp, vp, vp], i32),
            "vsr_batch_config": ([vp, P(i32), P(i32), P(i32)], i32),
            "vsr_batch_config_ex": ([vp, P(i32), P(i32), P(i32), P(i32)], i32),
            "vsr_batch_set_mode": ([vp, i32], i32),
            "vsr_batch_free": ([vp], None),
            "vsr_serve_create": ([P(ServeCfg), P(vp)], i32),
            "vsr_serve_add_scene": ([vp, vp, i64, P(i32)], i32),
            "vsr_serve_submit": ([vp, P(Request), P(ctypes.c_uint64)], i32),
            "vsr_serve_poll": ([vp, ctypes.c_uint64, P(Result)], i32),
            "vsr_serve_wait": ([vp, ctypes.c_uint64, P(Result)], i32),
            "vsr_serve_cancel": ([vp, ctypes.c_uint64], i32),
            "vsr_serve_stats_get": ([vp, P(ServeStats)], i32),
            "vsr_serve_now": ([], ctypes.c_double),
            "vsr_serve_destroy": ([vp], i32),
            "vsr_render_host": ([vp, vp, vp, i64, vp, vp, vp, vp, vp], i32),
            "vsr_render_host_async": ([vp, vp, vp, i64, vp, vp, vp, vp, vp], i32),
            "vsr_render_host_wait": ([vp], i32),
            "vsr_frags_create": ([P(vp)], i32),
            "vsr_frags_free": ([vp], None),
            "vsr_raster_shaded": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
            "vsr_raster_backward": ([vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
            "vsr_status_str": ([i32], ctypes.c_char_p),
            "vsr_last_device_status": ([], i32),
            "vsr_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def check(code, what=""):
    if code != VSR_OK:
        raise VsrError(code, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _cam_array(cam):
    c = np.ascontiguousarray(np.asarray(cam, dtype=np.float32).ravel())
    if c.size != 12:
        raise ValueError("camera must have 12 floats: eye xyz then 3x3 rotation")
    return c


def last_device_status():
    """Synchronise and return (and clear) the device-side status word."""
    return load().vsr_last_device_status()


class Map:
    """A device-resident perspective map (float4 [H, W] = G xyz, delta) with
    its tile view cones."""

    def __init__(self, W, H, k, l, s, omega_deg, aov=AOV_HORIZONTAL, strict=False, stream=None, _handle=None):
        L = load()
        self.h = ctypes.c_void_p()
        if _handle is not None:
            self.h = _handle
        else:
            p = MapParams(k, l, s, omega_deg, W, H, aov, int(strict))
            check(L.vsr_make_map_ex(ctypes.byref(p), _stream_ptr(stream), ctypes.byref(self.h)), "vsr_make_map_ex")
        self._keep = None

    @classmethod
    def from_spec(cls, kind, W, H, param=(), distortion=(), aov=AOV_HORIZONTAL, derivatives=False, stream=None):
        """A map of another projection (MAP_RECTILINEAR, MAP_PANORAMA,
        MAP_DOME, MAP_EQUIRECT, MAP_CUBE) or a Universal / rectilinear map
        with Brown-Conrady distortion (k1, k2, p1, p2, q1, q2).
        derivatives=True keeps the map's differences for raster(pstep=True)."""
        sp = MapSpec()
        sp.kind, sp.W, sp.H, sp.aov = int(kind), int(W), int(H), int(aov)
        sp.flags = MAP_DERIVATIVES if derivatives else 0
        for q, x in enumerate(param):
            sp.param[q] = float(x)
        for q, x in enumerate(distortion):
            sp.distortion[q] = float(x)
        h = ctypes.c_void_p()
        check(load().vsr_make_map_spec(ctypes.byref(sp), _stream_ptr(stream), ctypes.byref(h)), "vsr_make_map_spec")
        return cls(W, H, 0, 0, 0, 0, _handle=h)

    @classmethod
    def from_tensor(cls, xyzd, stream=None):
        """Map from a CUDA float32 tensor [H, W, 4] (copied)."""
        import torch
        if not (xyzd.is_cuda and xyzd.dtype == torch.float32 and xyzd.dim() == 3 and xyzd.shape[2] == 4):
            raise ValueError("expected a CUDA float32 tensor [H, W, 4]")
        xyzd = xyzd.contiguous()
        h = ctypes.c_void_p()
        H, W = xyzd.shape[:2]
        check(load().vsr_map_from_device(_dptr(xyzd), W, H, _stream_ptr(stream), ctypes.byref(h)),
              "vsr_map_from_device")
        m = cls(W, H, 0, 0, 0, 0, _handle=h)
        m._keep = xyzd  # alive until the async copy is done
        return m

    def update(self, W, H, k, l, s, omega_deg, aov=AOV_HORIZONTAL, strict=False, stream=None):
        p = MapParams(k, l, s, omega_deg, W, H, aov, int(strict))
        check(load().vsr_map_update(self.h, ctypes.byref(p), _stream_ptr(stream)), "vsr_map_update")

    @property
    def shape(self):
        W, H = ctypes.c_int(), ctypes.c_int()
        check(load().vsr_map_data(self.h, None, ctypes.byref(W), ctypes.byref(H)), "vsr_map_data")
        return H.value, W.value

    def params(self):
        p = MapParams()
        check(load().vsr_map_params_effective(self.h, ctypes.byref(p)), "vsr_map_params_effective")
        return dict(k=p.k, l=p.l, s=p.s, omega_deg=p.omega_deg, W=p.W, H=p.H, aov=p.aov, strict=p.strict_limits)

    def download(self):
        H, W = self.shape
        out = np.empty((H, W, 4), dtype=np.float32)
        check(load().vsr_map_download(self.h, out.ctypes.data_as(ctypes.c_void_p)), "vsr_map_download")
        return out

    def download_derivatives(self):
        """(d_i G, d_j G) [H, W, 6] of a map made with derivatives=True."""
        H, W = self.shape
        out = np.empty((H, W, 8), dtype=np.float32)
        check(load().vsr_map_download_derivatives(self.h, out.ctypes.data_as(ctypes.c_void_p)),
              "vsr_map_download_derivatives")
        return np.concatenate([out[..., 0:3], out[..., 4:7]], axis=-1)

    def tensor(self):
        """A torch copy of the map, [H, W, 4] float32 on the device."""
        import torch
        H, W = self.shape
        return torch.from_numpy(self.download()).cuda()

    def free(self):
        if self.h:
            load().vsr_map_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Scene:
    """Set-up records of T triangles for one camera (device-resident)."""

    def __init__(self, tris=None, cam=None, stream=None):
        L = load()
        self.h = ctypes.c_void_p()
        check(L.vsr_scene_create(ctypes.byref(self.h)), "vsr_scene_create")
        if tris is not None:
            self.update(tris, cam, stream)

    def update(self, tris, cam=None, stream=None):
        import torch
        if cam is None:
            cam = [0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1]
        if not (tris.is_cuda and tris.dtype == torch.float32):
            raise ValueError("triangles must be a CUDA float32 tensor [T, 3, 3]")
        tris = tris.contiguous()
        T = tris.numel() // 9
        c = _cam_array(cam)
        check(load().vsr_scene_update(self.h, _dptr(tris) if T else None, T, c.ctypes.data_as(ctypes.c_void_p),
                                      _stream_ptr(stream)), "vsr_scene_update")
        self._keep = tris

    @property
    def T(self):
        return int(load().vsr_scene_size(self.h))

    def bin_pairs(self, stream=None):
        n = ctypes.c_int64()
        check(load().vsr_scene_bin_pairs(self.h, _stream_ptr(stream), ctypes.byref(n)), "vsr_scene_bin_pairs")
        return n.value

    def free(self):
        if self.h:
            load().vsr_scene_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def bin(m: Map, sc: Scene, stream=None):
    """Build the tile bins of (m, sc) (vsr_bin)."""
    check(load().vsr_bin(m.h, sc.h, _stream_ptr(stream)), "vsr_bin")


def raster_pstep(m: Map, sc: Scene, out=None, stream=None):
    """Rasterize with the per-fragment pixel step (vsr_raster_pstep); the map
    needs derivatives.  Returns id (int32 view of uint32), depth, cov."""
    import torch
    H, W = m.shape
    dev = torch.device("cuda")
    if out is None:
        out = {"id": torch.empty((H, W), dtype=torch.int32, device=dev),
               "depth": torch.empty((H, W), dtype=torch.float32, device=dev),
               "cov": torch.empty((H, W), dtype=torch.float32, device=dev)}
    check(load().vsr_raster_pstep(m.h, sc.h, _dptr(out.get("id")), _dptr(out.get("depth")), _dptr(out.get("cov")),
                                  _stream_ptr(stream)), "vsr_raster_pstep")
    return out


def raster(m: Map, sc: Scene, out=None, stats=False, n_inside=False, stream=None, binned=False):
    """Rasterize: returns dict of CUDA tensors id (int32 view of uint32),
    depth, cov [H, W]; with stats=True also n_alg, n_exec (python ints, sync);
    with n_inside=True the per-pixel count of centre-inside triangles.
    stats="exec" counts only the evaluated pairs (the kernel then culls as in
    a timed run; counting algorithmic tests disables the edge-plane cull).
    binned=True reuses the bins of the last bin() call (vsr_raster_tiles)."""
    import torch
    H, W = m.shape
    dev = torch.device("cuda")
    if out is None:
        out = {"id": torch.empty((H, W), dtype=torch.int32, device=dev),
               "depth": torch.empty((H, W), dtype=torch.float32, device=dev),
               "cov": torch.empty((H, W), dtype=torch.float32, device=dev)}
    st = None
    cnt = None
    if stats or n_inside:
        cnt = torch.zeros(2, dtype=torch.int64, device=dev)
        if n_inside:
            out["n_inside"] = torch.empty((H, W), dtype=torch.int32, device=dev)
        st = RasterStats(cnt.data_ptr() if stats is True else None, cnt.data_ptr() + 8 if stats else None,
                         out["n_inside"].data_ptr() if n_inside else None)
    fn = load().vsr_raster_tiles if binned else load().vsr_raster_ex
    check(fn(m.h, sc.h, _dptr(out.get("id")), _dptr(out.get("depth")), _dptr(out.get("cov")),
             ctypes.byref(st) if st is not None else None, _stream_ptr(stream)), "vsr_raster")
    if stats:
        c = cnt.cpu()
        out["n_alg"], out["n_exec"] = int(c[0]), int(c[1])
    return out


def raster_dense(m: Map, sc: Scene, out=None, stream=None):
    """The dense reference (vsr_raster_dense): every pixel against every
    triangle of the scene, no tile bins.  Same outputs as raster()."""
    import torch
    H, W = m.shape
    dev = torch.device("cuda")
    if out is None:
        out = {"id": torch.empty((H, W), dtype=torch.int32, device=dev),
               "depth": torch.empty((H, W), dtype=torch.float32, device=dev),
               "cov": torch.empty((H, W), dtype=torch.float32, device=dev)}
    check(load().vsr_raster_dense(m.h, sc.h, _dptr(out.get("id")), _dptr(out.get("depth")), _dptr(out.get("cov")),
                                  _stream_ptr(stream)), "vsr_raster_dense")
    return out


def _host_frame_args(m, tris, cam, want, out):
    if cam is None:
        cam = [0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1]
    tris = np.ascontiguousarray(tris, dtype=np.float32)
    T = tris.size // 9
    if out is None:
        H, W = m.shape
        out = {}
        if "id" in want:
            out["id"] = np.empty((H, W), dtype=np.uint32)
        if "depth" in want:
            out["depth"] = np.empty((H, W), dtype=np.float32)
        if "cov" in want:
            out["cov"] = np.empty((H, W), dtype=np.float32)
    c = _cam_array(cam)

    def p(a):  # the array's address (cheaper than a.ctypes.data_as)
        return None if a is None else ctypes.c_void_p(a.__array_interface__["data"][0])

    return (p(tris), T, p(c), p(out.get("id")), p(out.get("depth")), p(out.get("cov"))), (tris, c), out


def render_host(m: Map, sc: Scene, tris: np.ndarray, cam=None, want=("id", "depth", "cov"), out=None, stream=None):
    """End to end from host memory (vsr_render_host): numpy triangles in,
    numpy id (uint32) / depth / cov out.  `out` may hold preallocated
    (ideally pinned) arrays."""
    args, _keep, out = _host_frame_args(m, tris, cam, want, out)
    check(load().vsr_render_host(m.h, sc.h, *args, _stream_ptr(stream)), "vsr_render_host")
    return out


def render_host_async(m: Map, sc: Scene, tris: np.ndarray, cam=None, want=("id", "depth", "cov"), out=None,
                      stream=None):
    """Queue one frame from host memory (vsr_render_host_async) and return its
    outputs (filled once render_host_wait(sc) has returned).  The arrays must
    stay alive and untouched until then; pinned ones are written in place."""
    args, keep, out = _host_frame_args(m, tris, cam, want, out)
    check(load().vsr_render_host_async(m.h, sc.h, *args, _stream_ptr(stream)), "vsr_render_host_async")
    sc._host_keep = (keep, out)
    return out


def render_host_wait(sc: Scene):
    """Wait for the scene's queued host frame: 0 (complete) or
    VSR_ERR_BIN_OVERFLOW (it outgrew the scene's bins: render it again);
    raises on a CUDA error."""
    r = load().vsr_render_host_wait(sc.h)
    sc._host_keep = None
    if r not in (0, VSR_ERR_BIN_OVERFLOW):
        check(r, "vsr_render_host_wait")
    return r


class Batch:
    """Batched multi-view rendering of one scene (vsr_batch_*): one CUDA
    graph of per-view chains over parallel streams, replayed while the
    configuration (maps, scene buffer, outputs) is unchanged."""

    def __init__(self):
        self.h = ctypes.c_void_p()
        check(load().vsr_batch_create(ctypes.byref(self.h)), "vsr_batch_create")
        self._keep = None

    def render(self, maps, tris, cams, outs, stream=None):
        """maps: list of Map; tris: CUDA float32 [T, 3, 3]; cams: [V, 12];
        outs: list of dicts with CUDA tensors id / depth / cov per view."""
        import torch
        V = len(maps)
        if not (tris.is_cuda and tris.dtype == torch.float32):
            raise ValueError("triangles must be a CUDA float32 tensor [T, 3, 3]")
        tris = tris.contiguous()
        T = tris.numel() // 9
        c = np.ascontiguousarray(np.asarray(cams, dtype=np.float32).reshape(V, 12))
        mh = (ctypes.c_void_p * V)(*[m.h.value for m in maps])

        def ptrs(key):
            return (ctypes.c_void_p * V)(*[o[key].data_ptr() if o.get(key) is not None else None for o in outs])

        ids, depths, covs = ptrs("id"), ptrs("depth"), ptrs("cov")
        check(load().vsr_batch_render(self.h, V, mh, _dptr(tris) if T else None, T,
                                      c.ctypes.data_as(ctypes.c_void_p), ids, depths, covs, _stream_ptr(stream)),
              "vsr_batch_render")
        self._keep = (tris, maps, outs)

    AUTO, CHAINS, POOLED = 0, 1, 2  # vsr_batch_set_mode

    def set_mode(self, mode):
        """Graph kinds the autotuner may keep (Batch.AUTO / CHAINS / POOLED)."""
        check(load().vsr_batch_set_mode(self.h, int(mode)), "vsr_batch_set_mode")

    def config(self):
        g, r, sp, po = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(load().vsr_batch_config_ex(self.h, ctypes.byref(g), ctypes.byref(r), ctypes.byref(sp), ctypes.byref(po)),
              "vsr_batch_config_ex")
        return {"streams": g.value, "graphed": bool(r.value), "split_max": sp.value, "pooled": bool(po.value),
                "pool_groups": po.value}

    def free(self):
        if self.h:
            load().vsr_batch_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Rendering server with continuous batching (vsr_serve_*)."""

    def __init__(self, budget_bytes=40 << 30, slots=8, max_maps=0):
        self.h = ctypes.c_void_p()
        cfg = ServeCfg(int(budget_bytes), int(slots), int(max_maps))
        check(load().vsr_serve_create(ctypes.byref(cfg), ctypes.byref(self.h)), "vsr_serve_create")
        self._scenes = []

    def add_scene(self, tris):
        """Resident triangles: a CUDA float32 tensor [T, 3, 3] kept alive here."""
        tris = tris.contiguous()
        self._scenes.append(tris)
        idx = ctypes.c_int()
        T = tris.numel() // 9
        check(load().vsr_serve_add_scene(self.h, _dptr(tris) if T else None, T, ctypes.byref(idx)),
              "vsr_serve_add_scene")
        return idx.value

    @staticmethod
    def now():
        return load().vsr_serve_now()

    def submit(self, scene, lens, cam, out):
        """lens: dict(W, H, k, l, s, omega[, aov, strict]); out: dict of
        CUDA tensors id / depth / cov (kept alive by the caller until done).
        Returns the ticket."""
        r = Request()
        r.scene = scene
        r.lens = MapParams(lens["k"], lens["l"], lens["s"], lens["omega"], lens["W"], lens["H"],
                           lens.get("aov", 0), int(lens.get("strict", False)))
        c = _cam_array(cam)
        for q in range(12):
            r.cam[q] = float(c[q])
        r.id_dev = out["id"].data_ptr() if out.get("id") is not None else None
        r.depth_dev = out["depth"].data_ptr() if out.get("depth") is not None else None
        r.cov_dev = out["cov"].data_ptr() if out.get("cov") is not None else None
        t = ctypes.c_uint64()
        check(load().vsr_serve_submit(self.h, ctypes.byref(r), ctypes.byref(t)), "vsr_serve_submit")
        return t.value

    @staticmethod
    def _res(res):
        return {"status": res.status, "done": bool(res.done), "map_cache_hit": bool(res.map_cache_hit),
                "t_submit": res.t_submit, "t_start": res.t_start, "t_done": res.t_done}

    def poll(self, ticket):
        res = Result()
        check(load().vsr_serve_poll(self.h, ticket, ctypes.byref(res)), "vsr_serve_poll")
        return self._res(res)

    def wait(self, ticket):
        res = Result()
        check(load().vsr_serve_wait(self.h, ticket, ctypes.byref(res)), "vsr_serve_wait")
        return self._res(res)

    def cancel(self, ticket):
        return load().vsr_serve_cancel(self.h, ticket) == VSR_OK

    def stats(self):
        st = ServeStats()
        check(load().vsr_serve_stats_get(self.h, ctypes.byref(st)), "vsr_serve_stats_get")
        return {n: getattr(st, n) for n, _ in ServeStats._fields_}

    def close(self):
        if self.h:
            load().vsr_serve_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Differentiable rendering: the shaded image I = front-to-back merge of
# c_t |N-hat_t . G| and its hand-written adjoint (vsr_raster_shaded /
# vsr_raster_backward).

class Frags:
    """Fragment lists of the last shaded forward and the backward workspace."""

    def __init__(self):
        self.h = ctypes.c_void_p()
        check(load().vsr_frags_create(ctypes.byref(self.h)), "vsr_frags_create")

    def free(self):
        if self.h:
            load().vsr_frags_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def raster_shaded(m: Map, sc: Scene, frags: Frags, colors=None, out=None, stream=None):
    """Shaded forward: dict of CUDA tensors image, cov, depth [H, W] float32
    and id (int32 view of uint32).  colors: CUDA float32 [T] or None (all 1)."""
    import torch
    H, W = m.shape
    dev = torch.device("cuda")
    if out is None:
        out = {"image": torch.empty((H, W), dtype=torch.float32, device=dev),
               "cov": torch.empty((H, W), dtype=torch.float32, device=dev),
               "depth": torch.empty((H, W), dtype=torch.float32, device=dev),
               "id": torch.empty((H, W), dtype=torch.int32, device=dev)}
    if colors is not None:
        if not (colors.is_cuda and colors.dtype == torch.float32 and colors.numel() == sc.T):
            raise ValueError("colors must be a CUDA float32 tensor with one value per triangle")
        colors = colors.contiguous()
    check(load().vsr_raster_shaded(m.h, sc.h, _dptr(colors), frags.h, _dptr(out.get("image")), _dptr(out.get("cov")),
                                   _dptr(out.get("id")), _dptr(out.get("depth")), _stream_ptr(stream)),
          "vsr_raster_shaded")
    return out


def raster_backward(m: Map, sc: Scene, frags: Frags, tris, colors=None, id=None, dimage=None, dcov=None,
                    ddepth=None, want=("tris", "colors", "lens"), stream=None):
    """Adjoint of the last raster_shaded of (m, sc) into frags: returns dict
    with dtris [T, 3, 3], dcolors [T] (float32 CUDA) and dlens (float64 CUDA
    [4] = d/d(k, l, s, Omega in degrees)), as requested by `want`."""
    import torch
    T = sc.T
    dev = torch.device("cuda")

    def c(t):
        return None if t is None else t.contiguous()

    dimage, dcov, ddepth, colors, tris = c(dimage), c(dcov), c(ddepth), c(colors), c(tris)
    out = {}
    if "tris" in want:
        out["dtris"] = torch.empty((T, 3, 3), dtype=torch.float32, device=dev)
    if "colors" in want:
        out["dcolors"] = torch.empty((T,), dtype=torch.float32, device=dev)
    if "lens" in want:
        out["dlens"] = torch.empty((4,), dtype=torch.float64, device=dev)
    check(load().vsr_raster_backward(m.h, sc.h, _dptr(tris), _dptr(colors), frags.h, _dptr(id), _dptr(dimage),
                                     _dptr(dcov), _dptr(ddepth), _dptr(out.get("dtris")), _dptr(out.get("dcolors")),
                                     _dptr(out.get("dlens")), _stream_ptr(stream)), "vsr_raster_backward")
    return out


class ShadedRenderer:
    """Device state of differentiable rendering at one resolution: the map
    (regenerated for each lens), the scene set-up and the fragment lists."""

    def __init__(self, W, H, aov=AOV_HORIZONTAL, cam=None):
        self.W, self.H, self.aov = int(W), int(H), int(aov)
        self.cam = [0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1] if cam is None else list(np.asarray(cam).ravel())
        self.map = None
        self.scene = Scene()
        self.frags = Frags()
        self.generation = 0  # forwards run so far; a backward must belong to the latest

    def set_lens(self, k, l, s, omega_deg, stream=None):
        if self.map is None:
            self.map = Map(self.W, self.H, k, l, s, omega_deg, self.aov, stream=stream)
        else:
            self.map.update(self.W, self.H, k, l, s, omega_deg, self.aov, stream=stream)
        p = self.map.params()
        return (p["k"], p["l"], p["s"], p["omega_deg"])


def _autograd_function():
    import torch

    class RenderShaded(torch.autograd.Function):
        """(tris [T,3,3] f32 CUDA, colors [T] f32 CUDA, lens [4] f64 (k, l, s,
        Omega deg), renderer) -> (image, cov, depth, id).  Backward through
        vsr_raster_backward; a lens parameter clamped by the limits gets a
        zero gradient."""

        @staticmethod
        def forward(ctx, tris, colors, lens, renderer):
            lv = [float(x) for x in lens.detach().cpu().double()]
            eff = renderer.set_lens(*lv)
            tris_c = tris.detach().contiguous()
            col_c = colors.detach().contiguous()
            renderer.scene.update(tris_c, renderer.cam)
            out = raster_shaded(renderer.map, renderer.scene, renderer.frags, col_c)
            renderer.generation += 1
            ctx.generation = renderer.generation
            ctx.renderer = renderer
            ctx.open = [abs(e - v) <= 1e-6 * max(1.0, abs(v)) for e, v in zip(eff, lv)]
            ctx.lens_meta = (lens.dtype, lens.device)
            ctx.save_for_backward(tris_c, col_c, out["id"])
            ctx.mark_non_differentiable(out["id"])
            return out["image"], out["cov"], out["depth"], out["id"]

        @staticmethod
        def backward(ctx, dimage, dcov, ddepth, did):
            tris, colors, ids = ctx.saved_tensors
            r = ctx.renderer
            if ctx.generation != r.generation:
                raise VsrError(-1, "backward of a shaded render whose renderer has run another forward since")
            want = []
            if ctx.needs_input_grad[0]:
                want.append("tris")
            if ctx.needs_input_grad[1]:
                want.append("colors")
            if ctx.needs_input_grad[2]:
                want.append("lens")
            g = raster_backward(r.map, r.scene, r.frags, tris, colors, ids, dimage, dcov, ddepth, want=tuple(want))
            dl = None
            if "dlens" in g:
                dl = g["dlens"].to(device=ctx.lens_meta[1], dtype=ctx.lens_meta[0])
                dl = dl * torch.tensor([1.0 if o else 0.0 for o in ctx.open], dtype=dl.dtype, device=dl.device)
            return g.get("dtris"), g.get("dcolors"), dl, None

    return RenderShaded


_render_fn = None


def render_shaded(tris, colors, lens, renderer: ShadedRenderer):
    """Differentiable render: (image, cov, depth, id) with gradients to tris,
    colors and lens (a float64 tensor [4] = k, l, s, Omega in degrees).
    One frame per renderer at a time: run backward before the renderer's
    next forward (a stale backward raises VsrError)."""
    global _render_fn
    if _render_fn is None:
        _render_fn = _autograd_function()
    return _render_fn.apply(tris, colors, lens, renderer)
