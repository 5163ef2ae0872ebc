"""FP64 CPU oracle of the visual-sphere rasterizer (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``vsr_oracle.c`` (plain C, double precision, brute
force over every pixel x triangle pair).  Each function there cites the part
of the paper it follows: the Universal perspective 2D->3D map and its limits
(Sec. 2), the global delta (Sec. 1.1.1), the edge-plane normals (Sec. 1.1), the
miter / smallest circle (Sec. 1.1.2), the ray-plane depth (Sec. 1.1.4) and the
front-to-back mask merge (Sec. 1.4).

Every function of this oracle is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force and textbook routines; none is marked
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

REC = 20  # doubles per set-up triangle
REC_N1, REC_N2, REC_N3, REC_S, REC_C, REC_N, REC_D, REC_VALID, REC_SIGMA, REC_SR = 0, 3, 6, 9, 12, 13, 16, 17, 18, 19
AOV = {"horizontal": 0, "diagonal": 1, "vertical": 2, "h4x3": 3}
NO_ID = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile vsr_oracle.c with gcc into oracle/_build/liboracle.so.

    -ffp-contract=off keeps x86 and Arm results identical (no fused
    multiply-adds the source does not write)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            vp = ctypes.c_void_p
            lib.orc_limits.argtypes = [d, d, d, d, i32, vp]
            lib.orc_view_coord.argtypes = [d, d, d, i32, vp]
            lib.orc_map_dir.argtypes = [d, d, vp, vp]
            lib.orc_map_dir.restype = i32
            lib.orc_map_dirs.argtypes = [i64, vp, vp, i32, i32, vp, i32, vp, vp]
            lib.orc_map_inverse.argtypes = [vp, vp, vp]
            lib.orc_map.argtypes = [i32, i32, vp, i32, vp, i32]
            lib.orc_map.restype = i32
            lib.orc_setup.argtypes = [i64, vp, vp, vp]
            lib.orc_raster.argtypes = [i32, i32, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, i32]
            lib.orc_raster.restype = i64
            lib.orc_shade.argtypes = [i32, i32, vp, i64, vp, vp, i64, vp, vp, i32]
            lib.orc_shade.restype = i32
            lib.orc_setup64.argtypes = [i64, vp, vp, vp]
            lib.orc_map_tangent.argtypes = [i32, i32, vp, i32, i32, vp]
            lib.orc_map_tangent.restype = i32
            lib.orc_shade_grad.argtypes = [i32, i32, vp, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_shade_grad.restype = i32
            lib.orc_setup_grad.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.orc_map_spec.argtypes = [i32, i32, i32, vp, vp, i32, vp, vp]
            lib.orc_raster_pstep.argtypes = [i32, i32, vp, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, i32]
            lib.orc_raster_pstep.restype = i64
            lib.orc_map_spec.restype = i32
            lib.orc_map_spec_dirs.argtypes = [i64, vp, vp, i32, i32, i32, vp, vp, i32, vp, vp]
            assert lib.orc_record_size() == REC
            _lib = lib
            del P
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def limits(k, l, s, omega_deg, strict=False):
    """Effective (k, l, s, omega_deg) after the paper's parameter limits."""
    out = np.zeros(4)
    _load().orc_limits(k, l, s, omega_deg, int(strict), _ptr(out))
    return tuple(float(v) for v in out)


def view_coord(fs, ft, aspect, aov=0):
    out = np.zeros(2)
    _load().orc_view_coord(fs, ft, aspect, aov, _ptr(out))
    return float(out[0]), float(out[1])


def map_dir(x, y, params):
    """Direction of view coordinate (x, y); params = effective (k,l,s,omega_deg).
    Returns (v[3], valid)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    v = np.zeros(3)
    ok = _load().orc_map_dir(float(x), float(y), _ptr(p), _ptr(v))
    return v, bool(ok)


def map_dirs(fs, ft, W, H, params, aov=0):
    """Vectorised map function at texture coordinates fs, ft (any shape)."""
    fs = np.ascontiguousarray(fs, dtype=np.float64)
    ft = np.ascontiguousarray(ft, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    n = fs.size
    v = np.zeros((n, 3))
    valid = np.zeros(n, dtype=np.int32)
    _load().orc_map_dirs(n, _ptr(fs), _ptr(ft), W, H, _ptr(p), aov, _ptr(v), _ptr(valid))
    return v.reshape(fs.shape + (3,)), valid.reshape(fs.shape).astype(bool)


def map_inverse(v, params):
    v = np.ascontiguousarray(v, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(2)
    _load().orc_map_inverse(_ptr(v), _ptr(p), _ptr(out))
    return float(out[0]), float(out[1])


def make_map(W, H, k, l, s, omega_deg, aov=0, strict=False, nthreads=0):
    """FP64 perspective map [H, W, 4] = (v_x, v_y, v_z, delta) and the
    effective parameters."""
    eff = np.asarray(limits(k, l, s, omega_deg, strict))
    out = np.zeros((H, W, 4))
    rc = _load().orc_map(W, H, _ptr(eff), aov, _ptr(out), nthreads)
    if rc != 0:
        raise ValueError(f"orc_map failed ({rc})")
    return out, tuple(eff)


def setup(tris, cam=None):
    """Set-up records [T, REC] from FP32 world triangles [T, 3, 3]."""
    tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    if cam is None:
        cam = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.float32)
    cam = np.ascontiguousarray(cam, dtype=np.float32)
    rec = np.zeros((tris.shape[0], REC))
    _load().orc_setup(tris.shape[0], _ptr(tris), _ptr(cam), _ptr(rec))
    return rec


def raster(map_, rec, pixels=None, nthreads=0, extras=False):
    """Brute-force raster.  map_: [H, W, 4] (float64 or float32, promoted
    exactly); rec: [T, REC]; pixels: flat indices j*W+i or None for all.

    Returns dict with id (uint32), depth, cov (float64), n_alg (int) and, with
    extras=True, sum_mf, n_inside, n_frag."""
    H, W = map_.shape[:2]
    m = np.ascontiguousarray(map_, dtype=np.float64)
    rec = np.ascontiguousarray(rec, dtype=np.float64)
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64).ravel()
        npix = pix.size
    out = {
        "id": np.zeros(npix, dtype=np.uint32),
        "depth": np.zeros(npix),
        "cov": np.zeros(npix),
    }
    sm = ni = nf = None
    if extras:
        sm = out["sum_mf"] = np.zeros(npix)
        ni = out["n_inside"] = np.zeros(npix, dtype=np.int32)
        nf = out["n_frag"] = np.zeros(npix, dtype=np.int32)
    n_alg = _load().orc_raster(W, H, _ptr(m), rec.shape[0], _ptr(rec), npix, _ptr(pix), _ptr(out["id"]),
                               _ptr(out["depth"]), _ptr(out["cov"]), _ptr(sm), _ptr(ni), _ptr(nf), nthreads)
    if n_alg < 0:
        raise ValueError("orc_raster: bad sizes")
    out["n_alg"] = int(n_alg)
    if pixels is None:
        for key in list(out):
            if isinstance(out[key], np.ndarray):
                out[key] = out[key].reshape(H, W)
    return out


def shade(map_, rec, colors, pixels=None, nthreads=0):
    """Shaded image (front-to-back merge of c_t |N-hat_t . G| over the
    fragments): [H, W] for pixels=None, else one value per listed pixel."""
    H, W = map_.shape[:2]
    m = np.ascontiguousarray(map_, dtype=np.float64)
    rec = np.ascontiguousarray(rec, dtype=np.float64)
    col = np.ascontiguousarray(colors, dtype=np.float64)
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64).ravel()
        npix = pix.size
    img = np.zeros(npix)
    if _load().orc_shade(W, H, _ptr(m), rec.shape[0], _ptr(rec), _ptr(col), npix, _ptr(pix), _ptr(img), nthreads):
        raise ValueError("orc_shade: bad sizes")
    return img.reshape(H, W) if pixels is None else img


IDENTITY_CAM = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.float64)


def setup64(tris, cam=None):
    """Set-up records from float64 world triangles [T, 3, 3] and camera."""
    tris = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
    cam = IDENTITY_CAM if cam is None else np.ascontiguousarray(cam, dtype=np.float64)
    rec = np.zeros((tris.shape[0], REC))
    _load().orc_setup64(tris.shape[0], _ptr(tris), _ptr(cam), _ptr(rec))
    return rec


def map_tangent(W, H, params, which, aov=0):
    """d(map)/d(param) [H, W, 4] for which in 0..3 = k, l, s, Omega (degrees),
    at the effective parameters `params` (complex step)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros((H, W, 4))
    if _load().orc_map_tangent(W, H, _ptr(p), aov, which, _ptr(out)):
        raise ValueError("orc_map_tangent failed")
    return out


def shade_grad(map_, rec, colors, dimage, pixels=None, dcov=None, ddepth=None):
    """Adjoint of the shaded image (plus coverage / depth) -> (drec [T, REC],
    dcolors [T], dmap [npix, 4] = d/d(G, delta))."""
    H, W = map_.shape[:2]
    m = np.ascontiguousarray(map_, dtype=np.float64)
    rec = np.ascontiguousarray(rec, dtype=np.float64)
    col = np.ascontiguousarray(colors, dtype=np.float64)
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64).ravel()
        npix = pix.size

    def vec(a):
        return None if a is None else np.ascontiguousarray(a, dtype=np.float64).ravel()

    dI, dC, dD = vec(dimage), vec(dcov), vec(ddepth)
    T = rec.shape[0]
    drec = np.zeros((T, REC))
    dcol = np.zeros(T)
    dmap = np.zeros((npix, 4))
    if _load().orc_shade_grad(W, H, _ptr(m), T, _ptr(rec), _ptr(col), npix, _ptr(pix), _ptr(dI), _ptr(dC),
                              _ptr(dD), _ptr(drec), _ptr(dcol), _ptr(dmap)):
        raise ValueError("orc_shade_grad: bad sizes")
    return drec, dcol, dmap


def setup_grad(tris, rec, drec, cam=None):
    """World-vertex gradients [T, 3, 3] from record gradients."""
    tris = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
    cam = IDENTITY_CAM if cam is None else np.ascontiguousarray(cam, dtype=np.float64)
    out = np.zeros((tris.shape[0], 9))
    _load().orc_setup_grad(tris.shape[0], _ptr(tris), _ptr(cam), _ptr(np.ascontiguousarray(rec)),
                           _ptr(np.ascontiguousarray(drec)), _ptr(out))
    return out.reshape(-1, 3, 3)


def render_grad(map_, params, tris, colors, dimage, pixels=None, dcov=None, ddepth=None, cam=None, aov=0,
                tangents=None):
    """The oracle's analytic gradient of sum(dimage * I + dcov * cov +
    ddepth * depth) over the listed pixels: returns dict with dtris [T, 3, 3],
    dcolors [T] and dlens [4] = d/d(k, l, s, Omega in degrees).

    map_ is the map the image is computed on (FP64, or an FP32 map promoted);
    params its effective parameters, for the map tangents."""
    H, W = map_.shape[:2]
    rec = setup64(tris, cam)
    drec, dcol, dmap = shade_grad(map_, rec, colors, dimage, pixels, dcov, ddepth)
    dtris = setup_grad(tris, rec, drec, cam)
    if tangents is None:
        tangents = [map_tangent(W, H, params, j, aov) for j in range(4)]
    dlens = np.zeros(4)
    for j in range(4):
        tj = tangents[j].reshape(-1, 4)
        if pixels is not None:
            tj = tj[np.asarray(pixels, dtype=np.int64).ravel()]
        dlens[j] = float(np.sum(tj * dmap))
    return {"dtris": dtris, "dcolors": dcol, "dlens": dlens, "dmap": dmap, "drec": drec}


def shade_fd(verts, colors, lens, pixels, W, H, h=1e-6, which=("k", "l", "s", "omega"), vert_idx=(),
             weights=None, cam=None, aov=0):
    """FP64 central differences of sum(weights * I) over `pixels` (test
    infrastructure for the gradient checks): d/dk, d/dl, d/ds, d/dOmega of the
    map (rebuilt at +-h) and d/d(vertex coordinate) for (t, v, c) in vert_idx,
    the vertices taken in float64 so that +-h is represented exactly."""
    verts = np.asarray(verts, dtype=np.float64)
    w = None if weights is None else np.asarray(weights, dtype=np.float64).ravel()

    def total(lens_, verts_):
        m, _ = make_map(W, H, lens_["k"], lens_["l"], lens_["s"], lens_["omega"], aov=aov)
        img = shade(m, setup64(verts_, cam), colors, pixels)
        return float(np.sum(img if w is None else img * w))

    out = {}
    for name in which:
        lp, lm = dict(lens), dict(lens)
        lp[name] += h
        lm[name] -= h
        out[name] = (total(lp, verts) - total(lm, verts)) / (2 * h)
    if vert_idx:
        m0, _ = make_map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"], aov=aov)
        for (t, v, c) in vert_idx:
            vp, vm = verts.copy(), verts.copy()
            vp[t, v, c] += h
            vm[t, v, c] -= h
            fp = shade(m0, setup64(vp, cam), colors, pixels)
            fm = shade(m0, setup64(vm, cam), colors, pixels)
            if w is not None:
                fp, fm = fp * w, fm * w
            out[(t, v, c)] = float(np.sum(fp) - np.sum(fm)) / (2 * h)
    return out


MAP_UNIVERSAL, MAP_RECTILINEAR, MAP_PANORAMA, MAP_DOME, MAP_EQUIRECT, MAP_CUBE = range(6)


def make_map_spec(W, H, kind, param=(), dist=(0, 0, 0, 0, 0, 0), aov=0, derivs=False):
    """FP64 map [H, W, 4] of another projection (Sec. 2.2) or of the
    Universal / rectilinear model with Brown-Conrady distortion (Sec. 2.3).
    param: kind-specific (see orc_map_spec); for the Universal kind the
    effective parameters (k, l, s, Omega_deg) after limits.  With
    derivs=True also returns the differences (d_i G, d_j G) [H, W, 6] the
    global delta is formed from (for pstep)."""
    p = np.zeros(4)
    p[:len(param)] = np.asarray(param, dtype=np.float64)
    d = np.zeros(6)
    d[:len(dist)] = np.asarray(dist, dtype=np.float64)
    out = np.zeros((H, W, 4))
    dv = np.zeros((H, W, 6)) if derivs else None
    if _load().orc_map_spec(W, H, kind, _ptr(p), _ptr(d), aov, _ptr(out), _ptr(dv)):
        raise ValueError("orc_map_spec: bad arguments")
    return (out, dv) if derivs else out


def raster_pstep(map_, dmap, rec, pixels=None, nthreads=0, extras=False):
    """Brute-force raster with the per-fragment pixel step: like raster()
    with dmap [H, W, 6] = (d_i G, d_j G) per pixel."""
    H, W = map_.shape[:2]
    m = np.ascontiguousarray(map_, dtype=np.float64)
    dm = np.ascontiguousarray(dmap, dtype=np.float64)
    rec = np.ascontiguousarray(rec, dtype=np.float64)
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64).ravel()
        npix = pix.size
    out = {"id": np.zeros(npix, dtype=np.uint32), "depth": np.zeros(npix), "cov": np.zeros(npix)}
    sm = ni = nf = None
    if extras:
        sm = out["sum_mf"] = np.zeros(npix)
        ni = out["n_inside"] = np.zeros(npix, dtype=np.int32)
        nf = out["n_frag"] = np.zeros(npix, dtype=np.int32)
    n_alg = _load().orc_raster_pstep(W, H, _ptr(m), _ptr(dm), rec.shape[0], _ptr(rec), npix, _ptr(pix),
                                     _ptr(out["id"]), _ptr(out["depth"]), _ptr(out["cov"]), _ptr(sm), _ptr(ni),
                                     _ptr(nf), nthreads)
    if n_alg < 0:
        raise ValueError("orc_raster_pstep: bad sizes")
    out["n_alg"] = int(n_alg)
    if pixels is None:
        for key in list(out):
            if isinstance(out[key], np.ndarray):
                out[key] = out[key].reshape(H, W)
    return out


def map_spec_dirs(fs, ft, W, H, kind, param=(), dist=(0, 0, 0, 0, 0, 0), aov=0):
    """The map function of make_map_spec at texture coordinates (fs, ft):
    (directions [n, 3], valid [n])."""
    fs = np.ascontiguousarray(fs, dtype=np.float64).ravel()
    ft = np.ascontiguousarray(ft, dtype=np.float64).ravel()
    p = np.zeros(4)
    p[:len(param)] = np.asarray(param, dtype=np.float64)
    d = np.zeros(6)
    d[:len(dist)] = np.asarray(dist, dtype=np.float64)
    v = np.zeros((fs.size, 3))
    ok = np.zeros(fs.size, dtype=np.int32)
    _load().orc_map_spec_dirs(fs.size, _ptr(fs), _ptr(ft), W, H, kind, _ptr(p), _ptr(d), aov, _ptr(v), _ptr(ok))
    return v, ok.astype(bool)
