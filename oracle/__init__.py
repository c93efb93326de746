"""FP64 CPU oracle (ctypes wrapper around ``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the library.  It shares no code
with the CUDA path; only the seeded input generator feeds both.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C++ compiler (portable flags only)."""
    src = [os.path.join(_HERE, "oracle.cpp")]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in src + [hdr])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-o", tmp] + src
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _View(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("w", C.c_uint32), ("h", C.c_uint32),
                ("spp", C.c_uint32), ("sample_base", C.c_uint32), ("pixel_base", C.c_uint64)]


class _Params(C.Structure):
    _fields_ = [("max_depth", C.c_uint32), ("seed", C.c_uint64), ("env", C.c_float * 3),
                ("sun_dir", C.c_float * 3), ("sun_E", C.c_float * 3), ("tex_res", C.c_uint32),
                ("tex", C.POINTER(C.c_float)), ("n_lights", C.c_uint32),
                ("lights", C.POINTER(C.c_float))]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u32p, u64p, f32p, f64p = (C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                      C.POINTER(C.c_float), C.POINTER(C.c_double))
            L.ora_philox.argtypes = [u32p, u32p, u32p]
            L.ora_scene_new.restype = C.c_void_p
            L.ora_scene_new.argtypes = [C.c_uint32, C.POINTER(f32p), u32p, C.POINTER(u32p), u32p,
                                        C.c_uint64, f32p, u32p]
            L.ora_scene_free.argtypes = [C.c_void_p]
            L.ora_scene_n_quads.restype = C.c_uint64
            L.ora_scene_n_quads.argtypes = [C.c_void_p]
            L.ora_intersect_quad.restype = C.c_int
            L.ora_intersect_quad.argtypes = [f64p, f64p, C.c_double, C.c_double, f64p, f64p, f64p, f64p]
            L.ora_trace_closest.argtypes = [C.c_void_p, f32p, C.c_uint64, C.c_int, f64p, u32p, u32p,
                                            f64p, f64p, C.c_int]
            L.ora_trace_any.argtypes = [C.c_void_p, f32p, C.c_uint64, C.c_int,
                                        C.POINTER(C.c_uint8), C.c_int]
            L.ora_camera_ray.argtypes = [C.POINTER(_View), C.c_uint32, C.c_uint32, C.c_double,
                                         C.c_double, f64p, f64p]
            L.ora_sample_cosine.argtypes = [f64p, C.c_double, C.c_double, f64p]
            L.ora_render.restype = C.c_int
            L.ora_render.argtypes = [C.c_void_p, C.POINTER(_View), f32p, C.POINTER(_Params),
                                     C.POINTER(C.c_int64), C.c_uint64, f64p, u32p, u32p, u32p,
                                     u32p, f64p, u64p, u64p, C.c_int]
            L.ora_tex_lookup.argtypes = [f32p, C.c_uint32, C.c_uint64, C.c_double, C.c_double, f64p]
            L.ora_light_sample.restype = C.c_int
            L.ora_light_sample.argtypes = [f32p, C.c_uint32, f64p, f64p, f64p, f64p, f64p, f64p]
            L.ora_render_grad.restype = C.c_int
            L.ora_render_grad.argtypes = [C.c_void_p, C.POINTER(_View), f32p, C.POINTER(_Params),
                                          C.POINTER(C.c_int64), C.c_uint64, f64p, f64p, C.c_int]
            _lib = L
    return _lib


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def intersect_quad(o, d, verts, tmin=0.0, tmax=np.inf):
    """Returns (hit, t, u, v) for one ray and one quad (4x3 vertices)."""
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    v = np.ascontiguousarray(verts, dtype=np.float64).reshape(12)
    t, u, w = C.c_double(), C.c_double(), C.c_double()
    hit = lib().ora_intersect_quad(_p(o, C.c_double), _p(d, C.c_double), tmin, tmax,
                                   _p(v, C.c_double), C.byref(t), C.byref(u), C.byref(w))
    return bool(hit), t.value, u.value, w.value


def sample_cosine(n, xi1, xi2) -> np.ndarray:
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros(3)
    lib().ora_sample_cosine(_p(n, C.c_double), float(xi1), float(xi2), _p(out, C.c_double))
    return out


def _view(v) -> _View:
    cv = _View()
    cv.eye[:] = [float(x) for x in v.eye]
    cv.look[:] = [float(x) for x in v.look]
    cv.up[:] = [float(x) for x in v.up]
    cv.vfov_deg = float(v.vfov_deg)
    cv.w, cv.h, cv.spp, cv.pixel_base = int(v.w), int(v.h), int(v.spp), int(v.pixel_base)
    cv.sample_base = int(getattr(v, "sample_base", 0))
    return cv


def _params(p):
    """(ctypes params, arrays to keep alive)."""
    cp = _Params()
    cp.max_depth = int(p.max_depth)
    cp.seed = int(p.seed)
    cp.env[:] = [float(x) for x in p.env]
    cp.sun_dir[:] = [float(x) for x in p.sun_dir]
    cp.sun_E[:] = [float(x) for x in p.sun_E]
    keep = []
    tex = getattr(p, "tex", None)
    if tex is not None:
        t = np.ascontiguousarray(tex, dtype=np.float32)
        keep.append(t)
        cp.tex_res = int(t.shape[1])
        cp.tex = _p(t, C.c_float)
    lights = getattr(p, "lights", None)
    if lights is not None and len(lights):
        lt = np.ascontiguousarray(lights, dtype=np.float32).reshape(-1, 12)
        keep.append(lt)
        cp.n_lights = int(lt.shape[0])
        cp.lights = _p(lt, C.c_float)
    return cp, keep


def tex_lookup(tex, row, u, v) -> np.ndarray:
    t = np.ascontiguousarray(tex, dtype=np.float32)
    out = np.zeros(3)
    lib().ora_tex_lookup(_p(t, C.c_float), int(t.shape[1]), int(row), float(u), float(v),
                         _p(out, C.c_double))
    return out


def light_sample(lights, xi, x, nx):
    """(hit, unit direction, distance, estimator [3]) of one key-light sample."""
    lt = np.ascontiguousarray(lights, dtype=np.float32).reshape(-1, 12)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    nx = np.ascontiguousarray(nx, dtype=np.float64)
    d = np.zeros(3)
    w = np.zeros(3)
    dist = C.c_double()
    ok = lib().ora_light_sample(_p(lt, C.c_float), lt.shape[0], _p(xi, C.c_double), _p(x, C.c_double),
                                _p(nx, C.c_double), _p(d, C.c_double), C.byref(dist), _p(w, C.c_double))
    return bool(ok), d, dist.value, w


def camera_ray(view, x, y, xi1, xi2):
    o = np.zeros(3)
    d = np.zeros(3)
    cv = _view(view)
    lib().ora_camera_ray(C.byref(cv), int(x), int(y), float(xi1), float(xi2),
                         _p(o, C.c_double), _p(d, C.c_double))
    return o, d


class OracleScene:
    """The oracle's own copy of a scene (inputs.Scene), with its own BVHs."""

    def __init__(self, scene):
        L = lib()
        self._keep = []
        nm = len(scene.meshes)
        vps = (C.POINTER(C.c_float) * nm)()
        qps = (C.POINTER(C.c_uint32) * nm)()
        nv = np.zeros(nm, dtype=np.uint32)
        nq = np.zeros(nm, dtype=np.uint32)
        for i, (v, q) in enumerate(scene.meshes):
            v = np.ascontiguousarray(v, dtype=np.float32)
            q = np.ascontiguousarray(q, dtype=np.uint32)
            self._keep += [v, q]
            vps[i] = _p(v, C.c_float)
            qps[i] = _p(q, C.c_uint32)
            nv[i] = v.shape[0]
            nq[i] = q.shape[0]
        xf = np.ascontiguousarray(scene.xforms, dtype=np.float32)
        ids = np.ascontiguousarray(scene.mesh_ids, dtype=np.uint32)
        self._h = L.ora_scene_new(nm, vps, _p(nv, C.c_uint32), qps, _p(nq, C.c_uint32),
                                  xf.shape[0], _p(xf, C.c_float), _p(ids, C.c_uint32))
        self._keep = None
        self.n_quads = int(L.ora_scene_n_quads(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_scene_free(h)
            self._h = None

    def trace_closest(self, rays, mode: int = 0, nthreads: int = 0):
        rays = np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 8)
        n = rays.shape[0]
        t = np.zeros(n)
        inst = np.zeros(n, dtype=np.uint32)
        prim = np.zeros(n, dtype=np.uint32)
        u = np.zeros(n)
        v = np.zeros(n)
        lib().ora_trace_closest(self._h, _p(rays, C.c_float), n, mode, _p(t, C.c_double),
                                _p(inst, C.c_uint32), _p(prim, C.c_uint32), _p(u, C.c_double),
                                _p(v, C.c_double), nthreads)
        return t, inst, prim, u, v

    def trace_any(self, rays, mode: int = 0, nthreads: int = 0):
        rays = np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 8)
        occ = np.zeros(rays.shape[0], dtype=np.uint8)
        lib().ora_trace_any(self._h, _p(rays, C.c_float), rays.shape[0], mode,
                            _p(occ, C.c_uint8), nthreads)
        return occ.astype(bool)

    def render(self, view, albedo, params, pixels=None, log: bool = False, nthreads: int = 0,
               rays: bool = False):
        """Returns dict(rgb=[n_pix,3] f64, escaped, truncated[, inst, prim, shadow][, rays]).
        pixels: frame pixel indices y*w + x (None = the whole frame in order).
        rays=True adds rays [n_paths, max_depth, 13]: per depth the origin and
        direction of the closest-hit ray traced there, the spawn point of its
        hit (origin of its shadow rays) and the direction and distance of the
        key-light shadow ray (zeros where there was none).  params may carry
        tex (float [n_quads, R, R, 3] per-face textures) and lights (float
        [n, 12] key lights)."""
        a = np.ascontiguousarray(albedo, dtype=np.float32).reshape(-1, 3)
        assert a.shape[0] == self.n_quads
        if pixels is None:
            px = None
            n_pix = int(view.w) * int(view.h)
        else:
            px = np.ascontiguousarray(pixels, dtype=np.int64)
            n_pix = px.shape[0]
        rgb = np.zeros((n_pix, 3))
        D = int(params.max_depth)
        n_paths = n_pix * int(view.spp)
        li = lp = ls = ll = lr = None
        if rays:
            lr = np.zeros((n_paths, D, 13))
        if log:
            li = np.zeros((n_paths, D), dtype=np.uint32)
            lp = np.zeros((n_paths, D), dtype=np.uint32)
            ls = np.zeros(n_paths, dtype=np.uint32)
            ll = np.zeros(n_paths, dtype=np.uint32)
        esc = C.c_uint64()
        tr = C.c_uint64()
        cv = _view(view)
        cp, keep = _params(params)
        rc = lib().ora_render(self._h, C.byref(cv), _p(a, C.c_float), C.byref(cp),
                              _p(px, C.c_int64), n_pix, _p(rgb, C.c_double),
                              _p(li, C.c_uint32), _p(lp, C.c_uint32), _p(ls, C.c_uint32),
                              _p(ll, C.c_uint32), _p(lr, C.c_double), C.byref(esc), C.byref(tr),
                              nthreads)
        del keep
        if rc != 0:
            raise ValueError(f"ora_render failed ({rc})")
        out = dict(rgb=rgb, escaped=esc.value, truncated=tr.value)
        if log:
            out.update(inst=li, prim=lp, shadow=ls, light=ll)
        if rays:
            out["rays"] = lr
        return out

    def grad(self, view, albedo, params, dimage, pixels=None, nthreads: int = 0):
        """d/d albedo of sum(dimage * I) -> float64 [n_quads, 3]."""
        a = np.ascontiguousarray(albedo, dtype=np.float32).reshape(-1, 3)
        px = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
        n_pix = int(view.w) * int(view.h) if px is None else px.shape[0]
        dimg = np.ascontiguousarray(dimage, dtype=np.float64).reshape(n_pix, 3)
        g = np.zeros((self.n_quads, 3))
        cv = _view(view)
        cp, keep = _params(params)
        rc = lib().ora_render_grad(self._h, C.byref(cv), _p(a, C.c_float), C.byref(cp),
                                   _p(px, C.c_int64), n_pix, _p(dimg, C.c_double),
                                   _p(g, C.c_double), nthreads)
        del keep
        if rc != 0:
            raise ValueError(f"ora_render_grad failed ({rc})")
        return g
