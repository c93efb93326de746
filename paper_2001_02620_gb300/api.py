"""Python front end of the qrt C ABI.  PyTorch supplies device memory and
streams; every step of the path runs in libqrt.so's kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N
from .inputs import Params, View


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def make_tuning(tuning: dict | None) -> N.qrt_tuning:
    t = N.qrt_tuning()
    for k, v in (tuning or {}).items():
        setattr(t, k, int(v))
    return t


def make_params(p: Params, tuning: dict | None = None, path_log: torch.Tensor | None = None,
                max_steps: int = 0, stage_times: bool = False,
                ray_log: torch.Tensor | None = None) -> N.qrt_params:
    cp = N.qrt_params()
    cp.max_depth = int(p.max_depth)
    cp.flags = N.QRT_FLAG_STAGE_TIMES if stage_times else 0
    cp.seed = int(p.seed)
    cp.env[:] = [float(x) for x in p.env]
    cp.sun_dir[:] = [float(x) for x in p.sun_dir]
    cp.sun_E[:] = [float(x) for x in p.sun_E]
    cp.max_steps = int(max_steps)
    cp.d_path_log = _ptr(path_log)
    cp.d_ray_log = _ptr(ray_log)
    cp.tuning = make_tuning(tuning)
    tex = getattr(p, "tex", None)
    if tex is not None:
        if not (isinstance(tex, torch.Tensor) and tex.is_cuda and tex.dtype == torch.float32
                and tex.is_contiguous() and tex.dim() == 4):
            raise TypeError("Params.tex must be a contiguous float32 CUDA tensor [n_quads, R, R, 3]")
        cp.d_tex = _ptr(tex)
        cp.tex_res = int(tex.shape[1])
    lights = getattr(p, "lights", None)
    if lights is not None and len(lights):
        lt = np.ascontiguousarray(lights, dtype=np.float32).reshape(-1, 12)
        cp.n_lights = int(lt.shape[0])
        cp.lights = lt.ctypes.data_as(C.POINTER(C.c_float))
        cp._keep = lt   # the library copies the lights during the call
    return cp


def make_views(views, outs) -> C.Array:
    arr = (N.qrt_view * len(views))()
    for k, (v, o) in enumerate(zip(views, outs)):
        cv = arr[k]
        cv.eye[:] = [float(x) for x in v.eye]
        cv.look[:] = [float(x) for x in v.look]
        cv.up[:] = [float(x) for x in v.up]
        cv.vfov_deg = float(v.vfov_deg)
        cv.w, cv.h, cv.spp = int(v.w), int(v.h), int(v.spp)
        cv.pixel_base = int(v.pixel_base)
        cv.sample_base = int(getattr(v, "sample_base", 0))
        cv.out_rgb = _ptr(o)
        cv.crop_x, cv.crop_y = int(getattr(v, "crop_x", 0)), int(getattr(v, "crop_y", 0))
        cv.crop_w, cv.crop_h = int(getattr(v, "crop_w", 0)), int(getattr(v, "crop_h", 0))
    return arr


def region(v) -> tuple:
    """(width, height) of the pixels a view renders: its crop, or the frame."""
    cw, ch = int(getattr(v, "crop_w", 0)), int(getattr(v, "crop_h", 0))
    return (int(v.w), int(v.h)) if cw == 0 and ch == 0 else (cw, ch)


def n_paths(views) -> int:
    return sum(region(v)[0] * region(v)[1] * int(v.spp) for v in views)


def path_log_words(views, max_depth: int) -> int:
    """Words of a path log: per path (inst, prim) per depth, sun and key-light shadow bits."""
    return n_paths(views) * (2 * int(max_depth) + 2)


# per path and depth: closest-hit ray (8), spawn point (3) and one unused,
# key-light shadow direction and distance (4)
RAY_LOG_FLOATS = 16


def ray_log_floats(views, max_depth: int) -> int:
    return n_paths(views) * int(max_depth) * RAY_LOG_FLOATS


class Scene:
    """A scene uploaded to the current CUDA device (owns its device memory)."""

    def __init__(self, scene, build_opts: dict | None = None):
        L = N.lib()
        meshes = scene.meshes
        self._host = []
        arr = (N.qrt_mesh * len(meshes))()
        for k, (v, q) in enumerate(meshes):
            v = np.ascontiguousarray(v, dtype=np.float32)
            q = np.ascontiguousarray(q, dtype=np.uint32)
            self._host += [v, q]
            arr[k].verts = v.ctypes.data_as(C.POINTER(C.c_float))
            arr[k].n_verts = v.shape[0]
            arr[k].quads = q.ctypes.data_as(C.POINTER(C.c_uint32))
            arr[k].n_quads = q.shape[0]
        xf = np.ascontiguousarray(scene.xforms, dtype=np.float32).reshape(-1)
        ids = np.ascontiguousarray(scene.mesh_ids, dtype=np.uint32)
        opts = None
        if build_opts:
            opts = N.qrt_build_opts()
            for k, v in build_opts.items():
                setattr(opts, k, int(v))
        h = C.c_void_p()
        N.check(L.qrt_scene_create(arr, len(meshes), xf.ctypes.data_as(C.POINTER(C.c_float)),
                                   ids.ctypes.data_as(C.POINTER(C.c_uint32)), ids.shape[0],
                                   C.byref(opts) if opts is not None else None, C.byref(h)))
        self._host = None
        self.handle = h
        st = N.qrt_scene_stats()
        N.check(L.qrt_scene_stats_get(h, C.byref(st)))
        self.stats = {f: getattr(st, f) for f, _ in N.qrt_scene_stats._fields_}
        self.stats["phase_seconds"] = list(st.phase_seconds)
        self.n_quads = int(st.n_quads)
        self.n_instances = int(st.n_instances)

    def close(self):
        if getattr(self, "handle", None):
            N.lib().qrt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ray queries ---------------------------------------------------------
    def trace_closest(self, rays: torch.Tensor, hits: torch.Tensor | None = None,
                      tuning: dict | None = None, stream=None) -> torch.Tensor:
        """rays: float32 [n, 8] on the GPU -> hits int32 [n, 4] (t bits, inst, prim, uv)."""
        n = rays.shape[0]
        if hits is None:
            hits = torch.empty((n, 4), dtype=torch.int32, device=rays.device)
        t = make_tuning(tuning)
        N.check(N.lib().qrt_trace_closest(self.handle, _ptr(rays), n, _ptr(hits), C.byref(t),
                                          _stream(stream)))
        return hits

    def trace_any(self, rays: torch.Tensor, bits: torch.Tensor | None = None,
                  tuning: dict | None = None, stream=None) -> torch.Tensor:
        """rays: float32 [n, 8] -> int32 [ceil(n/32)] occlusion bit words."""
        n = rays.shape[0]
        if bits is None:
            bits = torch.empty(((n + 31) // 32,), dtype=torch.int32, device=rays.device)
        t = make_tuning(tuning)
        N.check(N.lib().qrt_trace_any(self.handle, _ptr(rays), n, _ptr(bits), C.byref(t),
                                      _stream(stream)))
        return bits

    def trace_stats(self, rays: torch.Tensor, any_hit: bool, out: torch.Tensor,
                    stats: torch.Tensor, tuning: dict | None = None, stream=None):
        t = make_tuning(tuning)
        N.check(N.lib().qrt_trace_stats(self.handle, 1 if any_hit else 0, _ptr(rays), rays.shape[0],
                                        _ptr(out), C.byref(t), _ptr(stats), _stream(stream)))

    # -- rendering -----------------------------------------------------------
    def render(self, views, albedo: torch.Tensor, params: Params, outs=None,
               tuning: dict | None = None, path_log: torch.Tensor | None = None,
               max_steps: int = 0, stats: torch.Tensor | None = None, stream=None,
               stage_times: bool = False, ray_log: torch.Tensor | None = None):
        """Renders views (list of inputs.View) into float32 [rh, rw, 3] tensors
        (rw x rh: the view's crop, or its whole frame)."""
        if isinstance(views, View):
            views = [views]
        if outs is None:
            outs = [torch.empty((region(v)[1], region(v)[0], 3), dtype=torch.float32,
                                device=albedo.device) for v in views]
        cv = make_views(views, outs)
        cp = make_params(params, tuning, path_log, max_steps, stage_times, ray_log)
        L = N.lib()
        if stats is None:
            N.check(L.qrt_render_spp(self.handle, cv, len(views), _ptr(albedo), C.byref(cp),
                                     _stream(stream)))
        else:
            N.check(L.qrt_render_spp_stats(self.handle, cv, len(views), _ptr(albedo), C.byref(cp),
                                           _ptr(stats), _stream(stream)))
        return outs

    def cost_maps(self, views, albedo: torch.Tensor, params: Params, stats: torch.Tensor,
                  outs=None, tuning: dict | None = None, stream=None):
        """Renders views and returns float [h, w] maps of the mean inner BVH
        nodes visited per sample (qrt_render_cost); traversal counters are
        added into stats (int64 [12])."""
        if isinstance(views, View):
            views = [views]
        if outs is None:
            outs = [torch.empty((region(v)[1], region(v)[0], 3), dtype=torch.float32,
                                device=albedo.device) for v in views]
        costs = [torch.empty((region(v)[1], region(v)[0]), dtype=torch.float32, device=albedo.device)
                 for v in views]
        cv = make_views(views, outs)
        cp = make_params(params, tuning)
        cptr = (C.c_void_p * len(views))(*[_ptr(c) for c in costs])
        N.check(N.lib().qrt_render_cost(self.handle, cv, len(views), _ptr(albedo), C.byref(cp), cptr,
                                        _ptr(stats), _stream(stream)))
        return costs

    def adjoint(self, views, albedo: torch.Tensor, dimages, grad: torch.Tensor, params: Params,
                tuning: dict | None = None, stream=None) -> torch.Tensor:
        """Adds the albedo gradient of sum(dimage * image) into grad [n_quads, 3]."""
        if isinstance(views, View):
            views = [views]
        cv = make_views(views, [None] * len(views))
        cp = make_params(params, tuning)
        dptr = (C.c_void_p * len(views))(*[_ptr(d) for d in dimages])
        N.check(N.lib().qrt_render_adjoint(self.handle, cv, len(views), _ptr(albedo), dptr,
                                           _ptr(grad), C.byref(cp), _stream(stream)))
        return grad

    def stage_times(self, reset: bool = True, stream=None) -> dict:
        """{stage: (total ms, launches)} of renders made with stage_times=True."""
        ms = (C.c_double * 5)()
        n = (C.c_uint32 * 5)()
        N.check(N.lib().qrt_stage_times(self.handle, _stream(stream), ms, n, 1 if reset else 0))
        return {name: (ms[k], n[k]) for k, name in enumerate(N.STAGES)}

    def check(self, stream=None) -> None:
        """Raises QrtError if a kernel flagged a stack overflow or step limit."""
        N.check(N.lib().qrt_check(self.handle, _stream(stream)))


class RenderGraph:
    """One render of fixed views captured as a CUDA graph; launch() replays it."""

    def __init__(self, scene: Scene, views, albedo: torch.Tensor, params: Params, outs=None,
                 tuning: dict | None = None):
        if isinstance(views, View):
            views = [views]
        if outs is None:
            outs = [torch.empty((region(v)[1], region(v)[0], 3), dtype=torch.float32,
                                device=albedo.device) for v in views]
        self.outs = outs
        self._keep = (scene, albedo)
        cv = make_views(views, outs)
        cp = make_params(params, tuning)
        h = C.c_void_p()
        N.check(N.lib().qrt_render_graph_create(scene.handle, cv, len(views), _ptr(albedo),
                                                C.byref(cp), C.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        N.check(N.lib().qrt_graph_launch(self.handle, _stream(stream)))
        return self.outs

    def close(self):
        if getattr(self, "handle", None):
            N.lib().qrt_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def read_bandwidth_gbs(nbytes: int, reps: int, stream=None) -> float:
    """GB/s of repeated L2-only reads over a fresh device buffer of nbytes
    (qrt_read_bandwidth, timed with CUDA events on the stream).  With nbytes
    well inside L2 this is the L2 read bandwidth."""
    buf = torch.zeros(nbytes // 4, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream() if stream is None else stream
    L = N.lib()
    N.check(L.qrt_read_bandwidth(_ptr(buf), buf.numel() * 4, 2, _ptr(sink), _stream(s)))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    N.check(L.qrt_read_bandwidth(_ptr(buf), buf.numel() * 4, reps, _ptr(sink), _stream(s)))
    e1.record(s)
    e1.synchronize()
    return buf.numel() * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9


def save_heat_map(cost: torch.Tensor, path: str, scale: float | None = None) -> float:
    """Writes a cost map (float [h, w], e.g. from Scene.cost_maps) as a binary
    PPM heat map, dark (cheap) -> red -> yellow -> white (expensive), the
    way the paper shows per-pixel cost.  scale: the cost drawn white
    (default: the 99th percentile).  Returns the scale used."""
    import numpy as np
    c = cost.detach().float().cpu().numpy()
    if scale is None:
        scale = float(np.percentile(c, 99.0)) or 1.0
    x = np.clip(c / scale, 0.0, 1.0)
    rgb = np.stack([np.clip(3 * x, 0, 1), np.clip(3 * x - 1, 0, 1), np.clip(3 * x - 2, 0, 1)], -1)
    img = (rgb * 255.0 + 0.5).astype(np.uint8)
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())
    return scale


def accumulate(frame_sum: torch.Tensor, frame: torch.Tensor, frames: int,
               mean: torch.Tensor | None = None, stream=None) -> torch.Tensor | None:
    """Progressive accumulation (qrt_accumulate): frame_sum += frame, and
    mean = frame_sum / frames when given (frames = frames summed so far)."""
    N.check(N.lib().qrt_accumulate(_ptr(frame_sum), _ptr(frame), _ptr(mean), frame.numel(),
                                   int(frames), _stream(stream)))
    return mean


def l2_loss(img: torch.Tensor, target: torch.Tensor, dimage: torch.Tensor | None = None,
            stream=None):
    """Mean squared error (FP64 scalar tensor) and, if given, its gradient into dimage."""
    loss = torch.empty((), dtype=torch.float64, device=img.device)
    N.check(N.lib().qrt_l2_loss(_ptr(img), _ptr(target), img.numel(), _ptr(loss), _ptr(dimage),
                                _stream(stream)))
    return loss


class RenderFn(torch.autograd.Function):
    """image = render(albedo); backward runs the path-replay adjoint kernel."""

    @staticmethod
    def forward(ctx, albedo: torch.Tensor, scene: Scene, view: View, params: Params,
                tuning: dict | None = None):
        albedo = albedo.contiguous()
        (img,) = scene.render([view], albedo, params, tuning=tuning)
        ctx.scene, ctx.view, ctx.params, ctx.tuning = scene, view, params, tuning
        ctx.save_for_backward(albedo)
        return img

    @staticmethod
    def backward(ctx, grad_img: torch.Tensor):
        (albedo,) = ctx.saved_tensors
        grad = torch.zeros_like(albedo)
        ctx.scene.adjoint([ctx.view], albedo, [grad_img.contiguous()], grad, ctx.params,
                          tuning=ctx.tuning)
        return grad, None, None, None, None


def render_differentiable(albedo, scene, view, params, tuning=None):
    return RenderFn.apply(albedo, scene, view, params, tuning)
