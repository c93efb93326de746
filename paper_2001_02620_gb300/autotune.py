"""Autotuner for the launch parameters of the renderer.

Searches node-fetch width, block size, the trace kernels' register budget
(resident warps per SM), the rays a lane claims per fetch (`batch`) and the
traversal stack depth, by timing renders of a proxy view (the target view at
reduced resolution, same spp and depth), and keeps the fastest
configuration that raised no device error.

The stack depth is searched only among depths that provably suffice for the
scene: a four-wide node pushes at most three entries before the traversal
descends, and a ray's stack holds the pending entries of the nodes on one
root-to-leaf path through the TLAS and one BLAS, so 3 * (TLAS depth + deepest
BLAS depth) entries always suffice (depths in wide-node levels, from
qrt_scene_stats).  A depth that merely sufficed on the proxy view could
overflow on another view, and an overflow changes results.  Where no
candidate below the library's 64 entries is proven, 64 is kept (overflows
there are still detected and reported by qrt_check).  The stack's place is
not searched: the per-thread stack in local memory (cached in L1) beat a
stack whose bottom 4-16 entries sit in shared memory in every measured
configuration, and the shared-memory branch cost 9 % even when switched off.

Results are cached as JSON keyed by (GPU name, SM count, scene class), so
later runs skip the search.  None of the parameters changes a rendered
value: images are bit-identical under every candidate.
"""
from __future__ import annotations

import dataclasses
import itertools
import json
import os
import time

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                             "autotune_cache", "qrt_tuning.json")

SPACE = {
    "block": [64, 128, 256],
    "fetch": [16, 32],
    "occupancy": [24, 32, 40, 48],
    "batch": [1, 2, 4, 8],
}
STACK_DEPTHS = (32, 64)   # the library's choices; 64 is its maximum


def proven_stack_depths(tlas_depth: int, max_blas_depth: int) -> list[int]:
    """Stack depths that cannot overflow on a scene with these BVH depths
    (at most three pending entries per wide-node level of one TLAS path and
    one BLAS path); the library maximum when none is proven."""
    need = 3 * (int(tlas_depth) + int(max_blas_depth))
    ok = [d for d in STACK_DEPTHS if d >= need]
    return ok or [max(STACK_DEPTHS)]


def candidates(space: dict | None = None) -> list[dict]:
    space = space or SPACE
    keys = sorted(space)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(space[k] for k in keys))]


def scene_class(scene) -> str:
    """Coarse key: scene name plus order of magnitude of quads and instances."""
    import math
    q = max(1, int(scene.n_quads))
    i = max(1, int(getattr(scene, "n_instances", None) or len(scene.xforms)))
    name = getattr(scene, "name", "") or "scene"
    return f"{name}:q1e{int(math.log10(q))}:i1e{int(math.log10(i))}"


def cache_key(gpu_name: str, sm_count: int, scene_cls: str, kind: str = "render") -> str:
    return f"{gpu_name}|{sm_count}|{scene_cls}|{kind}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(entry_key: str, value: dict, path: str = DEFAULT_CACHE) -> None:
    d = load_cache(path)
    d[entry_key] = value
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick_best(timings: dict) -> tuple[str, float]:
    """timings: candidate-json -> seconds (None = failed).  Returns the fastest."""
    ok = {k: v for k, v in timings.items() if v is not None}
    if not ok:
        raise RuntimeError("no tuning candidate ran without error")
    k = min(ok, key=lambda c: (ok[c], c))
    return k, ok[k]


def proxy_view(view, max_paths: int = 1 << 22):
    """The view scaled down (same aspect and spp) to at most max_paths paths.
    The proxy must still fill the GPU several times over: with a small one
    the launch tail dominates and the tuner prefers the wrong occupancy."""
    paths = view.w * view.h * view.spp
    s = min(1.0, (max_paths / paths) ** 0.5)
    return dataclasses.replace(view, w=max(32, int(view.w * s)), h=max(32, int(view.h * s)))


def _time_render(scene, view, albedo, params, out, cand, reps: int) -> float:
    """Best of `reps` timed renders (after one untimed) with CUDA events."""
    import torch
    scene.render([view], albedo, params, outs=[out], tuning=cand)
    scene.check()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        scene.render([view], albedo, params, outs=[out], tuning=cand)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    scene.check()
    return min(ts)


def tune(scene, view, albedo, params, space: dict | None = None, reps: int = 3,
         cache_path: str | None = DEFAULT_CACHE, scene_name: str | None = None,
         force: bool = False, log=None, finalists: int = 4, proxy_paths: int = 1 << 22) -> dict:
    """Returns the best tuning dict for rendering `view` of `scene` (api.Scene).

    Every candidate is timed on a proxy view of at most proxy_paths paths; when the
    view is larger, the `finalists` fastest are timed again on the view
    itself and the fastest there wins.  (A proxy renders from a warm L2 and
    a smaller working set: on a scene of tens of GB the full frame preferred
    40 resident warps per SM, 2.6 % faster, where the proxy chose 32.)"""
    import torch

    from . import _native as N
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    cls = scene_class(type("S", (), {"n_quads": scene.n_quads, "n_instances": scene.n_instances,
                                     "name": scene_name or ""})())
    key = cache_key(props.name, props.multi_processor_count, cls)
    if cache_path and not force:
        hit = load_cache(cache_path).get(key)
        if hit:
            return hit["tuning"]
    pv = proxy_view(view, proxy_paths)
    out = torch.empty((pv.h, pv.w, 3), device=albedo.device)
    timings = {}
    space = dict(space or SPACE)
    if "stack" not in space:
        space["stack"] = proven_stack_depths(scene.stats["tlas_depth"], scene.stats["max_blas_depth"])
    for cand in candidates(space):
        ck = json.dumps(cand, sort_keys=True)
        try:
            timings[ck] = _time_render(scene, pv, albedo, params, out, cand, reps)
        except N.QrtError:
            timings[ck] = None
        if log:
            log(f"tune {ck}: {timings[ck]}")
    best, t = pick_best(timings)
    final = {}
    if finalists > 1 and (pv.w, pv.h) != (view.w, view.h):
        ranked = sorted((v, k) for k, v in timings.items() if v is not None)[:finalists]
        full = torch.empty((view.h, view.w, 3), device=albedo.device)
        for _, ck in ranked:
            try:
                final[ck] = _time_render(scene, view, albedo, params, full, json.loads(ck), 2)
            except N.QrtError:
                final[ck] = None
            if log:
                log(f"tune (whole view) {ck}: {final[ck]}")
        del full
        best, t = pick_best(final)
    result = json.loads(best)
    if cache_path:
        store_cache(key, {"tuning": result, "seconds": t, "proxy": [pv.w, pv.h, pv.spp],
                          "whole_view_finalists": final,
                          "when": time.strftime("%Y-%m-%dT%H:%M:%S")}, cache_path)
    return result
