"""Benchmark of the instanced-quad path tracer on one GB300 (or N replicas).

A step is one qrt_render_spp of the Moana-scale workload: 5000 prototypes
(261.1 M unique quads) instanced 39.3 M times (82.4 G instanced quads, the
Moana Island statistics of Section 1), 1920x1080, 16 spp, path depth 8,
environment + sun with shadow rays.  value = all rays traced per second
(closest-hit + shadow), the accounting of the paper's Mray/s (Section 6,
"Results").  The mid workload (5.73 M unique quads, 100 k instances,
1024x1024, 4 spp, depth 5) is measured in the same run as a sub-measurement
(key "mid"), with the batched-views and adjoint workloads that are defined
on it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload moana|mid] [--moana-scale S]
Under torchrun each rank renders its own frame (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s closest-hit & path samples/s, batched vs plain launch; adjoint/primal"
# per kernel kind (closest-hit, then shadow): rays, nodes, quads, instance
# entries, fp64 re-tests, shaded vertices
STAT_WORDS = 12
# the closest-hit kernel's code and the scene build that shapes its traffic
KERNEL_SOURCES = ["paper_2001_02620_gb300/csrc/traverse.cuh", "paper_2001_02620_gb300/csrc/wavefront.cu",
                  "paper_2001_02620_gb300/csrc/qrt_layout.h", "paper_2001_02620_gb300/csrc/shading.cuh",
                  "paper_2001_02620_gb300/csrc/bvh_build.cpp", "paper_2001_02620_gb300/csrc/bvh_build.h",
                  "paper_2001_02620_gb300/csrc/capi.cpp"]


def kernel_source_hash() -> str:
    """Hash of the code in KERNEL_SOURCES with comments and layout removed, so
    that an edit of comments alone does not retire a measurement."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, tuning=None):
    """DRAM bytes per launch of the closest-hit trace kernel as recorded from
    a committed ncu capture (not measured in this run), if that capture was
    taken on the current kernel sources and with this run's launch
    parameters (tuning None = the library defaults, which the record's
    "launch" entry lists): (bytes, kernel, source note)."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None, None, None
    e = d.get(workload)
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None, None, None
    launch = e.get("launch", {})
    if tuning and any(tuning.get(k, v) != v for k, v in launch.items()):
        return None, None, None
    return (float(e["dram_bytes_per_launch"]), e.get("kernel"),
            "recorded, not measured in this run: " + e.get("source", "profiles/roofline_traffic.json"))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"qrt_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def mid_workload():
    from paper_2001_02620_gb300 import inputs as I
    sc = I.mid_scene()
    return sc, I.mid_view(), I.mid_params(), I.albedo(sc.n_quads)


def moana_workload(scale: float):
    from paper_2001_02620_gb300 import inputs as I
    sc = I.moana_scene(scale)
    return sc, I.moana_view(sc.meta["extent"]), I.moana_params(), I.albedo(sc.n_quads)


WORKLOADS = {
    "mid": "mid: 64 prototypes (log-uniform 2^12..2^16 quads) + 2048^2-quad terrain = 5.73M "
           "unique quads, 100k instances, 1024x1024, 4 spp, depth 5, env + sun shadow rays",
    "moana": "moana-scale: 5000 prototypes (1000 Zipf 8M..~20k quads + 4000 of 16..512) + "
             "2048^2 terrain = 261.1M unique quads, 39.3M clustered instances (82.4G instanced "
             "quads), 1920x1080, 16 spp, depth 8, env + sun shadow rays",
}
# what stands between timed steps and the L2 (the same words on both arms)
L2_NOTE = {
    "mid": "no flush: scene (0.4 GB) and per-path state (0.7 GB) exceed the 129 MB L2",
    "moana": "no flush: scene (25 GB) and per-path state (5.5 GB) exceed the 129 MB L2",
}


def workload_config(workload: str, scale: float) -> dict:
    """The config dict both arms print (identical for the same workload)."""
    w = WORKLOADS[workload]
    if workload == "moana" and scale != 1.0:
        w += f" x {scale}"
    return {"workload": w, "l2": L2_NOTE[workload]}


def load_workload(workload: str, scale: float):
    return moana_workload(scale) if workload == "moana" else mid_workload()


def oracle_sample(osc, view, params, alb, budget_s: float, frame: str, seed: int = 99,
                  build_s: float | None = None):
    """Times the FP64 oracle (all host cores) on a bounded random pixel sample
    of the workload's frame: batches of 256, 512, ... pixels (all spp) until
    budget_s seconds of oracle time are spent."""
    rng = np.random.default_rng(seed)
    npix = view.w * view.h
    n = 256
    rays = 0
    elapsed = 0.0
    done = 0
    while elapsed < budget_s and done < npix:
        px = np.sort(rng.choice(npix, size=min(n, npix), replace=False))
        t = time.time()
        r = osc.render(view, alb, params, pixels=px, log=True)
        dt = time.time() - t
        hits = int((r["inst"] != 0xFFFFFFFF).sum())
        sh = r["shadow"]
        shadow = sum(int(((sh >> (2 * i)) & 1).sum()) for i in range(min(16, params.max_depth)))
        rays += hits + int(r["escaped"]) + shadow
        elapsed += dt
        done += len(px)
        n *= 2
    cores = os.cpu_count() or 1
    extra = f", oracle BVH build {build_s:.1f} s excluded" if build_s is not None else ""
    return {"value": rays / elapsed / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} random pixels x {view.spp} spp of the {frame} frame "
                      f"({rays} rays, {elapsed:.1f} s FP64{extra})",
            "paths_per_s": done * view.spp / elapsed}


def _time(fn, reps: int, warm: int = 2) -> float:
    """Median seconds of fn() measured with CUDA events on the current stream."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    return float(np.median(ts))


def dumped_rays(api, scene, view, d_alb, params, n: int, tuning=None):
    """Ray sets dumped from a render of the workload's camera through the ray
    log (enough samples per pixel for n camera rays): 'primary' = the camera
    rays, 'diffuse' = the rays leaving the first hit (depth 2), 'shadow' =
    the shadow rays toward the sun; each float32 [<= n, 8] on the device, in
    the order the renderer traces them."""
    import dataclasses
    import torch
    spp = max(1, -(-n // (view.w * view.h)))
    v = dataclasses.replace(view, spp=spp)
    D = params.max_depth
    rlog = torch.zeros(api.ray_log_floats([v], D), dtype=torch.float32, device=d_alb.device)
    scene.render([v], d_alb, params, ray_log=rlog, tuning=tuning)
    scene.check()
    r = rlog.view(-1, D, api.RAY_LOG_FLOATS)
    out = {}
    for name, k in (("primary", 0), ("diffuse", 1)):
        rk = r[:, k, 0:8]
        out[name] = rk[rk[:, 7] != 0][:n].contiguous()
    so = r[:, :, 8:11].reshape(-1, 3)   # spawn points of the hits: the shadow rays' origins
    so = so[(so != 0).any(1)][:n]
    sun = torch.tensor(params.sun_dir, dtype=torch.float64)
    sh = torch.zeros((so.shape[0], 8), dtype=torch.float32, device=so.device)
    sh[:, 0:3] = so
    sh[:, 4:7] = (sun / sun.norm()).float().to(so.device)
    sh[:, 7] = float("inf")
    out["shadow"] = sh
    del rlog, r
    return out


def bench_trace(api, scene, view, d_alb, params, dev, tuning=None, n=1 << 22):
    """trace_closest / trace_any throughput on ray sets dumped from a render
    of the workload's view: camera rays, first diffuse bounces, shadow rays.
    The query kernels return each hit's (u, v), which the render's
    closest-hit kernel drops, so they carry more state: each query is timed
    with the render's register budget and with 32 warps/SM, the faster
    reported (both budgets give the same hits)."""
    import torch
    out = {}
    base = dict(tuning or {})
    budgets = sorted({base.get("occupancy", 40), 32})
    for name, d in dumped_rays(api, scene, view, d_alb, params, n, tuning).items():
        m = d.shape[0]
        hits = torch.empty((m, 4), dtype=torch.int32, device=dev)
        bits = torch.empty(((m + 31) // 32,), dtype=torch.int32, device=dev)
        tc = ta = None
        for occ in budgets:
            t = dict(base, occupancy=occ)
            c = _time(lambda: scene.trace_closest(d, hits, tuning=t), 5)
            a = _time(lambda: scene.trace_any(d, bits, tuning=t), 5)
            if tc is None or c < tc[0]:
                tc = (c, occ)
            if ta is None or a < ta[0]:
                ta = (a, occ)
        st = torch.zeros(6, dtype=torch.int64, device=dev)
        scene.trace_stats(d, False, hits, st)
        s = st.cpu().numpy()
        out[name] = {"rays": m, "closest_mrays_s": m / tc[0] / 1e6, "any_mrays_s": m / ta[0] / 1e6,
                     "closest_warps_per_sm": tc[1], "any_warps_per_sm": ta[1],
                     "hit_rate": float((hits[:, 1] != -1).float().mean().item()),
                     "nodes_per_ray": float(s[1]) / m, "quads_per_ray": float(s[2]) / m,
                     "instances_per_ray": float(s[3]) / m}
    scene.check()
    out["source"] = ("rays dumped from a render of the workload's view (qrt_params.d_ray_log), "
                     "in the order the renderer traces them")
    return out


def bench_batched(api, scene, d_alb, dev, tuning=None, views=None):
    """Uneven views of the mid scene (default: the 32 views of the batched
    workload): one graph-captured launch sequence over all views versus one
    plain launch sequence per view on one stream; images must be
    bit-identical."""
    import torch
    from paper_2001_02620_gb300 import inputs as I
    views = views or I.batched_views()
    params = I.mid_params()
    paths = sum(v.w * v.h * v.spp for v in views)
    outs_b = [torch.empty((v.h, v.w, 3), device=dev) for v in views]
    outs_p = [torch.empty((v.h, v.w, 3), device=dev) for v in views]
    graph = api.RenderGraph(scene, views, d_alb, params, outs=outs_b, tuning=tuning)

    def plain():
        for v, o in zip(views, outs_p):
            scene.render([v], d_alb, params, outs=[o], tuning=tuning)

    tb = _time(graph.launch, 3, warm=1)
    tp = _time(plain, 3, warm=1)
    scene.check()
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_p))
    return {"views": len(views), "paths": paths, "batched_paths_per_s": paths / tb,
            "plain_paths_per_s": paths / tp, "speedup": tp / tb, "bit_identical": same,
            "batched_ms": tb * 1e3, "plain_ms": tp * 1e3}


def bench_progressive(api, scene, view, d_alb, params, dev, tuning=None, warm=64, frames=64):
    """Progressive rendering as the paper runs it (Section 5.4: one sample
    per pixel per frame, accumulated; Section 6: 64 warm-up frames, then 64
    measured): each frame renders spp = 1 at sample_base = frame number and
    adds into a device sum (qrt_accumulate), which also writes the mean."""
    import dataclasses
    import torch
    img = torch.empty((view.h, view.w, 3), device=dev)
    acc = torch.zeros_like(img)
    mean = torch.empty_like(img)

    def frame(f):
        fv = dataclasses.replace(view, spp=1, sample_base=f)
        scene.render([fv], d_alb, params, outs=[img], tuning=tuning)
        api.accumulate(acc, img, f + 1, mean)

    for f in range(warm):
        frame(f)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for f in range(warm, warm + frames):
        frame(f)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / frames
    # rays of the measured frames: one counting render of the same samples
    stats = torch.zeros(12, dtype=torch.int64, device=dev)
    scene.render([dataclasses.replace(view, spp=frames, sample_base=warm)], d_alb, params,
                 outs=[torch.empty_like(img)], stats=stats, tuning=tuning)
    st = stats.cpu().numpy()
    rays = int(st[0] + st[6]) / frames
    scene.check()
    return {"frames": frames, "warmup_frames": warm, "spp_per_frame": 1,
            "resolution": [view.w, view.h], "ms_per_frame": ms, "fps": 1e3 / ms,
            "rays_per_frame": rays, "mrays_s": rays / (ms * 1e-3) / 1e6}


def bench_cost_map(api, scene, view, d_alb, params, dev, tuning=None):
    """Per-pixel traversal cost of the frame (the paper's cost heat map):
    mean inner BVH nodes visited per sample, summarised."""
    import torch
    stats = torch.zeros(12, dtype=torch.int64, device=dev)
    (cost,) = scene.cost_maps([view], d_alb, params, stats, tuning=tuning)
    c = cost.flatten().double()
    q = torch.quantile(c[torch.randperm(c.numel(), device=c.device)[:1 << 20]],
                       torch.tensor([0.5, 0.9, 0.99], dtype=torch.float64, device=c.device))
    return {"unit": "inner BVH nodes visited per path sample (closest-hit and shadow rays)",
            "mean": float(c.mean()), "p50": float(q[0]), "p90": float(q[1]), "p99": float(q[2]),
            "max": float(c.max()), "pixels": int(c.numel())}


def bench_device_build(api, scene, sc, view, d_alb, params, dev, tuning=None, rays=0):
    """The same scene with its TLAS, then also its BLASes, built on the device
    (linear BVHs over Morton order) instead of the host's binned SAH: build
    times, render throughput, and how many pixels differ from the SAH scene's
    image."""
    import torch
    ref = torch.empty((view.h, view.w, 3), device=dev)
    out = torch.empty_like(ref)
    t_sah = _time(lambda: scene.render([view], d_alb, params, outs=[ref], tuning=tuning), 5)
    res = {"sah": {"blas_build_s": scene.stats["phase_seconds"][0],
                   "tlas_build_s": scene.stats["phase_seconds"][3],
                   "tlas_depth": scene.stats["tlas_depth"], "max_blas_depth": scene.stats["max_blas_depth"],
                   "mrays_s": rays / t_sah / 1e6},
           "note": "build seconds cover the build and the host invariant check of that level"}
    for name, opts in (("device_tlas", dict(tlas_builder=1)),
                       ("device_blas_and_tlas", dict(tlas_builder=1, blas_builder=1))):
        t0 = time.time()
        s2 = api.Scene(sc, build_opts=opts)
        build_s = time.time() - t0
        t_dev = _time(lambda: s2.render([view], d_alb, params, outs=[out], tuning=tuning), 5)
        s2.check()
        ph = s2.stats["phase_seconds"]
        res[name] = {"blas_build_s": ph[0] + ph[1], "tlas_build_s": ph[3], "scene_build_s": build_s,
                     "tlas_depth": s2.stats["tlas_depth"], "max_blas_depth": s2.stats["max_blas_depth"],
                     "mrays_s": rays / t_dev / 1e6,
                     "pixels_differing": float((out != ref).any(dim=-1).float().mean().item())}
        s2.close()
        del s2
    res["sah"]["blas_build_s"] += scene.stats["phase_seconds"][1]
    return res


def bench_adjoint(api, scene, sc, dev, tuning=None):
    """Adjoint workload (512x512, 8 spp, depth 4): replay adjoint vs primal."""
    import torch
    from paper_2001_02620_gb300 import inputs as I
    view, params = I.adjoint_view(), I.adjoint_params()
    a0 = I.albedo(sc.n_quads)
    alb = torch.from_numpy(a0).to(dev)
    tgt_alb = torch.from_numpy(I.perturbed_albedo(a0)).to(dev)
    (target,) = scene.render([view], tgt_alb, params)
    img = torch.empty_like(target)
    dimg = torch.empty_like(target)
    grad = torch.zeros_like(alb)
    tp = _time(lambda: scene.render([view], alb, params, outs=[img], tuning=tuning), 5)
    api.l2_loss(img, target, dimg)
    ta = _time(lambda: scene.adjoint([view], alb, [dimg], grad, params, tuning=tuning), 5)
    scene.check()
    return {"primal_ms": tp * 1e3, "adjoint_ms": ta * 1e3, "ratio": ta / tp,
            "paths": view.w * view.h * view.spp, "n_params": int(a0.size)}


def bench_shading(api, scene, sc, view, d_alb, params, dev, tuning=None):
    """Richer shading on the same frame: per-face textures (4x4 RGB texels
    per quad, the Ptex stand-in) modulating the albedo, and the 23 key
    lights sampled at every vertex beside the sun (one more shadow ray per
    vertex); rays and time against the plain frame."""
    import dataclasses
    import torch
    from paper_2001_02620_gb300 import inputs as I
    tex = torch.from_numpy(I.face_textures(sc.n_quads)).to(dev)
    lit = dataclasses.replace(params, tex=tex, lights=I.mid_lights())
    img = torch.empty((view.h, view.w, 3), device=dev)
    out = {}
    for name, p in (("plain", params), ("textures_and_key_lights", lit)):
        t = _time(lambda: scene.render([view], d_alb, p, outs=[img], tuning=tuning), 5)
        stats = torch.zeros(STAT_WORDS, dtype=torch.int64, device=dev)
        scene.render([view], d_alb, p, outs=[img], stats=stats, tuning=tuning)
        st = stats.cpu().numpy()
        rays = int(st[0] + st[6])
        out[name] = {"ms": t * 1e3, "rays": rays, "mrays_s": rays / t / 1e6,
                     "path_samples_per_s": view.w * view.h * view.spp / t}
    scene.check()
    out["texture"] = "4x4 RGB texels per quad, bilinear in quad (u, v), times the quad albedo"
    out["lights"] = "23 square key lights (side 120, height 600), one sample per vertex"
    del tex
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle (the plain CPU implementation the
    GPU path is checked against) timed on the host cores, each step a
    bounded random pixel sample of the same workload's frame."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    sc, view, params, alb = load_workload(args.workload, args.moana_scale)
    t0 = time.time()
    osc = O.OracleScene(sc)
    build_s = time.time() - t0
    per, secs = [], []
    base = None
    frame = f"{view.w}x{view.h} {args.workload}"
    for k in range(args.warmup + args.steps):
        t0 = time.time()
        r = oracle_sample(osc, view, params, alb, budget_s=5.0 if k >= args.warmup else 1.0,
                          frame=frame, seed=1000 + k, build_s=build_s)
        if k >= args.warmup:
            secs.append(time.time() - t0)
            per.append(r["value"])
            base = r
    v = float(np.median(per))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mrays/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": 1e3 * float(np.mean(secs)), "scaling": "weak",
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, args.moana_scale),
            "setup": {"parallelism": f"{base['cores']} host threads (FP64 oracle)",
                      "oracle_build_s": build_s},
            "cpu_baseline": {"value": v, "unit": "Mrays/s", "cores": base["cores"], "kind": "oracle",
                             "sample": f"per step: {base['sample']}"},
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)


def measure(scene, view, d_alb, params, tuning, steps, warmup, world, dev, clocks=None):
    """One workload's headline numbers: traversal counters of one render,
    then `warmup` untimed steps and `steps` timed steps (barrier and device
    synchronisation on both sides, CUDA events on the launch stream, max over
    ranks), then the same steps again with a CUDA event pair around every
    stage launch (stages in order) for the per-kernel times."""
    import torch
    import torch.distributed as dist
    stream = torch.cuda.current_stream()
    img = torch.empty((view.h, view.w, 3), device=dev)

    def step(stage_times=False):
        scene.render([view], d_alb, params, outs=[img], tuning=tuning, stage_times=stage_times)

    stats = torch.zeros(STAT_WORDS, dtype=torch.int64, device=dev)
    scene.render([view], d_alb, params, outs=[img], stats=stats, tuning=tuning)
    scene.check()
    st = [int(x) for x in stats.cpu().numpy()]
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    scene.stage_times(reset=True)
    if world > 1:
        dist.barrier()
    if clocks:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / steps
    clk = clocks.stop() if clocks else None
    scene.check()
    scene.stage_times(reset=True)
    for _ in range(steps):
        step(stage_times=True)
    torch.cuda.synchronize()
    stages = scene.stage_times(reset=True)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    c_rays, c_nodes, c_quads, c_insts, c_fb, verts = st[0:6]
    s_rays, s_nodes, s_quads, s_insts, s_fb, _ = st[6:12]
    # algorithmic bytes: 64 B per node, 48 B per quad tested, 64 B per
    # instance entry; per closest-hit ray 32 B ray + 4 B queue slot read and a
    # 16 B hit written; per shadow ray 16 B origin + 4 B slot + 16 B pending
    # term read and 16 B radiance updated
    closest_bytes = 64 * c_nodes + 48 * c_quads + 64 * c_insts + (32 + 4 + 16) * c_rays
    shadow_bytes = 64 * s_nodes + 48 * s_quads + 64 * s_insts + (16 + 4 + 16 + 16) * s_rays
    frame_bytes = closest_bytes + shadow_bytes + (12 + 48 + 64) * verts + 12 * view.w * view.h
    rays = c_rays + s_rays
    staged_ms = sum(v[0] for v in stages.values()) / steps
    tr_ms, tr_n = stages["trace_closest"]
    return {"ms": ms, "rays": rays, "paths": view.w * view.h * view.spp, "img": img, "clocks": clk,
            "stages": stages, "staged_ms": staged_ms, "tuning": tuning,
            "closest_ms_step": tr_ms / steps, "closest_launches_step": tr_n / steps,
            "closest_bytes": closest_bytes, "frame_bytes": frame_bytes,
            "launches_step": sum(v[1] for v in stages.values()) / steps,
            "counters": {"closest": {"rays": c_rays, "nodes": c_nodes, "quads": c_quads,
                                     "instance_entries": c_insts, "fp64_retests": c_fb},
                         "shadow": {"rays": s_rays, "nodes": s_nodes, "quads": s_quads,
                                    "instance_entries": s_insts, "fp64_retests": s_fb},
                         "vertices": verts}}


def roofline(m, workload, world, hbm, peak_kind, l2_gbs):
    """Roofline of the dominant kernel (closest-hit trace): its algorithmic
    bytes per launch over its CUDA-event launch time, against the HBM copy
    peak (a scene far larger than L2) or the measured L2 read bandwidth (a
    scene whose hot set stays in L2)."""
    ms_launch = m["closest_ms_step"] / max(1.0, m["closest_launches_step"])
    bytes_launch = m["closest_bytes"] / max(1.0, m["closest_launches_step"])
    achieved = bytes_launch / (ms_launch * 1e-3) / 1e9 if ms_launch > 0 else None
    traffic, traffic_kernel, traffic_src = recorded_traffic(workload, m.get("tuning"))
    bound, peak, unit_kind = ("hbm", hbm, f"{peak_kind} hbm_gbs") if workload == "moana" else \
        ("l2", l2_gbs, "measured here: qrt_read_bandwidth over a 64 MB buffer, 40 sweeps")
    value = world * m["rays"] / (m["ms"] * 1e-3) / 1e6
    return {"bound": bound,
            "kernel": "wave_trace<closest> (closest-hit trace, "
                      f"{m['closest_launches_step']:.0f} launches per step, "
                      f"{100 * m['closest_ms_step'] / m['staged_ms']:.1f}% of a step whose stages run in order)",
            "kernel_timing": "CUDA events around each launch on its stream in a second pass of the same "
                             "steps with the stages in order (the headline pass overlaps shadow and "
                             "closest-hit launches on two streams)",
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "peak_kind": unit_kind + (" (of measured)" if peak_kind == "measured" or bound == "l2"
                                      else " (of fallback)"),
            "traffic": traffic, "traffic_kernel": traffic_kernel,
            "traffic_source": traffic_src or "no ncu capture of the current kernel sources",
            "algorithmic_bytes_per_launch": bytes_launch,
            "hbm_gbs": hbm, "hbm_frac": achieved / hbm if achieved else None,
            "l2_read_gbs": l2_gbs, "l2_frac": achieved / l2_gbs if achieved else None,
            # loose upper bound: 48 compulsory bytes per ray (32 B ray in,
            # 16 B hit out) against the HBM copy bandwidth
            "compulsory_bound_grays_s": hbm / 48.0,
            "compulsory_frac": (value / 1e3) / (hbm / 48.0),
            "frame_algorithmic_gbs": m["frame_bytes"] / (m["ms"] * 1e-3) / 1e9}


def e2e(scene, view, alb, d_alb, params, tuning, steps, dev):
    """The metric end to end through the public API with host buffers: every
    step uploads its albedo from pinned host memory and reads its image
    back; the upload of step k + 1 runs on a copy stream into a second
    device buffer while step k renders (double buffering, as a caller
    feeding a new albedo every frame would)."""
    import torch
    stream = torch.cuda.current_stream()
    h_alb = torch.from_numpy(alb).pin_memory()
    d_albs = [d_alb, torch.empty_like(d_alb)]
    imgs = [torch.empty((view.h, view.w, 3), device=dev) for _ in range(2)]
    h_imgs = [torch.empty((view.h, view.w, 3)).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    uploaded = [torch.cuda.Event() for _ in range(2)]
    rendered = [torch.cuda.Event() for _ in range(2)]

    def upload(k):
        b = k % 2
        copy_stream.wait_event(rendered[b])        # the render that last read buffer b
        with torch.cuda.stream(copy_stream):
            d_albs[b].copy_(h_alb, non_blocking=True)
        uploaded[b].record(copy_stream)

    def steps_(n):
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            b = k % 2
            stream.wait_event(uploaded[b])
            scene.render([view], d_albs[b], params, outs=[imgs[b]], tuning=tuning)
            rendered[b].record(stream)
            h_imgs[b].copy_(imgs[b], non_blocking=True)

    steps_(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps_(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del d_albs[1]
    return ms, int(alb.nbytes), int(view.w * view.h * 3 * 4)


def sub_measurement(api, I, args, dev, world, hbm, peak_kind, l2_gbs, extras):
    """The mid workload measured beside the headline, with the batched-views
    and adjoint workloads that are defined on the mid scene."""
    sc, view, params, alb = mid_workload()
    t0 = time.time()
    scene = api.Scene(sc)
    build_s = time.time() - t0
    d_alb = torch_from(alb, dev)
    tuning = None
    if not args.no_tune:
        from paper_2001_02620_gb300 import autotune
        tuning = autotune.tune(scene, view, d_alb, params, scene_name="mid")
    m = measure(scene, view, d_alb, params, tuning, max(5, args.steps // 2), 3, world, dev)
    out = {"workload": WORKLOADS["mid"], "value": world * m["rays"] / (m["ms"] * 1e-3) / 1e6,
           "unit": "Mrays/s", "ms_per_step": m["ms"],
           "path_samples_per_s": world * m["paths"] / (m["ms"] * 1e-3),
           "rays_per_step": m["rays"], "counters": m["counters"],
           "roofline": roofline(m, "mid", world, hbm, peak_kind, l2_gbs),
           "stages_ms_per_step": {k: v[0] / max(5, args.steps // 2) for k, v in m["stages"].items()},
           "scene_build_s": build_s, "tuning": tuning}
    if "trace" in extras:
        out["trace"] = bench_trace(api, scene, view, d_alb, params, dev, tuning)
    if "batched" in extras:
        out["batched_vs_plain"] = bench_batched(api, scene, d_alb, dev, tuning)
        # many small views (32-128 px, 1-4 spp): where one launch per view
        # leaves the GPU idle between launches and in each launch's tail
        out["batched_small_vs_plain"] = bench_batched(
            api, scene, d_alb, dev, tuning,
            views=I.batched_views(n_views=64, min_log2=5.0, max_log2=7.0, max_spp=4))
    if "adjoint" in extras:
        out["adjoint_vs_primal"] = bench_adjoint(api, scene, sc, dev, tuning)
    if "progressive" in extras:
        out["progressive"] = bench_progressive(api, scene, view, d_alb, params, dev, tuning)
    if "shading" in extras:
        out["richer_shading"] = bench_shading(api, scene, sc, view, d_alb, params, dev, tuning)
    scene.close()
    return out


def torch_from(a, dev):
    import torch
    return torch.from_numpy(a).to(dev)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", default="trace,batched,adjoint,progressive,costmap,device_build,shading,mid",
                    help="comma list of sub-measurements to add (or 'none')")
    ap.add_argument("--res", type=int, default=0,
                    help="override the view side (small profiling captures only)")
    ap.add_argument("--spp", type=int, default=0, help="override spp (profiling only)")
    ap.add_argument("--no-tune", action="store_true", help="library default launch parameters")
    ap.add_argument("--workload", default="moana", choices=sorted(WORKLOADS))
    ap.add_argument("--tlas-builder", type=int, default=0, choices=[0, 1],
                    help="TLAS builder: 0 binned SAH on the host, 1 linear BVH on the device")
    ap.add_argument("--blas-builder", type=int, default=0, choices=[0, 1],
                    help="BLAS builder: 0 binned SAH on the host, 1 linear BVHs on the device")
    ap.add_argument("--moana-scale", type=float, default=1.0,
                    help="moana workload: fraction of the full counts (1 = 261M quads)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_2001_02620_gb300 import api, inputs as I
    from paper_2001_02620_gb300 import build as B
    B.build()
    extras = [] if args.extras == "none" else args.extras.split(",")
    t_gen = time.time()
    sc, view, params, alb = load_workload(args.workload, args.moana_scale)
    gen_s = time.time() - t_gen
    if args.res:
        view.w = view.h = args.res
    if args.spp:
        view.spp = args.spp
    view.pixel_base = rank * view.w * view.h  # each rank renders its own frame
    t0 = time.time()
    bopts = {k: v for k, v in (("tlas_builder", args.tlas_builder), ("blas_builder", args.blas_builder)) if v}
    scene = api.Scene(sc, build_opts=bopts or None)
    build_s = time.time() - t0
    dev = torch.device("cuda", local)
    d_alb = torch_from(alb, dev)

    tuning = None
    tune_s = 0.0
    if not args.no_tune:
        from paper_2001_02620_gb300 import autotune
        t0 = time.time()
        tuning = autotune.tune(scene, view, d_alb, params, scene_name=args.workload)
        tune_s = time.time() - t0
    # L2 read bandwidth of this GPU (a 64 MB L2-resident buffer swept 40
    # times with L2-only loads): the roofline denominator of an L2-resident scene
    l2_gbs = api.read_bandwidth_gbs(64 << 20, 40)
    hbm, peak_kind = peaks()

    m = measure(scene, view, d_alb, params, tuning, args.steps, args.warmup, world, dev,
                clocks=Clocks(local))
    e2e_ms, h2d, d2h = e2e(scene, view, alb, d_alb, params, tuning, args.steps, dev)
    value = world * m["rays"] / (m["ms"] * 1e-3) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.workload, args.moana_scale),
        "setup": {"parallelism": f"replicas{world}",
                  "tlas_builder": "device linear BVH" if args.tlas_builder else "host binned SAH",
                  "blas_builder": "device linear BVHs" if args.blas_builder else "host binned SAH",
                  "device_bytes": scene.stats["device_bytes"],
                  "view": [view.w, view.h, view.spp, params.max_depth]},
        "path_samples_per_s": world * m["paths"] / (m["ms"] * 1e-3),
        "rays_per_step": m["rays"], "paths_per_step": m["paths"],
        "counters": m["counters"],
        "roofline": roofline(m, args.workload, world, hbm, peak_kind, l2_gbs),
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in m["stages"].items()},
        "staged_ms_per_step": m["staged_ms"],
        "e2e": {"value": world * m["rays"] / (e2e_ms * 1e-3) / 1e6, "unit": "Mrays/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "pipelining": "step k+1's albedo upload (pinned host -> device, copy stream) "
                              "overlaps step k's render; each image is read back after its render"},
        "gpu_launches": int(round(m["launches_step"] * args.steps)),
        "clocks": m["clocks"],
        "scene_build_s": build_s, "scene_gen_s": gen_s,
        "scene": {k: scene.stats[k] for k in ("n_quads", "n_instances", "blas_nodes", "tlas_nodes",
                                              "device_bytes", "max_blas_depth", "tlas_depth")},
        "build_phase_s": dict(zip(("blas_build", "blas_check", "instances", "tlas", "concat", "upload"),
                                  scene.stats["phase_seconds"])),
        "tuning": tuning, "tune_s": tune_s,
    }
    if "trace" in extras:
        line["trace"] = bench_trace(api, scene, view, d_alb, params, dev, tuning)
    if "costmap" in extras:
        line["cost_map"] = bench_cost_map(api, scene, view, d_alb, params, dev, tuning)
    if "progressive" in extras:
        line["progressive"] = bench_progressive(api, scene, view, d_alb, params, dev, tuning)
    if args.workload == "mid":
        if "batched" in extras:
            line["batched_vs_plain"] = bench_batched(api, scene, d_alb, dev, tuning)
            line["batched_small_vs_plain"] = bench_batched(
                api, scene, d_alb, dev, tuning,
                views=I.batched_views(n_views=64, min_log2=5.0, max_log2=7.0, max_spp=4))
        if "adjoint" in extras:
            line["adjoint_vs_primal"] = bench_adjoint(api, scene, sc, dev, tuning)
        if "shading" in extras:
            line["richer_shading"] = bench_shading(api, scene, sc, view, d_alb, params, dev, tuning)
    if "device_build" in extras and not (args.tlas_builder or args.blas_builder):
        line["device_build"] = bench_device_build(api, scene, sc, view, d_alb, params, dev, tuning,
                                                  rays=m["rays"])
    scene.close()
    del scene, d_alb
    torch.cuda.empty_cache()
    if "mid" in extras and args.workload != "mid":
        line["mid"] = sub_measurement(api, I, args, dev, world, hbm, peak_kind, l2_gbs, extras)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        import oracle as O
        t0 = time.time()
        osc = O.OracleScene(sc)
        ob = time.time() - t0
        line["cpu_baseline"] = oracle_sample(osc, view, params, alb, budget_s=12.0,
                                             frame=f"{view.w}x{view.h} {args.workload}", build_s=ob)
        del osc
    import resource
    line["host_peak_rss_gb"] = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1e6
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
