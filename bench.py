"""Benchmark of the instanced-quad path tracer on one GB300 (or N replicas).

A step is one qrt_render_spp of the mid workload: 64 prototypes + terrain
(5.73 M unique quads), 100k instances, 1024x1024, 4 spp, path depth 5,
environment + sun with shadow rays.  value = all rays traced per second
(closest-hit + shadow), the accounting of the paper's Mray/s (Section 6, "Results").

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
                  "paper_2001_02620_gb300/csrc/bvh_build.cpp", "paper_2001_02620_gb300/csrc/capi.cpp"]


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


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the closest-hit trace kernel from the committed
    ncu summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None, None
    e = d.get(workload)
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None, None
    return float(e["dram_bytes_per_launch"]), e.get("kernel")


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


def oracle_sample(sc, view, params, alb, budget_s: float, frame: str = "1024x1024 mid"):
    """Times the FP64 oracle on a bounded pixel sample of the same workload."""
    import oracle as O
    t0 = time.time()
    osc = O.OracleScene(sc)
    build_s = time.time() - t0
    rng = np.random.default_rng(99)
    npix = view.w * view.h
    n = 256
    rays = 0
    elapsed = 0.0
    done = 0
    while elapsed < budget_s and done < npix:
        px = rng.choice(npix, size=n, replace=False)
        t = time.time()
        r = osc.render(view, alb, params, pixels=px, log=True)
        dt = time.time() - t
        hits = int((r["inst"] != 0xFFFFFFFF).sum())
        sh = r["shadow"]
        shadow = sum(int(((sh >> (2 * i)) & 1).sum()) for i in range(params.max_depth))
        rays += hits + int(r["escaped"]) + shadow
        elapsed += dt
        done += n
        n *= 2
    cores = os.cpu_count() or 1
    return {"value": rays / elapsed / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} random pixels x {view.spp} spp of the {frame} frame "
                      f"({rays} rays, {elapsed:.1f} s FP64, oracle BVH build {build_s:.1f} s excluded)",
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


def bench_trace(scene, sc, dev, tuning=None, eye=(2048.0, -300.0, 450.0)):
    """trace_closest / trace_any throughput on 4M-ray sets over the scene:
    a coherent bundle from the camera, incoherent rays from random origins,
    and parallel rays toward the sun."""
    import torch
    from paper_2001_02620_gb300 import inputs as I
    ext = float(sc.meta.get("extent", 4096.0))
    lo = np.array([0.0, 0.0, -150.0])
    hi = np.array([ext, ext, 250.0])
    n = 1 << 22
    sets = {
        "primary": I.rays_focused(n, eye, lo, hi, seed=51),
        "incoherent": I.rays_random(n, lo, hi, seed=52),
        "shadow": I.rays_parallel(n, lo, hi, I.MID_SUN_DIR, seed=53),
    }
    out = {}
    hits = torch.empty((n, 4), dtype=torch.int32, device=dev)
    bits = torch.empty(((n + 31) // 32,), dtype=torch.int32, device=dev)
    for name, rays in sets.items():
        d = torch.from_numpy(rays).to(dev)
        tc = _time(lambda: scene.trace_closest(d, hits, tuning=tuning), 5)
        ta = _time(lambda: scene.trace_any(d, bits, tuning=tuning), 5)
        st = torch.zeros(6, dtype=torch.int64, device=dev)
        scene.trace_stats(d, False, hits, st)
        s = st.cpu().numpy()
        out[name] = {"closest_mrays_s": n / tc / 1e6, "any_mrays_s": n / ta / 1e6,
                     "hit_rate": float((hits[:, 1] != -1).float().mean().item()),
                     "nodes_per_ray": float(s[1]) / n, "quads_per_ray": float(s[2]) / n,
                     "instances_per_ray": float(s[3]) / n}
    scene.check()
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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, view, params, alb = mid_workload()
    per = []
    secs = []
    base = None
    for k in range(args.warmup + args.steps):
        t0 = time.time()
        r = oracle_sample(sc, view, params, alb, budget_s=8.0 if k >= args.warmup else 2.0)
        if k >= args.warmup:
            secs.append(time.time() - t0)
            per.append(r["value"])
            base = r
    v = float(np.median(per))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mrays/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": 1e3 * float(np.mean(secs)), "scaling": "weak",
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["mid"],
                       "parallelism": f"{base['cores']} host threads (FP64 oracle)"},
            "cpu_baseline": {"value": v, "unit": "Mrays/s", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", default="trace,batched,adjoint,progressive,costmap,device_build",
                    help="comma list of sub-measurements to add (or 'none')")
    ap.add_argument("--res", type=int, default=0,
                    help="override the view side (small profiling captures only)")
    ap.add_argument("--spp", type=int, default=0, help="override spp (profiling only)")
    ap.add_argument("--no-tune", action="store_true", help="library default launch parameters")
    ap.add_argument("--workload", default="mid", choices=sorted(WORKLOADS))
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
    t_gen = time.time()
    if args.workload == "moana":
        sc, view, params, alb = moana_workload(args.moana_scale)
    else:
        sc, view, params, alb = mid_workload()
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
    d_alb = torch.from_numpy(alb).to(dev)
    img = torch.empty((view.h, view.w, 3), device=dev)
    stream = torch.cuda.current_stream()

    tuning = None
    tune_s = 0.0
    if not args.no_tune:
        from paper_2001_02620_gb300 import autotune
        t0 = time.time()
        tuning = autotune.tune(scene, view, d_alb, params, scene_name="mid")
        tune_s = time.time() - t0

    def step(stage_times=False):
        scene.render([view], d_alb, params, outs=[img], tuning=tuning, stage_times=stage_times)

    # counters of one render (same launch configuration, counters added)
    stats = torch.zeros(STAT_WORDS, dtype=torch.int64, device=dev)
    scene.render([view], d_alb, params, outs=[img], stats=stats, tuning=tuning)
    scene.check()
    st = [int(x) for x in stats.cpu().numpy()]
    c_rays, c_nodes, c_quads, c_insts, c_fb, verts = st[0:6]
    s_rays, s_nodes, s_quads, s_insts, s_fb, _ = st[6:12]
    rays, nodes, quads, insts, fallbacks = (c_rays + s_rays, c_nodes + s_nodes, c_quads + s_quads,
                                            c_insts + s_insts, c_fb + s_fb)
    paths = view.w * view.h * view.spp
    # L2 read bandwidth of this GPU (a 64 MB L2-resident buffer swept 40
    # times with L2-only loads): the second roofline denominator
    l2_gbs = api.read_bandwidth_gbs(64 << 20, 40)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    scene.stage_times(reset=True)
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    clk = clocks.stop()
    scene.check()
    # per-kernel times: the same K steps again with a CUDA event pair around
    # every stage launch.  A timed render runs its stages in order (the
    # headline pass above overlaps each depth's shadow rays with the next
    # depth's closest-hit rays on a second stream), so these are the
    # kernels' own durations.
    scene.stage_times(reset=True)
    for _ in range(args.steps):
        step(stage_times=True)
    torch.cuda.synchronize()
    stages = scene.stage_times(reset=True)
    staged_ms = sum(v[0] for v in stages.values()) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the public API with host buffers: every step
    # uploads its albedo from pinned host memory and reads its image back.
    # The upload of step k + 1 runs on a copy stream into a second device
    # buffer while step k renders (double buffering, as a caller feeding a
    # new albedo every frame would do).
    h_alb = torch.from_numpy(alb).pin_memory()
    d_albs = [d_alb, torch.empty_like(d_alb)]
    imgs = [img, torch.empty_like(img)]
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

    def e2e_steps(n):
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            b = k % 2
            stream.wait_event(uploaded[b])
            scene.render([view], d_albs[b], params, outs=[imgs[b]], tuning=tuning)
            rendered[b].record(stream)
            h_imgs[b].copy_(imgs[b], non_blocking=True)

    e2e_steps(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    hbm, peak_kind = peaks()
    # algorithmic bytes: 64 B per node, 48 B per quad tested, 64 B per instance
    # entry; per ray of the closest-hit kernel also 32 B ray + 4 B queue slot
    # read and a 16 B hit written
    closest_bytes = 64 * c_nodes + 48 * c_quads + 64 * c_insts + (32 + 4 + 16) * c_rays
    shadow_bytes = 64 * s_nodes + 48 * s_quads + 64 * s_insts + (16 + 4 + 16 + 16) * s_rays
    frame_bytes = closest_bytes + shadow_bytes + (12 + 48 + 64) * verts + 12 * view.w * view.h
    tr_ms, tr_n = stages["trace_closest"]
    tr_ms_step = tr_ms / args.steps
    launches_step = tr_n / args.steps
    achieved = closest_bytes / (tr_ms_step * 1e-3) / 1e9 if tr_ms_step > 0 else None
    traffic, traffic_kernel = recorded_traffic(args.workload)
    value = world * rays / (ms * 1e-3) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] if args.workload != "moana" or
                   args.moana_scale == 1.0 else WORKLOADS["moana"] + f" x {args.moana_scale}",
                   "parallelism": f"replicas{world}",
                   "tlas_builder": "device linear BVH" if args.tlas_builder else "host binned SAH",
                   "blas_builder": "device linear BVHs" if args.blas_builder else "host binned SAH",
                   "l2": f"working set {scene.stats['device_bytes'] / 1e9:.2f} GB > L2 (no flush)"},
        "path_samples_per_s": world * paths / (ms * 1e-3),
        "rays_per_step": rays, "paths_per_step": paths,
        "counters": {"closest": {"rays": c_rays, "nodes": c_nodes, "quads": c_quads,
                                 "instance_entries": c_insts, "fp64_retests": c_fb},
                     "shadow": {"rays": s_rays, "nodes": s_nodes, "quads": s_quads,
                                "instance_entries": s_insts, "fp64_retests": s_fb},
                     "vertices": verts},
        "roofline": {"bound": "hbm", "kernel": "wave_trace<closest> (closest-hit trace, "
                     f"{launches_step:.0f} launches per step, {100 * tr_ms_step / staged_ms:.1f}% of a "
                     "step whose stages run in order)",
                     "kernel_timing": "CUDA events around each launch in a second pass of the same "
                                      "steps with the stages in order (the headline pass overlaps "
                                      "shadow and closest-hit launches on two streams)",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None,
                     "traffic": traffic, "traffic_kernel": traffic_kernel,
                     "algorithmic_bytes_per_launch": closest_bytes / max(1.0, launches_step),
                     "peak_kind": f"{peak_kind} hbm_gbs ({'of measured' if peak_kind == 'measured' else 'of fallback'})",
                     "l2_read_gbs": l2_gbs, "l2_frac": achieved / l2_gbs if achieved else None,
                     # loose upper bound: 48 compulsory bytes per ray (32 B ray in,
                     # 16 B hit out) against the HBM copy bandwidth
                     "compulsory_bound_grays_s": hbm / 48.0,
                     "compulsory_frac": (value / 1e3) / (hbm / 48.0),
                     "l2_kind": "measured here: qrt_read_bandwidth over a 64 MB buffer, 40 sweeps",
                     "frame_algorithmic_gbs": frame_bytes / (ms * 1e-3) / 1e9},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "staged_ms_per_step": staged_ms,
        "e2e": {"value": world * rays / (e2e_ms * 1e-3) / 1e6, "unit": "Mrays/s",
                "h2d_bytes_per_step": int(alb.nbytes), "d2h_bytes_per_step": int(img.numel() * 4),
                "ms_per_step": e2e_ms,
                "pipelining": "step k+1's albedo upload (pinned host -> device, copy stream) "
                              "overlaps step k's render; each image is read back after its render"},
        "gpu_launches": int(sum(v[1] for v in stages.values())),
        "clocks": clk,
        "scene_build_s": build_s, "scene_gen_s": gen_s,
        "scene": {k: scene.stats[k] for k in ("n_quads", "n_instances", "blas_nodes", "tlas_nodes",
                                              "device_bytes", "max_blas_depth", "tlas_depth")},
        "build_phase_s": dict(zip(("blas_build", "blas_check", "instances", "tlas", "concat", "upload"),
                                  scene.stats["phase_seconds"])),
        "tuning": tuning, "tune_s": tune_s,
    }
    extras = [] if args.extras == "none" else args.extras.split(",")
    if args.workload != "mid":
        extras = [e for e in extras if e in ("trace", "progressive", "costmap", "device_build")]
    if "trace" in extras:
        line["trace"] = bench_trace(scene, sc, dev, tuning, eye=view.eye)
    if "batched" in extras:
        line["batched_vs_plain"] = bench_batched(api, scene, d_alb, dev, tuning)
        # many small views (32-128 px, 1-4 spp): where one launch per view
        # leaves the GPU idle between launches and in each launch's tail
        line["batched_small_vs_plain"] = bench_batched(
            api, scene, d_alb, dev, tuning,
            views=I.batched_views(n_views=64, min_log2=5.0, max_log2=7.0, max_spp=4))
    if "adjoint" in extras:
        line["adjoint_vs_primal"] = bench_adjoint(api, scene, sc, dev, tuning)
    if "costmap" in extras:
        line["cost_map"] = bench_cost_map(api, scene, view, d_alb, params, dev, tuning)
    if "progressive" in extras:
        line["progressive"] = bench_progressive(api, scene, view, d_alb, params, dev, tuning)
    if "device_build" in extras and not (args.tlas_builder or args.blas_builder):
        line["device_build"] = bench_device_build(api, scene, sc, view, d_alb, params, dev, tuning,
                                                  rays=rays)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = oracle_sample(sc, view, params, alb, budget_s=12.0,
                                             frame=f"{view.w}x{view.h} {args.workload}")
    import resource
    line["host_peak_rss_gb"] = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1e6
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
