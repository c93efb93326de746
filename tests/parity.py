"""Helpers for comparing the CUDA path with the oracle.

Hit IDs must be identical except on rays whose answer is decided by a near
tie: the GPU's quad, re-evaluated in FP64, is hit at a t within 1e-6 relative
of the oracle's, or the ray passes within a normalised edge margin of 1e-6 of
either quad's boundary.  Such rays are counted; any other mismatch fails.
"""
import numpy as np

NONE = 0xFFFFFFFF
REL_T = 1e-6
EDGE = 1e-6


def world_quad(scene, inst, prim):
    v, q = scene.meshes[int(scene.mesh_ids[inst])]
    P = v[q[prim]].astype(np.float64)
    M = scene.xforms[inst].reshape(3, 4).astype(np.float64)
    return P @ M[:, :3].T + M[:, 3]


def _tri(o, d, a, b, c):
    """Moller-Trumbore without rejection: (t, min barycentric, det)."""
    e1, e2 = b - a, c - a
    p = np.cross(d, e2)
    det = np.dot(e1, p)
    if det == 0.0:
        return np.inf, -np.inf, 0.0
    s = o - a
    u = np.dot(s, p) / det
    q = np.cross(s, e1)
    v = np.dot(d, q) / det
    t = np.dot(e2, q) / det
    return t, min(u, v, 1.0 - u - v), det


def quad_eval(o, d, V, tmin=0.0, tmax=np.inf):
    """FP64 quad test: (hit, t, signed margin) -- margin > 0 inside."""
    best_t, best_m, hit = np.inf, -np.inf, False
    for (a, b, c) in ((V[0], V[1], V[2]), (V[0], V[2], V[3])):
        t, m, det = _tri(o, d, a, b, c)
        if det == 0.0:
            continue
        best_m = max(best_m, m)
        if m >= 0 and tmin < t < tmax and t < best_t:
            best_t, hit = t, True
    return hit, best_t, best_m


def classify_closest(scene, rays, g_inst, g_prim, o_t, o_inst, o_prim):
    """Returns (n_mismatch, n_accepted, unexplained list)."""
    mism = np.nonzero((g_inst != o_inst) | (g_prim != o_prim))[0]
    accepted, bad = 0, []
    for k in mism:
        r = rays[k].astype(np.float64)
        o, d, tmin, tmax = r[0:3], r[4:7], r[3], r[7]
        ok = False
        margins = []
        if g_inst[k] != NONE:
            hit, t, m = quad_eval(o, d, world_quad(scene, g_inst[k], g_prim[k]), tmin, tmax)
            margins.append(abs(m))
            if hit and o_inst[k] != NONE and abs(t - o_t[k]) <= REL_T * abs(o_t[k]):
                ok = True
        if o_inst[k] != NONE:
            hit, t, m = quad_eval(o, d, world_quad(scene, o_inst[k], o_prim[k]), tmin, tmax)
            margins.append(abs(m))
        if not ok and margins and min(margins) <= EDGE:
            ok = True
        if ok:
            accepted += 1
        else:
            bad.append(int(k))
    return len(mism), accepted, bad


LOG_EXTRA = 2        # path log words after the hits: sun and key-light shadow bits
RAY_REC = 16         # GPU ray log floats per depth: ray (8), spawn point (3+1), light ray (4)


def split_log(glog, D):
    """GPU path log [P, 2D+2] -> (inst [P, D], prim [P, D], shadow [P], light [P])."""
    glog = glog.reshape(-1, 2 * D + LOG_EXTRA)
    return glog[:, 0:2 * D:2], glog[:, 1:2 * D:2], glog[:, 2 * D], glog[:, 2 * D + 1]


def path_agreement(glog, ref, D):
    gi, gp, gs, gl = split_log(glog, D)
    return ((gi == ref["inst"]).all(1) & (gp == ref["prim"]).all(1) & (gs == ref["shadow"])
            & (gl == ref["light"]))


# --------------------------------------------------------------------------
# Divergent render paths.  Past the camera ray the two sides trace different
# rays: the GPU spawns each bounce from an FP32 hit point and samples its
# direction in FP32, the oracle does both in FP64.  Where such a small
# difference moves a ray across a quad edge or past a near-equal hit, the
# paths part.  explain_divergences() takes every path whose hit IDs or
# shadow bits differ, finds the first depth where they do, and requires that
#   (a) the ray the GPU traced there is the oracle's ray up to FP32 rounding:
#       direction within DIR_TOL, origin within ORIGIN_TOL * (1 + |p|) / c,
#       where c = |cos| of the angle at the hit the origin was spawned from
#       (a grazing hit turns a rounding-size error in the ray into a larger
#       error in the hit distance, hence in the spawn point), and
#   (b) on that very FP32 ray the oracle gives the GPU's answer, or the
#       GPU's answer is an FP64 near-tie (classify_closest / the any-hit
#       analogue).
# Paths failing (a) or (b) are unexplained.
# --------------------------------------------------------------------------
ORIGIN_TOL = 1e-4
DIR_TOL = 1e-4


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def world_normal(scene, inst, prim):
    """FP64 unit geometric normal of a quad in world space (cross of the
    diagonals moved by the inverse transpose), unfaced."""
    v, q = scene.meshes[int(scene.mesh_ids[inst])]
    P = v[q[prim]].astype(np.float64)
    n = np.cross(P[2] - P[0], P[3] - P[1])
    M = scene.xforms[inst].reshape(3, 4).astype(np.float64)[:, :3]
    return _unit(np.linalg.inv(M).T @ n)


def first_divergence(gi, gp, gs, oi, op, osh, gl=None, ol=None):
    """Per path: (depth k >= 1 of the first difference or 0, kind) where kind
    is 'hit' (instance or quad of the depth-k hit), 'shadow' (the sun shadow
    bits of vertex k, hits equal through depth k) or 'light' (the key-light
    shadow bits of vertex k, sun bits equal there)."""
    P, D = gi.shape
    hit_bad = (gi != oi) | (gp != op)
    kh = np.where(hit_bad.any(1), hit_bad.argmax(1) + 1, D + 1)
    nv = min(D, 16)
    sh = np.stack([((gs >> (2 * i)) & 3) != ((osh >> (2 * i)) & 3) for i in range(nv)], 1)
    ks = np.where(sh.any(1), sh.argmax(1) + 1, D + 1)
    if gl is None:
        gl = ol = np.zeros_like(gs)
    lb = np.stack([((gl >> (2 * i)) & 3) != ((ol >> (2 * i)) & 3) for i in range(nv)], 1)
    kl = np.where(lb.any(1), lb.argmax(1) + 1, D + 1)
    k = np.minimum(np.minimum(kh, ks), kl)
    kind = np.where(k == kh, "hit", np.where(k == ks, "shadow", "light"))
    k = np.where(k > D, 0, k)
    return k, kind


def explain_divergences(scene, osc, glog, grays, ref, D, sun_dir, gpu_closest=None, lights=None):
    """glog: GPU path log [P, 2D+2] (uint32); grays: GPU ray log [P, D, 16]
    (float32); ref: oracle render dict with log=True, rays=True for the same
    paths.  gpu_closest(rays float32 [n, 8]) -> (inst, prim) traces rays on
    the GPU (used to name the occluder of a shadow ray only the GPU found
    blocked).  Returns a dict of counts, the largest ray deviations seen and
    the list of unexplained path indices."""
    gi, gp, gs, glt = split_log(glog, D)
    oi, op, osh, olt = ref["inst"], ref["prim"], ref["shadow"], ref["light"]
    orays = ref["rays"]
    k, kind = first_divergence(gi, gp, gs, oi, op, osh, glt, olt)
    div = np.nonzero(k)[0]
    sun = np.asarray(sun_dir, dtype=np.float64)
    l64 = sun / np.linalg.norm(sun)
    l32 = l64.astype(np.float32)
    out = dict(paths=len(gi), divergent=len(div), by_ray=0, near_tie=0, grazing_sun=0,
               unexplained=[], max_origin_dev=0.0, max_dir_dev=0.0, depths={})
    hit_paths = [p for p in div if kind[p] == "hit"]
    sh_paths = [p for p in div if kind[p] == "shadow"]
    lt_paths = [p for p in div if kind[p] == "light"]
    # (a) the GPU ray at the divergence is the oracle's ray up to rounding
    ok_ray = {}
    for p in div:
        j = k[p] - 1
        if kind[p] == "hit":
            og, dg = grays[p, j, 0:3].astype(np.float64), grays[p, j, 4:7].astype(np.float64)
            oo, do = orays[p, j, 0:3], orays[p, j, 3:6]
            dev_d = float(np.abs(_unit(dg) - _unit(do)).max())
            src = j - 1          # the hit this origin was spawned from (none for the camera ray)
        else:
            og, oo = grays[p, j, 8:11].astype(np.float64), orays[p, j, 6:9]
            dev_d = 0.0
            if kind[p] == "light" and (glt[p] >> (2 * j)) & (olt[p] >> (2 * j)) & 1:
                # both traced a key-light shadow ray: compare the directions
                dev_d = float(np.abs(_unit(grays[p, j, 12:15].astype(np.float64))
                                     - _unit(orays[p, j, 9:12])).max())
            src = j
        cosv = 1.0
        if src >= 0:
            nrm = world_normal(scene, oi[p, src], op[p, src])
            cosv = max(abs(float(nrm @ _unit(orays[p, src, 3:6]))), 1e-3)
        dev_o = float(np.abs(og - oo).max() / (1.0 + np.abs(oo).max())) * cosv
        out["max_origin_dev"] = max(out["max_origin_dev"], dev_o)
        out["max_dir_dev"] = max(out["max_dir_dev"], dev_d)
        ok_ray[p] = dev_o <= ORIGIN_TOL and dev_d <= DIR_TOL
        out["depths"][int(k[p])] = out["depths"].get(int(k[p]), 0) + 1
    # (b) closest-hit divergences: the oracle on the GPU's own FP32 ray
    if hit_paths:
        rays = np.stack([grays[p, k[p] - 1, 0:8] for p in hit_paths]).astype(np.float32)
        g_i = np.array([gi[p, k[p] - 1] for p in hit_paths], dtype=np.uint32)
        g_p = np.array([gp[p, k[p] - 1] for p in hit_paths], dtype=np.uint32)
        o_t, o_i, o_p, _, _ = osc.trace_closest(rays)
        same = (o_i == g_i) & (o_p == g_p)
        _, _, bad = classify_closest(scene, rays, g_i, g_p, o_t, o_i, o_p)
        bad = set(bad)
        for n, p in enumerate(hit_paths):
            if not ok_ray[p]:
                out["unexplained"].append(int(p))
            elif same[n]:
                out["by_ray"] += 1
            elif n not in bad:
                out["near_tie"] += 1
            else:
                out["unexplained"].append(int(p))
    # shadow divergences at vertex k (hits equal through depth k)
    if sh_paths:
        rays = np.zeros((len(sh_paths), 8), dtype=np.float32)
        for n, p in enumerate(sh_paths):
            rays[n, 0:3] = grays[p, k[p] - 1, 8:11]
            rays[n, 4:7] = l32
            rays[n, 7] = np.inf
        occ_o = osc.trace_any(rays)
        need_gpu = []
        for n, p in enumerate(sh_paths):
            j = k[p] - 1
            g_bits, o_bits = (gs[p] >> (2 * j)) & 3, (osh[p] >> (2 * j)) & 3
            if (g_bits & 1) != (o_bits & 1):
                # one side traced a shadow ray, the other did not: n.l is
                # within rounding of zero at this vertex
                nrm = world_normal(scene, gi[p, j], gp[p, j])
                if abs(float(nrm @ l64)) <= 1e-5:
                    out["grazing_sun"] += 1
                else:
                    out["unexplained"].append(int(p))
                continue
            if not ok_ray[p]:
                out["unexplained"].append(int(p))
                continue
            g_occ = bool(g_bits & 2)
            if occ_o[n] == g_occ:
                out["by_ray"] += 1
            elif not g_occ:
                # the oracle finds an occluder the GPU missed: it must be grazed
                t, i_, q_, _, _ = osc.trace_closest(rays[n:n + 1])
                _, _, m = quad_eval(rays[n, 0:3].astype(np.float64), l64,
                                    world_quad(scene, i_[0], q_[0]))
                if abs(m) <= EDGE:
                    out["near_tie"] += 1
                else:
                    out["unexplained"].append(int(p))
            else:
                need_gpu.append((n, p))
        if need_gpu:
            sel = np.stack([rays[n] for n, _ in need_gpu])
            if gpu_closest is None:
                out["unexplained"] += [int(p) for _, p in need_gpu]
            else:
                ci, cq = gpu_closest(sel)
                for m_, (n, p) in enumerate(need_gpu):
                    if ci[m_] == NONE:
                        out["unexplained"].append(int(p))
                        continue
                    _, _, m = quad_eval(sel[m_, 0:3].astype(np.float64), l64,
                                        world_quad(scene, ci[m_], cq[m_]))
                    if abs(m) <= EDGE:
                        out["near_tie"] += 1
                    else:
                        out["unexplained"].append(int(p))
    # key-light shadow divergences at vertex k (hits and sun bits equal)
    for p in lt_paths:
        j = k[p] - 1
        g_bits, o_bits = (glt[p] >> (2 * j)) & 3, (olt[p] >> (2 * j)) & 3
        if (g_bits & 1) != (o_bits & 1):
            # one side sampled a point it could see, the other not: the point
            # lies within rounding of the vertex's horizon or the light's plane
            src = orays[p, j, 9:12] if o_bits & 1 else grays[p, j, 12:15].astype(np.float64)
            nrm = world_normal(scene, gi[p, j], gp[p, j])
            if abs(float(nrm @ _unit(src))) <= 1e-5 or _light_grazing(src, lights):
                out["grazing_sun"] += 1
            else:
                out["unexplained"].append(int(p))
            continue
        if not ok_ray[p]:
            out["unexplained"].append(int(p))
            continue
        ray = np.zeros((1, 8), dtype=np.float32)
        ray[0, 0:3] = grays[p, j, 8:11]
        ray[0, 4:7] = grays[p, j, 12:15]
        ray[0, 7] = grays[p, j, 15]
        g_occ = bool(g_bits & 2)
        o_occ = bool(osc.trace_any(ray)[0])
        if o_occ == g_occ:
            out["by_ray"] += 1
            continue
        # an occluder found by one side only must be grazed by the ray
        if g_occ and gpu_closest is not None:
            ci, cq = gpu_closest(ray)
            i_, q_ = ci[0], cq[0]
        else:
            _, i_a, q_a, _, _ = osc.trace_closest(ray)
            i_, q_ = i_a[0], q_a[0]
        if i_ == NONE:
            out["unexplained"].append(int(p))
            continue
        hit, t, m = quad_eval(ray[0, 0:3].astype(np.float64), ray[0, 4:7].astype(np.float64),
                              world_quad(scene, i_, q_), 0.0, np.inf)
        if abs(m) <= EDGE or (hit and abs(t - float(ray[0, 7])) <= REL_T * float(ray[0, 7])):
            out["near_tie"] += 1
        else:
            out["unexplained"].append(int(p))
    return out


def _light_grazing(direction, lights) -> bool:
    """True when a direction toward a key-light point is within rounding of
    a light's plane (cos at the light within 1e-5)."""
    if lights is None:
        return False
    d = _unit(np.asarray(direction, dtype=np.float64))
    for L in np.asarray(lights, dtype=np.float64):
        n = np.cross(L[3:6], L[6:9])
        if abs(float(d @ _unit(n))) <= 1e-5:
            return True
    return False


def count_rays(glog, D):
    """Closest-hit and shadow rays of logged paths (for the near-tie rate)."""
    gi, _, gs, gl = split_log(glog, D)
    hits = (gi != NONE).sum()
    escapes = ((gi == NONE).any(1)).sum()  # the ray after a path's last hit left the scene
    shadow = sum(int(((gs >> (2 * i)) & 1).sum() + ((gl >> (2 * i)) & 1).sum()) for i in range(min(D, 16)))
    return int(hits + escapes + shadow)


def texture_slack(scene, ref, spp, tex):
    """Per-pixel relative radiance slack of a textured render (0 without
    textures).  A ray's FP32 rounding -- about 2^-22 of its length scale in
    origin and direction -- moves its hit point along the surface by
    2^-22 (|p| + t + 1) / |cos theta|; over a quad of smallest edge s that is
    a shift of the quad-space (u, v) of at most that over s, and the bilinear
    texture changes by at most R * (texel spread) per unit of (u, v), i.e. by
    R * spread / min texel relative.  Summed over the path's hits (each
    hit's factor multiplies the path's radiance), times a safety factor 16.
    Returns [n_pix] slacks (max over the pixel's samples)."""
    if tex is None:
        return None
    R = tex.shape[1]
    tmin, tmax = float(tex.min()), float(tex.max())
    gain = R * (tmax - tmin) / max(tmin, 1e-6)
    inst, prim, rays = ref["inst"], ref["prim"], ref["rays"]
    P, D = inst.shape
    slack = np.zeros(P)
    edge_cache = {}
    for p in range(P):
        for k in range(D):
            i, q = inst[p, k], prim[p, k]
            if i == NONE:
                break
            o, d, sp = rays[p, k, 0:3], rays[p, k, 3:6], rays[p, k, 6:9]
            key = (int(i), int(q))
            if key not in edge_cache:
                V = world_quad(scene, i, q)
                e = [np.linalg.norm(V[(a + 1) % 4] - V[a]) for a in range(4)]
                n = world_normal(scene, i, q)
                edge_cache[key] = (max(min(e), 1e-12), n)
            s_min, n = edge_cache[key]
            c = max(abs(float(n @ _unit(d))), 1e-4)
            t = float(np.linalg.norm(sp - o))
            du = 2.0 ** -22 * (np.abs(sp).max() + t + 1.0) / (c * s_min)
            slack[p] += gain * du
    return 16.0 * slack.reshape(-1, spp).max(1)


def render_parity(api, gs, osc, scene, view, alb, params, pixels=None, tuning=None):
    """Renders `view` (whole frame, the given launch tuning) on the GPU with
    path and ray logs, renders the sampled pixels (None = all) with the
    oracle, and compares: returns (pix_ok [n] bool, per-pixel radiance error
    where every sample's path agrees, oracle rgb there, divergence report
    from explain_divergences with 'rays' = rays of the compared paths)."""
    import torch
    D = params.max_depth
    spp = int(view.spp)
    alb_d = torch.from_numpy(alb).cuda()
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    rlog = torch.zeros(api.ray_log_floats([view], D), dtype=torch.float32, device="cuda")
    gparams = params
    if getattr(params, "tex", None) is not None and not isinstance(params.tex, torch.Tensor):
        import dataclasses
        gparams = dataclasses.replace(params, tex=torch.from_numpy(params.tex).cuda())
    (img,) = gs.render([view], alb_d, gparams, path_log=log, ray_log=rlog, tuning=tuning)
    gs.check()
    npix = int(view.w) * int(view.h)
    if pixels is None:
        pixels = np.arange(npix, dtype=np.int64)
    px = torch.from_numpy(np.asarray(pixels, dtype=np.int64)).cuda()
    paths = (px[:, None] * spp + torch.arange(spp, device="cuda")[None, :]).reshape(-1)
    glog = log.view(-1, 2 * D + LOG_EXTRA)[paths].cpu().numpy().view(np.uint32)
    grays = rlog.view(-1, D, RAY_REC)[paths].cpu().numpy()
    g = img.reshape(-1, 3)[px].double().cpu().numpy()
    ref = osc.render(view, alb, params, pixels=pixels, log=True, rays=True)
    agree = path_agreement(glog, ref, D)
    pix_ok = agree.reshape(-1, spp).all(1)
    r = ref["rgb"]
    err = np.abs(g[pix_ok] - r[pix_ok])
    tex = getattr(params, "tex", None)
    slack = texture_slack(scene, ref, spp, None if tex is None else np.asarray(tex))
    if slack is not None:
        # textured paths: allowed error = the 1e-4 bound plus the texture
        # slack of the pixel's paths; err is rescaled so that callers keep
        # asserting err <= 1e-4 |r| + 1e-6
        r_ok = np.abs(r[pix_ok])
        extra = slack[pix_ok][:, None] * r_ok
        tex_raw = err > 1e-4 * r_ok + 1e-6
        err = np.maximum(err - extra, 0.0)

    def gpu_closest(rays):
        h = gs.trace_closest(torch.from_numpy(np.ascontiguousarray(rays)).cuda())
        h = h.cpu().numpy().view(np.uint32)
        return h[:, 1], h[:, 2]

    rep = explain_divergences(scene, osc, glog, grays, ref, D, params.sun_dir, gpu_closest,
                              getattr(params, "lights", None))
    rep["rays"] = count_rays(glog, D)
    if slack is not None:
        # agreeing pixels that needed the texture slack beyond 1e-4
        rep["tex_slack_pixels"] = int(tex_raw.any(1).sum())
    rep["divergent_path_frac"] = rep["divergent"] / max(1, rep["paths"])
    rep["near_tie_ray_frac"] = rep["near_tie"] / max(1, rep["rays"])
    return pix_ok, err, r[pix_ok], rep


def report_line(name, rep) -> str:
    return (f"{name}: {rep['divergent']}/{rep['paths']} paths diverge "
            f"({rep['divergent_path_frac']:.2e}): {rep['by_ray']} by the FP32 ray, "
            f"{rep['near_tie']} FP64 near-ties ({rep['near_tie_ray_frac']:.1e} of {rep['rays']} rays), "
            f"{rep['grazing_sun']} grazing sun or light, {len(rep['unexplained'])} unexplained; "
            f"first depths {dict(sorted(rep['depths'].items()))}; max ray deviation "
            f"origin {rep['max_origin_dev']:.1e} (x cos at its hit) direction {rep['max_dir_dev']:.1e}")


def rays_from_render(api, gs, view, alb_d, params, depth_sets=(1, 2)):
    """Ray sets dumped from a render through the ray log: {'depth1': camera
    rays, 'depth2': the first diffuse bounce rays, 'shadow': the shadow rays
    toward the sun} as float32 [n, 8] qrt_ray arrays (rays a path did not
    trace are left out)."""
    import torch
    D = params.max_depth
    rlog = torch.zeros(api.ray_log_floats([view], D), dtype=torch.float32, device="cuda")
    gs.render([view], alb_d, params, ray_log=rlog)
    gs.check()
    r = rlog.view(-1, D, RAY_REC)
    out = {}
    for k in depth_sets:
        rk = r[:, k - 1, 0:8]
        keep = rk[:, 7] != 0  # tmax = inf on a traced ray, 0 on an empty record
        out[f"depth{k}"] = rk[keep].cpu().numpy()
    so = r[:, :, 8:11].reshape(-1, 3)   # spawn points: the shadow rays' origins
    keep = (so != 0).any(1)
    so = so[keep].cpu().numpy()
    sun = np.asarray(params.sun_dir, dtype=np.float64)
    l = (sun / np.linalg.norm(sun)).astype(np.float32)
    sh = np.zeros((so.shape[0], 8), dtype=np.float32)
    sh[:, 0:3] = so
    sh[:, 4:7] = l
    sh[:, 7] = np.inf
    out["shadow"] = sh
    return out
