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


def split_log(glog, D):
    """GPU path log [P, 2D+1] -> (inst [P, D], prim [P, D], shadow [P])."""
    glog = glog.reshape(-1, 2 * D + 1)
    return glog[:, 0:2 * D:2], glog[:, 1:2 * D:2], glog[:, 2 * D]


def path_agreement(glog, ref, D):
    gi, gp, gs = split_log(glog, D)
    return (gi == ref["inst"]).all(1) & (gp == ref["prim"]).all(1) & (gs == ref["shadow"])
