"""The divergence classifier of the render parity tests, checked on the CPU
with the oracle on both sides: the oracle's own path and ray logs, packed
as the GPU's logs, agree with themselves; a hit planted in them that the
oracle does not find, or a ray moved off the oracle's ray, is reported as
unexplained; a first divergence is found at the right depth and kind."""
import numpy as np

import oracle as O
from paper_2001_02620_gb300 import inputs as I

from parity import NONE, explain_divergences, first_divergence


def _as_gpu_logs(ref, D):
    """Packs the oracle's logs in the GPU's layouts: path log [P, 2D+2]
    (uint32) and ray log [P, D, 16] (float32)."""
    P = ref["inst"].shape[0]
    glog = np.zeros((P, 2 * D + 2), dtype=np.uint32)
    glog[:, 0:2 * D:2] = ref["inst"]
    glog[:, 1:2 * D:2] = ref["prim"]
    glog[:, 2 * D] = ref["shadow"]
    glog[:, 2 * D + 1] = ref["light"]
    grays = np.zeros((P, D, 16), dtype=np.float32)
    r = ref["rays"]
    grays[:, :, 0:3] = r[:, :, 0:3]
    grays[:, :, 4:7] = r[:, :, 3:6]
    grays[:, :, 7] = np.where((r[:, :, 3:6] != 0).any(-1), np.inf, 0.0)
    grays[:, :, 8:11] = r[:, :, 6:9]
    grays[:, :, 12:16] = r[:, :, 9:13]
    return glog, grays


def _setup():
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w, view.h, view.spp = 64, 48, 2
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0),
                      tex=I.face_textures(sc.n_quads), lights=I.tiny_lights())
    ref = osc.render(view, I.albedo(sc.n_quads), params, log=True, rays=True)
    return sc, osc, view, params, ref


def test_first_divergence_depth_and_kind():
    gi = np.array([[1, 2, 3], [1, 2, 3], [1, 2, 3]], dtype=np.uint32)
    gp = gi.copy()
    oi = gi.copy()
    oi[1, 1] = 9                      # hit of depth 2 differs
    gs = np.array([0b000011, 0b11, 0b0111], dtype=np.uint32)
    osh = np.array([0b000011, 0b11, 0b0011], dtype=np.uint32)   # path 2: vertex 2's shadow
    k, kind = first_divergence(gi, gp, gs, oi, gp, osh)
    assert list(k) == [0, 2, 2] and kind[1] == "hit" and kind[2] == "shadow"
    gl = np.array([0, 0, 0b110000], dtype=np.uint32)
    ol = np.array([0, 0, 0b010000], dtype=np.uint32)   # path 2: vertex 3's key-light shadow
    k, kind = first_divergence(gi, gp, gs, gi, gp, gs, gl, ol)
    assert list(k) == [0, 0, 3] and kind[2] == "light"


def test_oracle_against_itself_agrees():
    sc, osc, view, params, ref = _setup()
    glog, grays = _as_gpu_logs(ref, params.max_depth)
    rep = explain_divergences(sc, osc, glog, grays, ref, params.max_depth, params.sun_dir,
                              lights=params.lights)
    assert rep["divergent"] == 0 and not rep["unexplained"]


def test_planted_wrong_hit_is_unexplained():
    sc, osc, view, params, ref = _setup()
    D = params.max_depth
    glog, grays = _as_gpu_logs(ref, D)
    # a path whose depth-2 ray hit something: claim another quad of that instance
    p = int(np.nonzero(ref["inst"][:, 1] != NONE)[0][0])
    glog[p, 3] = (glog[p, 3] + 1000) % 4096
    rep = explain_divergences(sc, osc, glog, grays, ref, D, params.sun_dir, lights=params.lights)
    assert rep["divergent"] == 1 and rep["unexplained"] == [p]


def test_planted_wrong_light_occlusion_is_unexplained():
    """A key-light shadow ray claimed occluded that the oracle finds clear
    (and no quad grazes) is unexplained."""
    sc, osc, view, params, ref = _setup()
    D = params.max_depth
    glog, grays = _as_gpu_logs(ref, D)
    traced_clear = np.nonzero((ref["light"] & 1) & ~((ref["light"] >> 1) & 1))[0]
    assert len(traced_clear) > 10
    p = int(traced_clear[0])
    glog[p, 2 * D + 1] |= 2      # vertex 1's light shadow ray "occluded"
    rep = explain_divergences(sc, osc, glog, grays, ref, D, params.sun_dir, lights=params.lights)
    assert rep["unexplained"] == [p]


def test_planted_wrong_ray_is_unexplained():
    sc, osc, view, params, ref = _setup()
    D = params.max_depth
    glog, grays = _as_gpu_logs(ref, D)
    # the depth-2 ray starts 0.5 units away from the oracle's spawn point, and
    # the hit recorded for it is the one that moved ray finds
    p = int(np.nonzero(ref["inst"][:, 1] != NONE)[0][3])
    grays[p, 1, 0:3] += np.float32(0.5)
    t, i_, q_, _, _ = osc.trace_closest(grays[p, 1, 0:8][None, :])
    if i_[0] == ref["inst"][p, 1] and q_[0] == ref["prim"][p, 1]:
        glog[p, 2], glog[p, 3] = NONE, NONE   # force a difference in the log
    else:
        glog[p, 2], glog[p, 3] = i_[0], q_[0]
    rep = explain_divergences(sc, osc, glog, grays, ref, D, params.sun_dir, lights=params.lights)
    assert rep["unexplained"] == [p]
