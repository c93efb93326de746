"""GPU parity on the tiny instanced scene (one 64x64-quad mesh, 256
instances): ray queries, path tracing, batching, graphs, the adjoint, and the
device error paths, all through the C ABI against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2001_02620_gb300 import inputs as I

from parity import NONE, classify_closest, path_agreement, render_parity, report_line

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_02620_gb300 import build as B
    B.build()
    from paper_2001_02620_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def tiny(api):
    sc = I.tiny_scene()
    return sc, api.Scene(sc), O.OracleScene(sc)


def _rays(sc):
    lo, hi = I.scene_box(sc)
    tg = I.instance_origins(sc)
    return np.concatenate([
        I.rays_focused(65536, (50, -120, 50), lo, hi, seed=31),
        I.rays_toward(131072, lo - 30, hi + 30, tg, 1.5, seed=32),
        I.rays_random(65536, lo, hi, seed=33),
    ])


SETTINGS = [dict(), dict(stack=32), dict(fetch=32), dict(block=64), dict(block=256, fetch=32)]


@pytest.mark.parametrize("tuning", SETTINGS)
def test_trace_closest_matches_oracle(api, tiny, tuning):
    sc, gs, osc = tiny
    rays = _rays(sc)
    d_rays = torch.from_numpy(rays).cuda()
    hits = gs.trace_closest(d_rays, tuning=tuning)
    gs.check()
    h = hits.cpu().numpy().view(np.uint32)
    o_t, o_i, o_p, _, _ = osc.trace_closest(rays)
    n, acc, bad = classify_closest(sc, rays, h[:, 1], h[:, 2], o_t, o_i, o_p)
    assert not bad, f"{len(bad)} unexplained mismatches, e.g. ray {bad[:5]}"
    assert acc / len(rays) < 1e-5, f"{acc} near-tie mismatches of {len(rays)}"
    hit = o_i != NONE
    assert hit.mean() > 0.2
    same = hit & (h[:, 1] == o_i) & (h[:, 2] == o_p)
    gt = h[:, 0].view(np.float32).astype(np.float64)
    # FP32 t: relative error plus an absolute part from rounding of coordinates ~100
    np.testing.assert_allclose(gt[same], o_t[same], rtol=2e-5, atol=1e-4)
    # misses report t = tmax
    miss = (o_i == NONE) & (h[:, 1] == NONE)
    assert np.all(gt[miss] == rays[miss, 7])


def test_trace_closest_interval_windows(api, tiny):
    """Rays with a window tmin < t < tmax cut out of their path (the open
    interval of the ray queries): hits before tmin or after tmax must not be
    reported, and the object-space re-centring at max(tmin, box entry) must
    keep the hits inside the window exact."""
    sc, gs, osc = tiny
    rays = _rays(sc)
    rng = np.random.default_rng(77)
    half = rng.random(len(rays)) < 0.5
    t0 = rng.uniform(0.0, 120.0, size=len(rays)).astype(np.float32)
    rays[half, 3] = t0[half]
    rays[half, 7] = t0[half] + rng.uniform(2.0, 60.0, size=half.sum()).astype(np.float32)
    d_rays = torch.from_numpy(rays).cuda()
    hits = gs.trace_closest(d_rays)
    gs.check()
    h = hits.cpu().numpy().view(np.uint32)
    o_t, o_i, o_p, _, _ = osc.trace_closest(rays)
    n, acc, bad = classify_closest(sc, rays, h[:, 1], h[:, 2], o_t, o_i, o_p)
    assert not bad, f"{len(bad)} unexplained mismatches, e.g. ray {bad[:5]}"
    assert acc / len(rays) < 1e-5
    hit = o_i != NONE
    assert hit[half].mean() > 0.05 and (~hit[half]).mean() > 0.05
    gt = h[:, 0].view(np.float32).astype(np.float64)
    got = h[:, 1] != NONE
    assert np.all(gt[got] > rays[got, 3]) and np.all(gt[got] < rays[got, 7])


@pytest.mark.parametrize("tuning", SETTINGS[:3])
def test_trace_any_matches_oracle(api, tiny, tuning):
    sc, gs, osc = tiny
    rays = _rays(sc)
    rays[::3, 7] = np.float32(40.0)   # finite tmax on a third of the rays
    d_rays = torch.from_numpy(rays).cuda()
    bits = gs.trace_any(d_rays, tuning=tuning).cpu().numpy().view(np.uint32)
    gs.check()
    occ = ((bits[np.arange(len(rays)) // 32] >> (np.arange(len(rays)) % 32)) & 1).astype(bool)
    ref = osc.trace_any(rays)
    mism = np.nonzero(occ != ref)[0]
    # any mismatch must be a near-grazing ray; classify with closest hits
    if len(mism):
        o_t, o_i, o_p, _, _ = osc.trace_closest(rays[mism])
        hits = gs.trace_closest(d_rays[torch.from_numpy(mism).cuda()]).cpu().numpy().view(np.uint32)
        n, acc, bad = classify_closest(sc, rays[mism], hits[:, 1], hits[:, 2], o_t, o_i, o_p)
        assert not bad
    assert len(mism) / len(rays) < 1e-5


def test_empty_and_ragged_ray_counts(api, tiny):
    sc, gs, osc = tiny
    rays = _rays(sc)
    for n in (0, 1, 31, 33, 1000, 4097):
        d = torch.from_numpy(rays[:n].copy()).cuda() if n else torch.empty((0, 8), device="cuda")
        h = gs.trace_closest(d)
        b = gs.trace_any(d)
        assert h.shape == (n, 4) and b.shape == ((n + 31) // 32,)
        if n:
            o_t, o_i, o_p, _, _ = osc.trace_closest(rays[:n])
            hh = h.cpu().numpy().view(np.uint32)
            assert (hh[:, 1] == o_i).mean() > 0.999
    gs.check()


def _check_paths(name, rep, max_divergent):
    """Every divergent path is explained (the GPU's FP32 ray at the first
    differing depth is the oracle's ray up to rounding, and on it the oracle
    agrees with the GPU or the GPU's answer is an FP64 near-tie); near-ties
    stay below 1e-5 of the rays; divergent paths stay below max_divergent."""
    print(report_line(name, rep))
    assert not rep["unexplained"], f"{name}: unexplained divergent paths {rep['unexplained'][:8]}"
    assert rep["near_tie"] <= max(1, 1e-5 * rep["rays"]), report_line(name, rep)
    assert rep["divergent_path_frac"] <= max_divergent, report_line(name, rep)


@pytest.mark.parametrize("mode", [1, 2])
def test_render_tiny_env_only(api, tiny, mode):
    sc, gs, osc = tiny
    view, params = I.tiny_view(), I.tiny_params()
    alb = I.albedo(sc.n_quads)
    pix_ok, err, r, rep = render_parity(api, gs, osc, sc, view, alb, params, tuning=dict(mode=mode))
    _check_paths(f"tiny env-only mode {mode}", rep, 3e-4)   # measured 6.1e-5 (4 of 65536)
    assert (err <= 1e-4 * np.abs(r) + 1e-6).all(), err.max()


def test_render_tiny_sun_and_depth(api, tiny):
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.spp = 3
    view.w, view.h = 200, 120   # ragged: not a multiple of the warp batch
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 2.0, 1.0),
                      env=(0.8, 1.0, 1.2))
    alb = I.albedo(sc.n_quads)
    pix_ok, err, r, rep = render_parity(api, gs, osc, sc, view, alb, params)
    _check_paths("tiny sun, depth 4, 3 spp", rep, 3e-4)   # measured 6.9e-5 (5 of 72000)
    assert (err <= 1e-4 * np.abs(r) + 1e-6).all(), err.max()


@pytest.mark.parametrize("mode", [2, 1])
def test_render_tiny_textures_and_key_lights(api, tiny, mode):
    """Per-face textures (the Ptex stand-in) and four key lights beside the
    sun: every divergent path explained, agreeing paths within 1e-4 of the
    oracle's radiance, and the key lights visibly contributing."""
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp = 160, 120, 2
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(2.0, 2.0, 2.0),
                      env=(0.6, 0.7, 0.8), tex=I.face_textures(sc.n_quads), lights=I.tiny_lights())
    alb = I.albedo(sc.n_quads)
    pix_ok, err, r, rep = render_parity(api, gs, osc, sc, view, alb, params, tuning=dict(mode=mode))
    _check_paths(f"tiny textures + key lights, mode {mode}", rep, 3e-3)
    assert (err <= 1e-4 * np.abs(r) + 1e-6).all(), err.max()
    # the lights matter: the image without them is darker somewhere
    r0 = osc.render(view, alb, dataclasses.replace(params, lights=None))["rgb"]
    assert (osc.render(view, alb, params)["rgb"] - r0).max() > 0.05


@pytest.mark.parametrize("chunk_log2,shading", [(10, False), (13, False), (21, False), (10, True),
                                                 (21, True)])
def test_wavefront_equals_single_kernel(api, tiny, chunk_log2, shading):
    """The two renderers compute the same paths with the same arithmetic; a
    tiny chunk size cuts chunks inside views and pixels' sample runs.  With
    per-face textures and key lights too (the wavefront adds a vertex's
    key-light term after its sun term, as the single kernel does)."""
    sc, gs, osc = tiny
    views = I.batched_views(n_views=5, min_log2=5.0, max_log2=7.0, max_spp=5)
    for v in views:
        v.eye = (50.0 + (v.eye[0] - 2048.0) / 40, -120.0, 50.0)
        v.look = (50.0, 50.0, 50.0)
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    if shading:
        params.tex = torch.from_numpy(I.face_textures(sc.n_quads)).cuda()
        params.lights = I.tiny_lights()
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    D = params.max_depth
    words = api.path_log_words(views, D)
    log1 = torch.zeros(words, dtype=torch.int32, device="cuda")
    log2 = torch.zeros(words, dtype=torch.int32, device="cuda")
    a = gs.render(views, alb, params, tuning=dict(mode=1), path_log=log1)
    b = gs.render(views, alb, params, tuning=dict(mode=2, chunk_log2=chunk_log2), path_log=log2)
    gs.check()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert torch.equal(log1, log2)


def test_overlapped_stages_equal_ordered_stages(api, tiny):
    """An untimed wavefront render runs each depth's shadow rays on a second
    stream beside the next depth's closest-hit rays; a timed render and the
    single-kernel renderer run everything in order.  A captured graph keeps
    the overlap.  All give the same bits, on a stream of the caller's."""
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp = 160, 96, 3
    params = I.Params(max_depth=5, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 2.0, 1.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        (a,) = gs.render([view], alb, params, tuning=dict(chunk_log2=12))
        (b,) = gs.render([view], alb, params, tuning=dict(chunk_log2=12), stage_times=True)
        (c,) = gs.render([view], alb, params, tuning=dict(mode=1))
        g = api.RenderGraph(gs, [view], alb, params, tuning=dict(chunk_log2=12))
        (d,) = g.launch()
    s.synchronize()
    gs.check()
    gs.stage_times(reset=True)
    assert torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d)
    g.close()


@pytest.mark.parametrize("mode", [2, 1])
def test_progressive_frames_equal_one_render(api, tiny, mode):
    """One sample per pixel per frame (sample_base = frame number), summed
    with qrt_accumulate, gives exactly the image of one render with spp =
    frames; each frame matches the oracle's sample of that index."""
    import dataclasses
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp = 96, 64, 6
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 2.0, 1.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    (ref,) = gs.render([view], alb, params, tuning=dict(mode=mode))
    acc = torch.zeros_like(ref)
    mean = torch.empty_like(ref)
    for f in range(view.spp):
        fv = dataclasses.replace(view, spp=1, sample_base=f)
        (frame,) = gs.render([fv], alb, params, tuning=dict(mode=mode))
        api.accumulate(acc, frame, f + 1, mean)
        if f == 3:
            pix_ok, err, r, rep = render_parity(api, gs, osc, sc, fv, I.albedo(sc.n_quads), params,
                                                tuning=dict(mode=mode))
            _check_paths(f"tiny progressive frame 3, mode {mode}", rep, 1e-3)  # measured 3.3e-4 (2 of 6144)
            assert (err <= 1e-4 * np.abs(r) + 1e-6).all()
    gs.check()
    assert torch.equal(mean, ref)


def test_cost_maps_count_every_node_visit(api, tiny):
    """qrt_render_cost: per-pixel mean inner-node visits over the pixel's
    samples; summed over the image they give back the launch's node counters
    exactly, and the image equals qrt_render_spp's."""
    sc, gs, osc = tiny
    views = [I.tiny_view(), I.tiny_view()]
    views[0].w, views[0].h, views[0].spp = 80, 48, 3
    views[1].w, views[1].h, views[1].spp, views[1].pixel_base = 40, 40, 2, 80 * 48
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 2.0, 1.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    stats = torch.zeros(12, dtype=torch.int64, device="cuda")
    imgs = [torch.empty((v.h, v.w, 3), device="cuda") for v in views]
    costs = gs.cost_maps(views, alb, params, stats, outs=imgs)
    refs = gs.render(views, alb, params)
    gs.check()
    for a, b in zip(imgs, refs):
        assert torch.equal(a, b)
    st = stats.cpu().numpy()
    total = sum(int(torch.round(c.double() * v.spp).sum().item()) for c, v in zip(costs, views))
    assert total == int(st[1] + st[7])
    assert all(float(c.min()) >= 1.0 for c in costs)   # every camera ray tests the TLAS root
    # small chunks cut the views into many chunks, whose per-path counters
    # are indexed chunk-locally.  Node-visit counts are not bit-reproducible
    # across schedules: a lane postpones a BLAS leaf while its warp tests
    # inner nodes, so when its hit distance tightens (and which stack entries
    # are culled) depends on the rays sharing the warp.  Each chunked map must
    # still add up to its own launch's counters, rays and hits must not
    # change, and the visits may differ only a little in total.
    stats2 = torch.zeros(12, dtype=torch.int64, device="cuda")
    imgs2 = [torch.empty_like(i) for i in imgs]
    costs2 = gs.cost_maps(views, alb, params, stats2, outs=imgs2, tuning=dict(chunk_log2=10))
    for a, b in zip(imgs, imgs2):
        assert torch.equal(a, b)
    st2 = stats2.cpu().numpy()
    total2 = sum(int(torch.round(c.double() * v.spp).sum().item()) for c, v in zip(costs2, views))
    assert total2 == int(st2[1] + st2[7])
    assert st2[0] == st[0] and st2[6] == st[6]          # closest-hit and shadow rays
    assert abs(total2 - total) <= 0.05 * total
    assert all(float(c.min()) >= 1.0 for c in costs2)
    with pytest.raises(api.N.QrtError):
        gs.cost_maps(views, alb, params, stats, tuning=dict(mode=1))


def test_accumulate_rejects_bad_arguments(api):
    L = api.N.lib()
    x = torch.zeros(16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.qrt_accumulate(x.data_ptr(), x.data_ptr(), None, 16, 0, s) == api.N.QRT_ERR_INVALID_ARG
    assert L.qrt_accumulate(None, x.data_ptr(), None, 16, 1, s) == api.N.QRT_ERR_INVALID_ARG
    assert L.qrt_accumulate(x.data_ptr() + 2, x.data_ptr(), None, 4, 1, s) == api.N.QRT_ERR_ALIGN
    assert L.qrt_accumulate(None, None, None, 0, 1, s) == api.N.QRT_OK


def test_adjoint_modes_agree(api, tiny):
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.spp = 2
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3, 3, 3))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    dimg = torch.from_numpy(np.random.default_rng(9).normal(size=(view.h, view.w, 3)).astype(np.float32)).cuda()
    g1 = torch.zeros_like(alb)
    g2 = torch.zeros_like(alb)
    gs.adjoint([view], alb, [dimg], g1, params, tuning=dict(mode=1))
    gs.adjoint([view], alb, [dimg], g2, params, tuning=dict(mode=2, chunk_log2=12))
    gs.check()
    # same terms, different atomic order
    torch.testing.assert_close(g1, g2, rtol=1e-5, atol=1e-7)


def _open_box():
    """Five inward faces of [-1,1]^3 (the top open), each an instance of one
    4x4-quad plane: paths bounce for many depths before they escape."""
    v, q = I.plane_mesh(4)
    faces = [
        (np.eye(3), (0.0, 0.0, -1.0)),                                   # floor
        (np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], float), (-1.0, 0.0, 0.0)),
        (np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], float), (1.0, 0.0, 0.0)),
        (np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float), (0.0, -1.0, 0.0)),
        (np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float), (0.0, 1.0, 0.0)),
    ]
    xf = np.array([np.concatenate([L, np.array(t)[:, None]], axis=1).ravel() for L, t in faces],
                  dtype=np.float32)
    return I.Scene([(v, q)], xf, np.zeros(len(faces), dtype=np.uint32))


def test_adjoint_beyond_recorded_shadow_depths(api):
    """The wavefront adjoint replays shadow-ray visibility from bits the
    primal records for depths 1..32 and traces the shadow rays of deeper
    vertices; the single-kernel adjoint traces every shadow ray again.  In an
    open box that keeps paths bouncing past depth 32 the two gradients agree."""
    sc = _open_box()
    gs = api.Scene(sc)
    view = I.View(eye=(0.1, 0.2, 0.6), look=(0.0, 0.0, -1.0), up=(0, 1, 0), vfov_deg=100.0,
                  w=64, h=64, spp=16)
    D = 40
    params = I.Params(max_depth=D, env=(0.5, 0.5, 0.5), sun_dir=(0.2, 0.3, 1.0), sun_E=(3, 2, 1))
    alb = torch.from_numpy(I.albedo(sc.n_quads, lo=0.85, hi=0.95)).cuda()
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    gs.render([view], alb, params, path_log=log)
    gl = log.cpu().numpy().view(np.uint32).reshape(-1, 2 * D + 2)
    assert (gl[:, 2 * 32] != NONE).sum() > 50          # hits at depth 33 exist
    dimg = torch.from_numpy(np.random.default_rng(5).normal(size=(view.h, view.w, 3))
                            .astype(np.float32)).cuda()
    g1 = torch.zeros_like(alb)
    g2 = torch.zeros_like(alb)
    gs.adjoint([view], alb, [dimg], g1, params, tuning=dict(mode=1))
    gs.adjoint([view], alb, [dimg], g2, params, tuning=dict(mode=2))
    gs.check()
    assert float(g1.abs().max()) > 0.0
    torch.testing.assert_close(g1, g2, rtol=1e-5, atol=1e-6 * float(g1.abs().max()))


def _tlas_check(api, boxes, builder):
    import ctypes as C
    N = api.N
    b = np.ascontiguousarray(boxes, dtype=np.float32)
    o = N.qrt_build_opts()
    o.tlas_builder = builder
    n, d = C.c_uint64(), C.c_uint32()
    rc = N.lib().qrt_tlas_build_check(b.ctypes.data, b.shape[0], C.byref(o), C.byref(n), C.byref(d))
    return rc, n.value, d.value, N.lib().qrt_last_error().decode()


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 300000])
def test_linear_tlas_on_device(api, n):
    """The linear-BVH TLAS built on the device passes the invariant check and
    has the shape of the same steps run on the host (same Morton order and
    radix tree; only the numbering of the wide nodes may differ)."""
    rng = np.random.default_rng(n)
    c = rng.uniform(-100, 100, size=(n, 3))
    e = rng.uniform(0.1, 5, size=(n, 3))
    boxes = np.concatenate([c - e, c + e], axis=1)
    rc, nodes, depth, msg = _tlas_check(api, boxes, 1)
    assert rc == 0, msg
    rc2, nodes2, depth2, msg2 = _tlas_check(api, boxes, 2)
    assert rc2 == 0, msg2
    assert (nodes, depth) == (nodes2, depth2)
    same = np.tile(np.array([[0, 0, 0, 1, 1, 1]], np.float32), (max(n, 2), 1))
    assert _tlas_check(api, same, 1)[0] == 0


def test_linear_blas_on_device(api):
    """Every mesh's linear BVH built on the device in one pass passes the
    invariant check and has the shape of the same steps run on the host."""
    import ctypes as C
    N = api.N
    rng = np.random.default_rng(3)
    meshes = [I.tiny_mesh(), I.displaced_grid(rng, 5000), I.noisy_blob(rng, 3000),
              I.sphere_mesh(10, 20), I.plane_mesh(1), I.plane_mesh(3), I.displaced_grid(rng, 65536)]
    vv = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    meshes.append((vv, np.tile(np.array([[0, 1, 2, 3]], dtype=np.uint32), (50, 1))))
    arr = (N.qrt_mesh * len(meshes))()
    keep = []
    for k, (v, q) in enumerate(meshes):
        v = np.ascontiguousarray(v, dtype=np.float32)
        q = np.ascontiguousarray(q, dtype=np.uint32)
        keep += [v, q]
        arr[k].verts = v.ctypes.data_as(C.POINTER(C.c_float))
        arr[k].n_verts = v.shape[0]
        arr[k].quads = q.ctypes.data_as(C.POINTER(C.c_uint32))
        arr[k].n_quads = q.shape[0]
    res = []
    for builder in (1, 2):
        o = N.qrt_build_opts()
        o.blas_builder = builder
        n, d = C.c_uint64(), C.c_uint32()
        rc = N.lib().qrt_blases_build_check(arr, len(meshes), C.byref(o), C.byref(n), C.byref(d))
        assert rc == 0, N.lib().qrt_last_error().decode()
        res.append((n.value, d.value))
    assert res[0] == res[1]


def test_device_built_tlas_matches_oracle(api, tiny):
    """A scene whose TLAS and BLAS come from the device's linear-BVH builds: ray
    queries match the oracle as the SAH-built scene's do, and renders agree
    with it."""
    sc, gs, osc = tiny
    g2 = api.Scene(sc, build_opts=dict(tlas_builder=1, blas_builder=1))
    rays = _rays(sc)
    d = torch.from_numpy(rays).cuda()
    h = g2.trace_closest(d).cpu().numpy().view(np.uint32)
    bits = g2.trace_any(d).cpu().numpy().view(np.uint32)
    g2.check()
    o_t, o_i, o_p, _, _ = osc.trace_closest(rays)
    n, acc, bad = classify_closest(sc, rays, h[:, 1], h[:, 2], o_t, o_i, o_p)
    assert not bad, f"{len(bad)} unexplained mismatches, e.g. ray {bad[:5]}"
    assert acc / len(rays) < 1e-5
    occ = ((bits[np.arange(len(rays)) // 32] >> (np.arange(len(rays)) % 32)) & 1).astype(bool)
    assert (occ != (o_i != NONE)).sum() <= acc
    h0 = gs.trace_closest(d).cpu().numpy().view(np.uint32)
    assert (h0[:, 1:3] != h[:, 1:3]).any(axis=1).mean() < 1e-5
    view = I.tiny_view()
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    a = gs.render([view], alb, params)[0]
    b = g2.render([view], alb, params)[0]
    g2.check()
    assert (a != b).any(dim=-1).float().mean().item() < 1e-3
    assert g2.stats["tlas_nodes"] > 0 and g2.stats["tlas_depth"] > 0


def test_autotuner_choice_is_valid_and_changes_no_pixel(api, tiny, tmp_path):
    from paper_2001_02620_gb300 import autotune
    sc, gs, osc = tiny
    view = I.tiny_view()
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    space = {"block": [64, 128], "stack": [32, 64], "occupancy": [24, 40], "batch": [1, 4]}
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(gs, view, alb, params, space=space, reps=1, cache_path=cache,
                         scene_name="tiny")
    assert set(best) == set(space) and all(best[k] in space[k] for k in space)
    assert autotune.tune(gs, view, alb, params, space=space, cache_path=cache,
                         scene_name="tiny") == best  # served from the cache
    ref = gs.render([view], alb, params)[0]
    for cand in autotune.candidates(space):
        assert torch.equal(gs.render([view], alb, params, tuning=cand)[0], ref)
    gs.check()


def test_autotuner_times_finalists_on_the_whole_view(api, tiny, tmp_path):
    """With a proxy smaller than the view, the fastest proxy candidates are
    timed again on the view itself and the winner is one of them."""
    import json

    from paper_2001_02620_gb300 import autotune
    sc, gs, osc = tiny
    view = I.tiny_view()
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    space = {"block": [64, 128, 256], "stack": [64], "occupancy": [32, 40], "batch": [1]}
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(gs, view, alb, I.tiny_params(), space=space, reps=1, cache_path=cache,
                         scene_name="tiny", finalists=3, proxy_paths=1 << 12)
    (entry,) = autotune.load_cache(cache).values()
    finals = entry["whole_view_finalists"]
    assert len(finals) == 3 and all(v is not None for v in finals.values())
    assert json.dumps(best, sort_keys=True) in finals
    assert finals[json.dumps(best, sort_keys=True)] == min(finals.values())
    assert entry["proxy"][0] * entry["proxy"][1] * view.spp <= 1 << 12
    gs.check()


def test_white_furnace_gpu(api):
    v, q = I.sphere_mesh(24, 48, 5.0)
    sc = I.Scene([(v, q)], I.IDENTITY_XFORM[None].copy(), np.zeros(1, dtype=np.uint32))
    gs = api.Scene(sc)
    view = I.View(eye=(0.0, -30.0, 4.0), look=(0.0, 0.0, 0.0), up=(0, 0, 1), vfov_deg=30.0,
                  w=96, h=64, spp=4)
    ones = torch.ones((sc.n_quads, 3), device="cuda")
    (img,) = gs.render([view], ones, I.Params(max_depth=256, env=(1.0, 1.0, 1.0)))
    gs.check()
    assert torch.all(img == 1.0)


def test_batched_equals_plain_bit_exact(api, tiny):
    sc, gs, osc = tiny
    views = I.batched_views(n_views=7, min_log2=5.0, max_log2=8.0, max_spp=4)
    for v in views:
        v.eye = (50.0 + (v.eye[0] - 2048.0) / 40, -120.0, 50.0)
        v.look = (50.0, 50.0, 50.0)
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    batched = gs.render(views, alb, params, tuning=dict(batch=2))
    plain = [gs.render([v], alb, params)[0] for v in views]
    graph = api.RenderGraph(gs, views, alb, params)
    g1 = [x.clone() for x in graph.launch()]
    g2 = graph.launch()
    gs.check()
    for b, p, x, y in zip(batched, plain, g1, g2):
        assert torch.equal(b, p)
        assert torch.equal(b, x)
        assert torch.equal(b, y)


def test_many_views_split_across_launches(api, tiny):
    sc, gs, osc = tiny
    views = []
    for k in range(70):   # more views than one launch holds
        views.append(I.View(eye=(50.0, -120.0 + k, 50.0), look=(50, 50, 50), up=(0, 0, 1),
                            vfov_deg=40.0, w=16, h=8 + k % 3, spp=1, pixel_base=1000 * k))
    params = I.tiny_params()
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    out = gs.render(views, alb, params)
    gs.check()
    for k in (0, 63, 64, 69):
        (one,) = gs.render([views[k]], alb, params)
        assert torch.equal(one, out[k])


@pytest.mark.parametrize("mode", [2, 1])
def test_crops_equal_whole_frame(api, tiny, mode):
    """A crop renders exactly the same pixels as the whole frame (the
    camera and random streams are the frame's), for ragged tiles at the
    frame's edges, many crops in one call, and the path and ray logs."""
    import dataclasses
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp, view.pixel_base = 150, 70, 3, 12345
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 2.0, 1.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    D = params.max_depth
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    rlog = torch.zeros(api.ray_log_floats([view], D), dtype=torch.float32, device="cuda")
    (full,) = gs.render([view], alb, params, path_log=log, ray_log=rlog, tuning=dict(mode=mode))
    tiles = [(0, 0, 32, 32), (128, 64, 22, 6), (37, 5, 1, 1), (0, 50, 150, 20), (149, 0, 1, 70)]
    crops = [dataclasses.replace(view, crop_x=x, crop_y=y, crop_w=w, crop_h=h) for x, y, w, h in tiles]
    clog = torch.zeros(api.path_log_words(crops, D), dtype=torch.int32, device="cuda")
    crl = torch.zeros(api.ray_log_floats(crops, D), dtype=torch.float32, device="cuda")
    outs = gs.render(crops, alb, params, path_log=clog, ray_log=crl, tuning=dict(mode=mode))
    gs.check()
    flog = log.view(view.h, view.w, view.spp, 2 * D + 2)
    frl = rlog.view(view.h, view.w, view.spp, D, 16)
    p0 = 0
    for (x, y, w, h), out in zip(tiles, outs):
        assert out.shape == (h, w, 3)
        assert torch.equal(out, full[y:y + h, x:x + w])
        n = w * h * view.spp
        assert torch.equal(clog.view(-1, 2 * D + 2)[p0:p0 + n].view(h, w, view.spp, -1),
                           flog[y:y + h, x:x + w])
        assert torch.equal(crl.view(-1, D, 16)[p0:p0 + n].view(h, w, view.spp, D, 16),
                           frl[y:y + h, x:x + w])
        p0 += n


@pytest.mark.parametrize("world", [2, 3])
def test_image_parallel_ranks_through_the_library(api, tiny, world):
    """The image-parallel renderer with `world` ranks emulated in one process
    (each rank's round-robin tiles rendered as crops through libqrt.so and
    packed, then unpacked as rank 0 would after the gather): the frame is
    bit-identical to a one-call render, and the ranks' tile gradients sum to
    the whole frame's adjoint (up to the order of the FP32 atomics)."""
    from paper_2001_02620_gb300 import shard
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp = 150, 70, 2
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    (full,) = gs.render([view], alb, params)
    render = shard.scene_renderer(gs, alb, params)
    parts = [shard.render_tiles(render, view, r, world, tile=32) for r in range(world)]
    frame = shard.gather_frame(None, view, 32, parts=parts)
    assert torch.equal(frame, full)
    dimg = torch.from_numpy(np.random.default_rng(5).normal(size=(view.h, view.w, 3))
                            .astype(np.float32)).cuda()
    ref = torch.zeros_like(alb)
    gs.adjoint([view], alb, [dimg], ref, params)
    total = torch.zeros_like(alb)
    adj = shard.scene_adjoint(gs, alb, params)
    for r in range(world):
        g = torch.zeros_like(alb)
        shard.adjoint_frame(adj, view, dimg, g, r, world, tile=32)
        total += g
    gs.check()
    torch.testing.assert_close(total, ref, rtol=1e-4, atol=1e-6 * float(ref.abs().max()))


def test_crop_rejects_rectangles_outside_the_frame(api, tiny):
    import dataclasses
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h = 64, 48
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    for x, y, w, h in ((60, 0, 8, 8), (0, 40, 8, 9), (0, 0, 0, 4), (0, 0, 4, 0), (2**31, 0, 2**31, 1)):
        bad = dataclasses.replace(view, crop_x=x, crop_y=y, crop_w=w, crop_h=h)
        with pytest.raises(api.N.QrtError) as e:
            gs.render([bad], alb, I.tiny_params(), outs=[torch.empty((max(h, 1), max(w, 1), 3),
                                                                     device="cuda")])
        assert e.value.code == api.N.QRT_ERR_INVALID_ARG


def test_spp_above_the_chunk_is_rejected(api, tiny):
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp = 8, 8, 2048
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    with pytest.raises(api.N.QrtError) as e:
        gs.render([view], alb, I.tiny_params(), tuning=dict(mode=2, chunk_log2=10))
    assert e.value.code == api.N.QRT_ERR_INVALID_ARG and "spp 2048" in str(e.value)


def test_adjoint_matches_oracle_gradient(api, tiny):
    sc, gs, osc = tiny
    view, params = I.tiny_view(), I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3, 3, 3))
    view.spp = 2
    alb = I.albedo(sc.n_quads)
    D = params.max_depth
    dimg = np.random.default_rng(8).normal(size=(view.h, view.w, 3)).astype(np.float32)
    d_alb = torch.from_numpy(alb).cuda()
    grad = torch.zeros_like(d_alb)
    gs.adjoint([view], d_alb, [torch.from_numpy(dimg).cuda()], grad, params)
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    gs.render([view], d_alb, params, path_log=log)
    gs.check()
    g = grad.double().cpu().numpy()
    ref = osc.render(view, alb, params, log=True)
    og = osc.grad(view, alb, params, dimg.reshape(-1, 3).astype(np.float64))
    agree = path_agreement(log.cpu().numpy().view(np.uint32), ref, D)
    # quads touched by a divergent path (either side) are excluded and counted
    gl = log.cpu().numpy().view(np.uint32).reshape(-1, 2 * D + 2)
    offs = sc.quad_offsets
    touched = set()
    for k in np.nonzero(~agree)[0]:
        for inst, prim in list(zip(ref["inst"][k], ref["prim"][k])) + list(zip(gl[k, 0:2 * D:2], gl[k, 1:2 * D:2])):
            if inst != NONE:
                touched.add(int(offs[sc.mesh_ids[inst]] + prim))
    mask = np.ones(sc.n_quads, dtype=bool)
    mask[list(touched)] = False
    big = np.abs(og).max()
    sel = mask[:, None] & (np.abs(og) > 1e-6 * big)
    assert sel.sum() > 1000
    rel = np.abs(g[sel] - og[sel]) / np.abs(og[sel])
    assert rel.max() < 1e-4, (rel.max(), len(touched))
    assert (~agree).mean() < 0.01


def _touched_quads(sc, glog, ref, agree, D):
    """Albedo rows on any path (either side's) that did not agree."""
    offs = sc.quad_offsets
    touched = set()
    for k in np.nonzero(~agree)[0]:
        for inst, prim in list(zip(ref["inst"][k], ref["prim"][k])) + \
                list(zip(glog[k, 0:2 * D:2], glog[k, 1:2 * D:2])):
            if inst != NONE:
                touched.add(int(offs[sc.mesh_ids[inst]] + prim))
    return touched


def test_render_fn_autograd(api, tiny):
    """The adjoint behind torch.autograd.Function: loss = mean((render(albedo)
    - target)^2) with render = api.RenderFn; loss.backward() fills
    albedo.grad with the replay adjoint of the loss's image gradient, which
    equals Scene.adjoint given that gradient (up to the order of the FP32
    atomics) and the FP64 oracle gradient within 1e-4 on quads whose paths
    agree with the oracle's."""
    sc, gs, osc = tiny
    view, params = I.tiny_view(), I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3, 3, 3))
    view.spp = 2
    D = params.max_depth
    a0 = I.albedo(sc.n_quads)
    (target,) = gs.render([view], torch.from_numpy(I.perturbed_albedo(a0)).cuda(), params)
    alb = torch.from_numpy(a0).cuda().requires_grad_(True)
    img = api.render_differentiable(alb, gs, view, params)
    assert img.requires_grad and img.shape == (view.h, view.w, 3)
    loss = ((img - target) ** 2).mean()
    (dimg,) = torch.autograd.grad(loss, img, retain_graph=True)
    loss.backward()
    gs.check()
    assert alb.grad is not None and alb.grad.shape == alb.shape
    direct = torch.zeros_like(alb)
    gs.adjoint([view], alb.detach(), [dimg.contiguous()], direct, params)
    gs.check()
    torch.testing.assert_close(alb.grad, direct, rtol=1e-5, atol=1e-9)
    # against the oracle's stored-path gradient of the same image gradient
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    gs.render([view], alb.detach(), params, path_log=log)
    ref = osc.render(view, a0, params, log=True)
    og = osc.grad(view, a0, params, dimg.double().cpu().numpy().reshape(-1, 3))
    glog = log.cpu().numpy().view(np.uint32).reshape(-1, 2 * D + 2)
    agree = path_agreement(glog, ref, D)
    mask = np.ones(sc.n_quads, dtype=bool)
    mask[list(_touched_quads(sc, glog, ref, agree, D))] = False
    g = alb.grad.double().cpu().numpy()
    sel = mask[:, None] & (np.abs(og) > 1e-6 * np.abs(og).max())
    assert sel.sum() > 1000
    rel = np.abs(g[sel] - og[sel]) / np.abs(og[sel])
    assert rel.max() < 1e-4, rel.max()


def test_adjoint_with_textures_and_key_lights_matches_oracle_gradient(api, tiny):
    """The replay adjoint with per-face textures and key lights (light
    shadow rays traced again in the replay) against the oracle's stored-path
    gradient, on quads whose paths agree, for both renderers.  The textures
    are constant over each face (a random factor per face): the gradient
    then does not depend on where a ray hits a face, which FP32 rays fix
    only to within their rounding (the render tests bound that effect)."""
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w, view.h, view.spp = 128, 96, 2
    k = np.random.default_rng(63).uniform(0.4, 1.0, size=(sc.n_quads, 1, 1, 3)).astype(np.float32)
    tex = np.ascontiguousarray(np.broadcast_to(k, (sc.n_quads, 4, 4, 3)))
    params = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(2, 2, 2), tex=tex, lights=I.tiny_lights())
    gparams = dataclasses.replace(params, tex=torch.from_numpy(tex).cuda())
    alb = I.albedo(sc.n_quads)
    D = params.max_depth
    dimg = np.random.default_rng(9).normal(size=(view.h, view.w, 3)).astype(np.float32)
    d_alb = torch.from_numpy(alb).cuda()
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    gs.render([view], d_alb, gparams, path_log=log)
    ref = osc.render(view, alb, params, log=True)
    og = osc.grad(view, alb, params, dimg.reshape(-1, 3).astype(np.float64))
    glog = log.cpu().numpy().view(np.uint32).reshape(-1, 2 * D + 2)
    agree = path_agreement(glog, ref, D)
    mask = np.ones(sc.n_quads, dtype=bool)
    mask[list(_touched_quads(sc, glog, ref, agree, D))] = False
    sel = mask[:, None] & (np.abs(og) > 1e-6 * np.abs(og).max())
    assert sel.sum() > 1000
    # every path term of the gradient is positive times the pixel's dimage
    # entry, so the oracle gradient of |dimage| is the sum of the terms'
    # magnitudes: FP32 rounding of each term bounds the error by a multiple
    # of it, however much the signed terms cancel
    mag = osc.grad(view, alb, params, np.abs(dimg).reshape(-1, 3).astype(np.float64))
    for mode in (2, 1):
        grad = torch.zeros_like(d_alb)
        gs.adjoint([view], d_alb, [torch.from_numpy(dimg).cuda()], grad, gparams, tuning=dict(mode=mode))
        gs.check()
        g = grad.double().cpu().numpy()
        rel = np.abs(g[sel] - og[sel]) / mag[sel]
        assert rel.max() < 1e-4, (mode, rel.max())
        # and against the signed value where the terms do not cancel much
        keep = np.abs(og[sel]) > 0.1 * mag[sel]
        assert keep.sum() > 500
        assert (np.abs(g[sel] - og[sel])[keep] / np.abs(og[sel])[keep]).max() < 1e-4


def test_l2_loss(api):
    rng = np.random.default_rng(1)
    a = rng.uniform(size=(37, 53, 3)).astype(np.float32)
    b = rng.uniform(size=(37, 53, 3)).astype(np.float32)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dimg = torch.empty_like(da)
    loss = api.l2_loss(da, db, dimg)
    ref = ((a.astype(np.float64) - b) ** 2).mean()
    assert abs(float(loss) - ref) < 1e-12 * max(1.0, ref)
    np.testing.assert_allclose(dimg.cpu().numpy(), 2 * (a.astype(np.float64) - b) / a.size, rtol=1e-6)


def test_read_bandwidth_helper(api):
    """The L2 read-bandwidth helper: argument checks, and a sweep of an
    L2-resident buffer reads faster than any HBM copy could."""
    import ctypes as C
    L = api.N.lib()
    buf = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.qrt_read_bandwidth(buf.data_ptr(), 0, 3, sink.data_ptr(), s) == api.N.QRT_OK
    assert L.qrt_read_bandwidth(buf.data_ptr() + 4, 1024, 1, sink.data_ptr(), s) == api.N.QRT_ERR_ALIGN
    assert L.qrt_read_bandwidth(buf.data_ptr(), 1000, 1, sink.data_ptr(), s) == api.N.QRT_ERR_ALIGN
    assert L.qrt_read_bandwidth(None, 1024, 1, sink.data_ptr(), s) == api.N.QRT_ERR_INVALID_ARG
    # all-zero data folds to zero
    api.N.check(L.qrt_read_bandwidth(buf.data_ptr(), buf.numel() * 4, 2, sink.data_ptr(), s))
    assert int(sink.item()) == 0
    gbs = api.read_bandwidth_gbs(32 << 20, 20)
    assert 8000.0 < gbs < 200000.0


def test_stack_overflow_is_reported(api):
    """A chain-shaped BLAS over coincident quads needs about three stack
    entries per level: a 32-entry stack overflows, the kernel stops that ray
    and raises the error word; the context stays usable."""
    vv = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    q = np.tile(np.array([[0, 1, 2, 3]], dtype=np.uint32), (300, 1))
    sc = I.Scene([(vv, q)], I.IDENTITY_XFORM[None].copy(), np.zeros(1, dtype=np.uint32))
    gs = api.Scene(sc, build_opts=dict(degenerate=1))
    rays = torch.from_numpy(I.ray_array(np.array([[0.5, 0.5, 5.0]]), np.array([[0.0, 0.0, -1.0]]))).cuda()
    gs.trace_closest(rays, tuning=dict(stack=32))
    with pytest.raises(api.N.QrtError) as e:
        gs.check()
    assert e.value.code == api.N.QRT_ERR_STACK_OVERFLOW
    gs.check()   # cleared after reading
    # a normal scene still traces afterwards
    sc2 = I.tiny_scene()
    gs2 = api.Scene(sc2)
    gs2.trace_closest(torch.from_numpy(_rays(sc2)[:1000]).cuda())
    gs2.check()


def test_step_limit_is_reported(api, tiny):
    sc, gs, osc = tiny
    view = I.tiny_view()
    view.w = view.h = 32
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    gs.render([view], alb, I.tiny_params(), max_steps=2)
    with pytest.raises(api.N.QrtError) as e:
        gs.check()
    assert e.value.code == api.N.QRT_ERR_STEP_LIMIT
    gs.render([view], alb, I.tiny_params())
    gs.check()


def test_invalid_arguments_rejected(api, tiny):
    sc, gs, osc = tiny
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    view = I.tiny_view()
    with pytest.raises(api.N.QrtError):
        gs.render([view], alb, I.Params(max_depth=0))
    with pytest.raises(api.N.QrtError):
        gs.render([view], alb, I.tiny_params(), tuning=dict(stack=48))
    bad = I.View(eye=(0, 0, 0), look=(0, 0, 0), up=(0, 0, 1), vfov_deg=40, w=8, h=8, spp=1)
    with pytest.raises(api.N.QrtError):
        gs.render([bad], alb, I.tiny_params())
    buf = torch.zeros(40 * 8 + 1, device="cuda")
    with pytest.raises(api.N.QrtError) as e:
        gs.trace_closest(buf[1:].view(40, 8))   # 4-byte offset: not 16-byte aligned
    assert e.value.code == api.N.QRT_ERR_ALIGN


def test_scene_without_instances(api):
    v, q = I.plane_mesh(2)
    sc = I.Scene([(v, q)], np.zeros((0, 12), dtype=np.float32), np.zeros(0, dtype=np.uint32))
    gs = api.Scene(sc)
    rays = torch.from_numpy(I.rays_random(100, [-1, -1, -1], [1, 1, 1], seed=1)).cuda()
    h = gs.trace_closest(rays).cpu().numpy().view(np.uint32)
    assert (h[:, 1] == NONE).all()
    view = I.View(eye=(0, -5, 0), look=(0, 0, 0), up=(0, 0, 1), vfov_deg=40, w=8, h=8, spp=1)
    (img,) = gs.render([view], torch.ones((sc.n_quads, 3), device="cuda"),
                       I.Params(max_depth=2, env=(0.25, 0.5, 1.0)))
    gs.check()
    assert torch.all(img == torch.tensor([0.25, 0.5, 1.0], device="cuda"))
