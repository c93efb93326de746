"""qrt_render_spp_static: the render entry point for callers that cannot
allocate device memory (frame loops that must not stall on cudaMalloc,
processes whose device memory belongs to another allocator).  It renders
with scratch held in a fixed array inside the library, so this test calls it
through the C ABI and checks that it gives exactly the images of
qrt_render_spp (the wavefront renderer is bit-reproducible across chunk
sizes), twice in a row (the array keeps the previous call's contents, which
must not leak into the next result), and that a call leaves the device's
free memory unchanged."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_02620_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_02620_gb300 import build as B
    B.build()
    from paper_2001_02620_gb300 import _native as N
    from paper_2001_02620_gb300 import api
    return N, api


def _call_static(N, api, scene, views, alb, params, tuning=None, outs=None):
    if outs is None:
        outs = [torch.full((v.h, v.w, 3), float("nan"), device="cuda") for v in views]
    cv = api.make_views(views, outs)
    cp = api.make_params(params, tuning)
    rc = N.lib().qrt_render_spp_static(scene.handle, cv, len(views), alb.data_ptr(), C.byref(cp),
                                       torch.cuda.current_stream().cuda_stream)
    return rc, outs


def test_static_render_matches_render_spp(lib_api):
    N, api = lib_api
    sc = I.tiny_scene()
    scene = api.Scene(sc)
    # several chunks of 2^17 paths, uneven views, sun and shadow rays
    views = [I.View(eye=(50.0, -120.0, 50.0), look=(50.0, 50.0, 50.0), up=(0.0, 0.0, 1.0),
                    vfov_deg=40.0, w=300, h=170, spp=3, pixel_base=0),
             I.View(eye=(40.0, -110.0, 60.0), look=(50.0, 50.0, 40.0), up=(0.0, 0.0, 1.0),
                    vfov_deg=50.0, w=97, h=61, spp=5, pixel_base=300 * 170)]
    params = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 2.0, 1.0))
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    ref = scene.render(views, alb, params)
    torch.cuda.synchronize()
    for k in range(2):
        outs = [torch.full((v.h, v.w, 3), float("nan"), device="cuda") for v in views]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc, outs = _call_static(N, api, scene, views, alb, params, outs=outs)
        N.check(rc)
        scene.check()
        torch.cuda.synchronize()
        if k == 1:  # the first call may still load kernel code; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
    scene.close()


def test_static_render_rejects_oversized_chunk(lib_api):
    N, api = lib_api
    sc = I.tiny_scene(n_inst=8)
    scene = api.Scene(sc)
    view = I.tiny_view()
    view.w = view.h = 16
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    rc, _ = _call_static(N, api, scene, [view], alb, I.tiny_params(), tuning=dict(chunk_log2=18))
    assert rc == N.QRT_ERR_INVALID_ARG
    assert b"static workspace" in N.lib().qrt_last_error()
    rc, _ = _call_static(N, api, scene, [view], alb, I.tiny_params(), tuning=dict(mode=1))
    assert rc == N.QRT_ERR_INVALID_ARG
    # a pixel's samples must fit one chunk of the static workspace
    one = I.tiny_view()
    one.w, one.h, one.spp = 1, 1, (1 << 17) + 1
    rc, _ = _call_static(N, api, scene, [one], alb, I.tiny_params())
    assert rc == N.QRT_ERR_INVALID_ARG
    assert b"spp 131073" in N.lib().qrt_last_error()
    scene.close()
