"""Moana-scale workload on the GPU: the same generator as the full 261 M-quad
benchmark at a reduced scale (QRT_MOANA_SCALE, default 0.02: 5.2 M unique
quads, 786 k clustered instances, 1.6 G instanced quads), rendered at the
full workload's launch configuration (1920x1080, 16 spp, depth 8), with
sampled pixels checked against the oracle."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2001_02620_gb300 import inputs as I

from parity import NONE, classify_closest, path_agreement

pytestmark = pytest.mark.gpu

SCALE = float(os.environ.get("QRT_MOANA_SCALE", "0.02"))


@pytest.fixture(scope="module")
def moana():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_02620_gb300 import build as B
    B.build()
    from paper_2001_02620_gb300 import api
    sc = I.moana_scene(SCALE)
    return api, sc, api.Scene(sc), O.OracleScene(sc)


def test_moana_statistics_follow_the_paper(moana):
    api, sc, gs, osc = moana
    n, c, terrain = I.moana_sizes(SCALE)
    assert abs(sc.n_quads - I.MOANA_QUADS * SCALE) < 2e-3 * I.MOANA_QUADS * SCALE
    n_tiles = sc.meta["terrain_meshes"][1]
    assert abs(len(sc.xforms) - n_tiles - I.MOANA_INSTANCES * SCALE) < 1e-3 * I.MOANA_INSTANCES * SCALE
    assert abs(sc.meta["instanced_quads"] - I.MOANA_INSTANCED_QUADS * SCALE) < 2e-2 * I.MOANA_INSTANCED_QUADS * SCALE
    assert gs.stats["n_quads"] == sc.n_quads


def test_moana_render_sampled_pixels(moana):
    api, sc, gs, osc = moana
    view, params = I.moana_view(sc.meta["extent"]), I.moana_params()
    alb = I.albedo(sc.n_quads)
    D = params.max_depth
    log = torch.zeros(api.path_log_words([view], D), dtype=torch.int32, device="cuda")
    (img,) = gs.render([view], torch.from_numpy(alb).cuda(), params, path_log=log)
    gs.check()
    px = np.sort(np.random.default_rng(23).choice(view.w * view.h, size=256, replace=False))
    ref = osc.render(view, alb, params, pixels=px, log=True)
    glog = log.view(-1, 2 * D + 1).reshape(view.w * view.h, view.spp, 2 * D + 1)
    glog = glog[torch.from_numpy(px).cuda()].reshape(-1, 2 * D + 1).cpu().numpy().view(np.uint32)
    agree = path_agreement(glog, ref, D)
    pix_ok = agree.reshape(-1, view.spp).all(1)
    g = img.reshape(-1, 3)[torch.from_numpy(px).cuda()].double().cpu().numpy()
    r = ref["rgb"]
    err = np.abs(g[pix_ok] - r[pix_ok])
    assert pix_ok.mean() > 0.9, f"divergent pixels {1 - pix_ok.mean():.3f}"
    assert (err <= 1e-4 * np.abs(r[pix_ok]) + 1e-6).all(), err.max()


def test_moana_trace_parity(moana):
    api, sc, gs, osc = moana
    ext = sc.meta["extent"]
    lo, hi = np.array([0.0, 0.0, -150.0]), np.array([ext, ext, 250.0])
    rays = np.concatenate([I.rays_focused(65536, I.moana_view(ext).eye, lo, hi, seed=61),
                           I.rays_random(65536, lo, hi, seed=62),
                           I.rays_toward(65536, lo, hi, I.instance_origins(sc), 2.0, seed=63)])
    h = gs.trace_closest(torch.from_numpy(rays).cuda()).cpu().numpy().view(np.uint32)
    gs.check()
    o_t, o_i, o_p, _, _ = osc.trace_closest(rays)
    n, acc, bad = classify_closest(sc, rays, h[:, 1], h[:, 2], o_t, o_i, o_p)
    assert not bad, bad[:5]
    assert acc / len(rays) < 1e-5
