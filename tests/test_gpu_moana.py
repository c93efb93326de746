"""Moana-scale workload on the GPU: the same generator as the full 261 M-quad
benchmark at a reduced scale (QRT_MOANA_SCALE, default 0.1: 26.1 M unique
quads, 3.93 M clustered instances, 8.2 G instanced quads), rendered at the
full workload's launch configuration (1920x1080, 16 spp, depth 8), with
sampled pixels checked against the oracle, and ray queries (primary,
instance-aimed, random, and rays dumped from a render) against it."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2001_02620_gb300 import inputs as I

from parity import NONE, classify_closest, rays_from_render, render_parity, report_line

pytestmark = pytest.mark.gpu

SCALE = float(os.environ.get("QRT_MOANA_SCALE", "0.1"))


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
    """The full workload's launch (1920x1080, 16 spp, depth 8) on 4096
    sampled pixels: every divergent path explained where it first diverges,
    agreeing paths within 1e-4 of the oracle's radiance."""
    api, sc, gs, osc = moana
    view, params = I.moana_view(sc.meta["extent"]), I.moana_params()
    alb = I.albedo(sc.n_quads)
    px = np.sort(np.random.default_rng(23).choice(view.w * view.h, size=4096, replace=False))
    pix_ok, err, r, rep = render_parity(api, gs, osc, sc, view, alb, params, pixels=px)
    print(report_line(f"moana x{SCALE} 1920x1080 16 spp depth 8", rep))
    print(f"moana x{SCALE}: TLAS depth {gs.stats['tlas_depth']}, deepest BLAS {gs.stats['max_blas_depth']}")
    assert not rep["unexplained"], rep["unexplained"][:8]
    assert rep["near_tie"] <= max(1, 1e-5 * rep["rays"]), report_line("moana", rep)
    # measured 1.7e-3 at scale 0.1 (113 of 65536 paths); the bound allows 3x that
    assert rep["divergent_path_frac"] < 5e-3, report_line("moana", rep)
    assert (err <= 1e-4 * np.abs(r) + 1e-6).all(), err.max()


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


def test_moana_dumped_rays_parity(moana):
    """Ray queries on rays dumped from a render of the workload's camera
    (camera rays, first diffuse bounces, shadow rays): closest and any hit
    against the oracle on a sample of each set."""
    api, sc, gs, osc = moana
    view, params = I.moana_view(sc.meta["extent"], w=480, h=270, spp=1), I.moana_params()
    alb = torch.from_numpy(I.albedo(sc.n_quads)).cuda()
    sets = rays_from_render(api, gs, view, alb, params)
    rng = np.random.default_rng(29)
    for name, rays in sets.items():
        assert len(rays) > 10000, name
        rays = rays[np.sort(rng.choice(len(rays), size=min(len(rays), 65536), replace=False))]
        d = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
        h = gs.trace_closest(d).cpu().numpy().view(np.uint32)
        bits = gs.trace_any(d).cpu().numpy().view(np.uint32)
        gs.check()
        o_t, o_i, o_p, _, _ = osc.trace_closest(rays)
        n, acc, bad = classify_closest(sc, rays, h[:, 1], h[:, 2], o_t, o_i, o_p)
        assert not bad, (name, bad[:5])
        assert acc <= max(1, 1e-5 * len(rays)), (name, acc)
        occ = ((bits[np.arange(len(rays)) // 32] >> (np.arange(len(rays)) % 32)) & 1).astype(bool)
        o_occ = osc.trace_any(rays)
        diff = np.nonzero(occ != o_occ)[0]
        # an any-hit disagreement must be a closest-hit near-tie as well
        assert all(k in set(np.nonzero((h[:, 1] != o_i) | (h[:, 2] != o_p))[0]) for k in diff), name


@pytest.fixture(scope="module")
def moana_full():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_02620_gb300 import api
    sc = I.moana_scene(1.0)
    return api, sc


def test_moana_full_scale_sampled_pixels(moana_full):
    """The benchmark's own workload and launch configuration at full size
    (261.1 M unique quads, 39.3 M instances, 1920x1080, 16 spp, depth 8,
    library defaults) on 1024 sampled pixels against the full-scale oracle:
    every divergent path explained, agreeing paths within 1e-4."""
    import gc
    api, sc = moana_full
    gs = api.Scene(sc)
    osc = O.OracleScene(sc)
    view, params = I.moana_view(sc.meta["extent"]), I.moana_params()
    alb = I.albedo(sc.n_quads)
    px = np.sort(np.random.default_rng(31).choice(view.w * view.h, size=1024, replace=False))
    pix_ok, err, r, rep = render_parity(api, gs, osc, sc, view, alb, params, pixels=px)
    print(report_line("moana x1.0 1920x1080 16 spp depth 8", rep))
    print(f"moana x1.0: TLAS depth {gs.stats['tlas_depth']}, deepest BLAS {gs.stats['max_blas_depth']}")
    assert gs.stats["n_quads"] == sc.n_quads and gs.stats["n_instances"] == len(sc.xforms)
    assert not rep["unexplained"], rep["unexplained"][:8]
    assert rep["near_tie"] <= max(1, 1e-5 * rep["rays"]), report_line("moana full", rep)
    assert rep["divergent_path_frac"] < 5e-3, report_line("moana full", rep)
    assert (err <= 1e-4 * np.abs(r) + 1e-6).all(), err.max()
    gs.close()
    del osc, gs
    gc.collect()
