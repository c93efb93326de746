"""Multi-rank logic on CPU: the image-parallel renderer (round-robin tiles as
crop views, the tensor gather to rank 0, the gradient all-reduce) with two
gloo ranks and the oracle standing in for the GPU scene; plus the
autotuner's host-side logic (candidate space, stack-depth bound, cache,
selection)."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2001_02620_gb300 import autotune, shard
from paper_2001_02620_gb300 import inputs as I


def test_tiles_cover_image_once():
    for w, h, t in [(64, 64, 32), (200, 120, 32), (33, 7, 16), (1, 1, 32)]:
        boxes = shard.tiles(w, h, t)
        seen = np.zeros(w * h, dtype=int)
        for world in (1, 2, 3):
            seen[:] = 0
            for r in range(world):
                px = shard.pixels_of_tiles(w, boxes, shard.tiles_of_rank(len(boxes), r, world))
                seen[px] += 1
            assert (seen == 1).all()


def test_round_robin_assignment():
    assert shard.tiles_of_rank(7, 0, 3) == [0, 3, 6]
    assert shard.tiles_of_rank(7, 2, 3) == [2, 5]
    with pytest.raises(ValueError):
        shard.tiles_of_rank(7, 3, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle_fns(osc, alb, params):
    """render_fn / adjoint_fn of the image-parallel renderer with the oracle
    standing in for the GPU scene (crops rendered as frame-pixel subsets)."""
    import torch

    def crop_pixels(v):
        return shard.pixels_of_tiles(v.w, [(v.crop_x, v.crop_y, v.crop_x + v.crop_w,
                                            v.crop_y + v.crop_h)], [0])

    def render(views):
        return [torch.from_numpy(osc.render(v, alb, params, pixels=crop_pixels(v), nthreads=2)["rgb"]
                                 .reshape(v.crop_h, v.crop_w, 3)) for v in views]

    def adjoint(views, dimages, grad):
        for v, d in zip(views, dimages):
            g = osc.grad(v, alb, params, d.numpy().reshape(-1, 3), pixels=crop_pixels(v), nthreads=2)
            grad += torch.from_numpy(g)

    return render, adjoint


def _tiny_setup():
    sc = I.tiny_scene(n_inst=64)
    view = I.tiny_view()
    view.w, view.h = 72, 40
    params = I.Params(max_depth=2, sun_dir=I.MID_SUN_DIR, sun_E=(2.0, 2.0, 2.0))
    alb = I.albedo(sc.n_quads)
    dimg = np.random.default_rng(4).normal(size=(view.h, view.w, 3))
    return sc, view, params, alb, dimg


def _worker(rank, world, port, outdir):
    import torch
    import torch.distributed as dist

    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc, view, params, alb, dimg = _tiny_setup()
    osc = O.OracleScene(sc)
    render, adjoint = _oracle_fns(osc, alb, params)
    img = shard.render_frame(render, view, rank, world, tile=16,
                             like=torch.zeros(0, dtype=torch.float64))
    grad = torch.zeros((sc.n_quads, 3), dtype=torch.float64)
    shard.adjoint_frame(adjoint, view, torch.from_numpy(dimg), grad, rank, world, tile=16)
    if rank == 0:
        np.save(os.path.join(outdir, "img.npy"), img.numpy())
    np.save(os.path.join(outdir, f"grad{rank}.npy"), grad.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_render_and_adjoint_match_single_rank():
    """Two gloo ranks: round-robin 16x16 tiles (ragged at the edges) as crop
    views, tensors gathered on rank 0 and the gradient all-reduced; the
    frame equals the one-rank oracle frame exactly, every rank holds the
    whole frame's gradient."""
    import torch.multiprocessing as mp

    import oracle as O
    O.build()
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), d), nprocs=2, start_method="spawn")
        img = np.load(os.path.join(d, "img.npy"))
        grads = [np.load(os.path.join(d, f"grad{r}.npy")) for r in range(2)]
    sc, view, params, alb, dimg = _tiny_setup()
    osc = O.OracleScene(sc)
    ref = osc.render(view, alb, params)["rgb"]
    np.testing.assert_array_equal(img.reshape(-1, 3), ref)
    gref = osc.grad(view, alb, params, dimg.reshape(-1, 3))
    assert np.abs(gref).max() > 0
    for g in grads:
        np.testing.assert_allclose(g, gref, rtol=1e-12, atol=1e-15 * np.abs(gref).max())


def test_pack_and_unpack_without_a_process_group():
    """Ranks emulated in one process: every rank's packed tiles unpack to
    exactly the frame, for ragged tiles and more ranks than some tiles."""
    import torch
    for w, h, tile, world in [(72, 40, 16, 2), (33, 7, 16, 3), (5, 5, 8, 4)]:
        frame = torch.arange(w * h * 3, dtype=torch.float32).reshape(h, w, 3)

        def render(views):
            return [frame[v.crop_y:v.crop_y + v.crop_h, v.crop_x:v.crop_x + v.crop_w] for v in views]

        view = I.View(eye=(0, 0, 0), look=(0, 1, 0), up=(0, 0, 1), vfov_deg=40, w=w, h=h, spp=1)
        parts = [shard.render_tiles(render, view, r, world, tile, like=frame) for r in range(world)]
        assert all(p.shape == parts[0].shape for p in parts)
        out = shard.gather_frame(None, view, tile, parts=parts)
        assert torch.equal(out, frame)


def test_autotune_candidates_and_cache(tmp_path):
    c = autotune.candidates()
    assert len(c) == 96 and all(set(x) == {"block", "fetch", "occupancy", "batch"} for x in c)
    assert len({tuple(sorted(x.items())) for x in c}) == 96
    # stack depths proven for a scene: 3 entries per wide-node level of a
    # TLAS path plus a BLAS path
    assert autotune.proven_stack_depths(4, 6) == [32, 64]
    assert autotune.proven_stack_depths(5, 6) == [64]
    assert autotune.proven_stack_depths(12, 12) == [64]   # nothing proven: the library maximum
    k, t = autotune.pick_best({'{"a": 1}': 0.5, '{"a": 2}': None, '{"a": 3}': 0.25})
    assert k == '{"a": 3}' and t == 0.25
    with pytest.raises(RuntimeError):
        autotune.pick_best({'{"a": 1}': None})
    path = str(tmp_path / "c.json")
    key = autotune.cache_key("GB300", 152, "mid:q1e6:i1e5")
    autotune.store_cache(key, {"tuning": {"block": 128}}, path)
    autotune.store_cache("other", {"tuning": {"block": 64}}, path)
    assert autotune.load_cache(path)[key]["tuning"] == {"block": 128}
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
    sc = I.tiny_scene()
    assert autotune.scene_class(sc).startswith("tiny:q1e3:i1e2")
    v = autotune.proxy_view(I.mid_view())
    assert (v.w, v.h, v.spp) == (1024, 1024, 4)
    v = autotune.proxy_view(I.moana_view())
    assert v.spp == 16 and v.w * v.h * v.spp <= 1 << 22 and abs(v.w / v.h - 16 / 9) < 0.01
