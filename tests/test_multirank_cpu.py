"""Multi-rank logic on CPU: round-robin tile sharding and the gather to rank 0
with two gloo ranks, the oracle standing in for the renderer; plus the
autotuner's host-side logic (candidate space, cache, selection)."""
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


def _worker(rank, world, port, outdir):
    import torch.distributed as dist

    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = I.tiny_scene(n_inst=64)
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w, view.h = 72, 40
    params = I.Params(max_depth=2)
    alb = I.albedo(sc.n_quads)
    px, rgb = shard.render_shard(lambda p: osc.render(view, alb, params, pixels=p, nthreads=2)["rgb"],
                                 view.w, view.h, rank, world, tile=16)
    img = shard.gather_image(px, rgb, view.w, view.h)
    if rank == 0:
        np.save(os.path.join(outdir, "img.npy"), img)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_render_matches_single_rank():
    import torch.multiprocessing as mp

    import oracle as O
    O.build()
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), d), nprocs=2, start_method="spawn")
        img = np.load(os.path.join(d, "img.npy"))
    sc = I.tiny_scene(n_inst=64)
    view = I.tiny_view()
    view.w, view.h = 72, 40
    ref = O.OracleScene(sc).render(view, I.albedo(sc.n_quads), I.Params(max_depth=2))["rgb"]
    np.testing.assert_array_equal(img.reshape(-1, 3), ref)


def test_autotune_candidates_and_cache(tmp_path):
    c = autotune.candidates()
    assert len(c) == 18 and all(set(x) == {"block", "fetch", "occupancy"} for x in c)
    assert len({tuple(sorted(x.items())) for x in c}) == 18
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
