"""Image-parallel rendering across ranks (Section 5.5, paragraph "The
Distributed FrameBuffer": the frame is cut into tiles that are assigned
round-robin to nodes which each hold the whole scene, and the tiles are
gathered on the head node).

A rank renders its tiles as crops of the frame (qrt_view.crop_*): the camera
and the random streams are those of the whole frame, so the gathered frame
is bit-identical to a one-rank render.  The gather moves tensors with
torch.distributed (NCCL or gloo): each rank packs its tiles into a buffer of
ceil(tiles / ranks) tile slots, rank 0 receives every rank's buffer
(dist.gather) and unpacks the frame.  The albedo gradient of a frame is the
sum of every rank's tile gradients: one all-reduce (SUM) of the gradient
tensor.  Pixels, samples and views are independent, so nothing else is
exchanged.

The renderer is a callback, render_fn(crop views) -> list of [ch, cw, 3]
tensors: scene_renderer() wraps a GPU scene (every step in libqrt.so); the
CPU tests pass the oracle instead.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def tiles(w: int, h: int, tile: int = 32) -> list[tuple[int, int, int, int]]:
    """(x0, y0, x1, y1) of every tile, row-major; edge tiles are ragged."""
    out = []
    for y0 in range(0, h, tile):
        for x0 in range(0, w, tile):
            out.append((x0, y0, min(x0 + tile, w), min(y0 + tile, h)))
    return out


def tiles_of_rank(n_tiles: int, rank: int, world: int) -> list[int]:
    """Round-robin assignment: tile t goes to rank t % world."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(range(rank, n_tiles, world))


def slots(n_tiles: int, world: int) -> int:
    """Tile slots of every rank's packed buffer (the largest share)."""
    return (n_tiles + world - 1) // world


def pixels_of_tiles(w: int, tile_boxes, which) -> np.ndarray:
    """Frame pixel indices y * w + x of the given tiles, tile by tile, row-major."""
    idx = []
    for t in which:
        x0, y0, x1, y1 = tile_boxes[t]
        ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        idx.append((ys * w + xs).ravel())
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def tile_views(view, tile_boxes, which) -> list:
    """One crop of `view` per tile (same camera, frame and random streams)."""
    return [dataclasses.replace(view, crop_x=x0, crop_y=y0, crop_w=x1 - x0, crop_h=y1 - y0)
            for (x0, y0, x1, y1) in (tile_boxes[t] for t in which)]


def rank_views(view, rank: int, world: int, tile: int = 32) -> list:
    """The crop views of this rank's tiles."""
    boxes = tiles(view.w, view.h, tile)
    return tile_views(view, boxes, tiles_of_rank(len(boxes), rank, world))


def pack_tiles(imgs, tile: int, n_slots: int, like):
    """Stacks a rank's tile images ([ch, cw, C] each) into a zero-padded
    [n_slots, tile, tile, C] tensor of `like`'s dtype and device."""
    import torch
    C = like.shape[-1] if like is not None and like.dim() else 3
    out = torch.zeros((n_slots, tile, tile, C), dtype=like.dtype, device=like.device)
    for k, im in enumerate(imgs):
        out[k, :im.shape[0], :im.shape[1]] = im
    return out


def unpack_frame(parts, tile_boxes, world: int, w: int, h: int):
    """Frame [h, w, C] from every rank's packed buffer (parts[r] from rank r)."""
    import torch
    C = parts[0].shape[-1]
    frame = torch.empty((h, w, C), dtype=parts[0].dtype, device=parts[0].device)
    for r in range(world):
        for k, t in enumerate(tiles_of_rank(len(tile_boxes), r, world)):
            x0, y0, x1, y1 = tile_boxes[t]
            frame[y0:y1, x0:x1] = parts[r][k, :y1 - y0, :x1 - x0]
    return frame


def gather_frame(packed, view, tile: int = 32, group=None, world: int | None = None,
                 rank: int | None = None, parts=None):
    """Collects every rank's packed tiles on rank 0 and returns the frame
    there (None on the other ranks).  With torch.distributed initialised the
    buffers travel by dist.gather; otherwise `parts` (all ranks' buffers,
    e.g. from ranks emulated in one process) is unpacked directly."""
    import torch.distributed as dist
    boxes = tiles(view.w, view.h, tile)
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        bufs = [packed.new_empty(packed.shape) for _ in range(world)] if rank == 0 else None
        dist.gather(packed, bufs, dst=0, group=group)
        if rank != 0:
            return None
        return unpack_frame(bufs, boxes, world, view.w, view.h)
    if parts is None:
        parts = [packed]
        world = 1
    return unpack_frame(parts, boxes, world or len(parts), view.w, view.h)


def render_tiles(render_fn, view, rank: int, world: int, tile: int = 32, like=None):
    """This rank's tiles rendered by render_fn and packed for the gather."""
    boxes = tiles(view.w, view.h, tile)
    views = tile_views(view, boxes, tiles_of_rank(len(boxes), rank, world))
    imgs = render_fn(views) if views else []
    ref = imgs[0] if imgs else like
    return pack_tiles(imgs, tile, slots(len(boxes), world), ref)


def render_frame(render_fn, view, rank: int, world: int, tile: int = 32, group=None, like=None):
    """Image-parallel frame: this rank renders its tiles, rank 0 returns the
    gathered [h, w, 3] frame (the other ranks None).  `like` gives dtype and
    device of an empty share (a rank with no tile)."""
    return gather_frame(render_tiles(render_fn, view, rank, world, tile, like), view, tile, group)


def allreduce_sum(t, group=None):
    """In-place SUM over ranks (no-op without torch.distributed)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def adjoint_frame(adjoint_fn, view, dimage, grad, rank: int, world: int, tile: int = 32,
                  group=None):
    """Albedo gradient of a frame split over ranks: this rank adds the
    adjoint of its tiles (adjoint_fn(crop views, dimage crops, grad)) into
    grad, then the ranks' gradients are summed by one all-reduce.  dimage:
    the whole frame's image gradient [h, w, 3] (each rank reads its crops)."""
    boxes = tiles(view.w, view.h, tile)
    which = tiles_of_rank(len(boxes), rank, world)
    views = tile_views(view, boxes, which)
    crops = [dimage[y0:y1, x0:x1].contiguous() for (x0, y0, x1, y1) in (boxes[t] for t in which)]
    if views:
        adjoint_fn(views, crops, grad)
    return allreduce_sum(grad, group)


def scene_renderer(scene, albedo, params, tuning=None):
    """render_fn of a GPU scene (api.Scene): one call renders all given crops."""
    return lambda views: scene.render(views, albedo, params, tuning=tuning)


def scene_adjoint(scene, albedo, params, tuning=None):
    """adjoint_fn of a GPU scene: the replay adjoint of all given crops."""
    return lambda views, dimages, grad: scene.adjoint(views, albedo, dimages, grad, params,
                                                      tuning=tuning)
