"""Image-parallel sharding across ranks (Section 5.5, paragraph "The
Distributed FrameBuffer": the image is split into tiles assigned round-robin to nodes that
each hold the whole scene, and the tiles are gathered on the head node).

Each rank renders the pixels of its tiles with a renderer callback
render_pixels(pixel_indices) -> float [n, 3]; gather_image assembles the frame
on rank 0.  Pixels, samples and views are independent, so no exchange happens
before the gather.
"""
from __future__ import annotations

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


def pixels_of_tiles(w: int, tile_boxes, which) -> np.ndarray:
    idx = []
    for t in which:
        x0, y0, x1, y1 = tile_boxes[t]
        ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        idx.append((ys * w + xs).ravel())
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def render_shard(render_pixels, w: int, h: int, rank: int, world: int, tile: int = 32):
    """Renders this rank's tiles: returns (pixel indices, rgb [n, 3])."""
    boxes = tiles(w, h, tile)
    px = pixels_of_tiles(w, boxes, tiles_of_rank(len(boxes), rank, world)).astype(np.int64)
    rgb = np.asarray(render_pixels(px), dtype=np.float64).reshape(-1, 3) if len(px) else \
        np.zeros((0, 3))
    return px, rgb


def gather_image(px: np.ndarray, rgb: np.ndarray, w: int, h: int, group=None):
    """Collects every rank's (pixels, rgb) on rank 0 and returns the [h, w, 3]
    image there (None elsewhere).  Uses torch.distributed when initialised."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        img = np.zeros((h * w, 3))
        img[px] = rgb
        return img.reshape(h, w, 3)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = [None] * world if rank == 0 else None
    dist.gather_object((px, rgb), parts, dst=0, group=group)
    if rank != 0:
        return None
    img = np.full((h * w, 3), np.nan)
    for p, c in parts:
        img[p] = c
    if np.isnan(img).any():
        raise RuntimeError("some pixels were not rendered by any rank")
    return img.reshape(h, w, 3)
