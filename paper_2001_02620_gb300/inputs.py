"""Seeded synthetic inputs: meshes, instances, albedo, cameras and light settings.

This module only *produces inputs*.  It holds none of the path's arithmetic
(no ray generation, no intersection, no BVH, no shading); both the CUDA path
and the FP64 oracle consume what it returns.  Every array is a plain numpy
array so the two sides can marshal it their own way.

Workloads (all deterministic from integer seeds; geometry seed 1, instance
seed 2, albedo seed 3, render seed 4):

* ``tiny``  -- one 64x64-quad jittered grid, 256 randomly rotated, scaled and
  translated instances in a 100^3 box, 256x256, 1 spp, depth 2, white
  environment light only.
* ``mid``   -- 64 prototypes (half displaced grids, half closed noisy blobs)
  with log-uniform quad counts in [2^12, 2^16], a 2048x2048-quad heightfield
  terrain in 8x8 tiles, 100k random affine instances standing on the
  terrain, 1024x1024, 4 spp, depth 5, environment plus a directional sun.
* ``batched`` -- 32 views of the mid scene with uneven resolution and spp.
* ``adjoint`` -- the mid scene at 512x512, 8 spp, depth 4, plus a perturbed
  target albedo.

They stand in for the Moana Island Scene (Section 4: 39.3 M instances of
prototypes ranging from a few dozen to millions of primitives, heavily
overlapping), which is not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_GEOMETRY = 1
SEED_INSTANCES = 2
SEED_ALBEDO = 3
SEED_RENDER = 4
SEED_VIEWS = 5
SEED_TARGET = 6
SEED_TEXTURE = 7
SEED_LIGHTS = 8


@dataclass
class Scene:
    """Meshes (prototypes) plus instances.

    meshes: list of (verts float32 [V,3], quads uint32 [Q,4]); quad vertices
            are listed in order around the quad.
    xforms: float32 [N,12] object->world, row-major 3x4 (last column = translation).
    mesh_ids: uint32 [N].
    """
    meshes: list
    xforms: np.ndarray
    mesh_ids: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_quads(self) -> int:
        return int(sum(q.shape[0] for _, q in self.meshes))

    @property
    def quad_offsets(self) -> np.ndarray:
        """First albedo row of each mesh (albedo is per unique quad)."""
        counts = np.array([q.shape[0] for _, q in self.meshes], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)


@dataclass
class View:
    eye: tuple
    look: tuple
    up: tuple
    vfov_deg: float
    w: int
    h: int
    spp: int
    pixel_base: int = 0
    sample_base: int = 0  # first sample index drawn (progressive frames)
    # rendered region: the whole w x h frame when crop_w = crop_h = 0, else
    # the crop_w x crop_h rectangle at (crop_x, crop_y) of that frame
    crop_x: int = 0
    crop_y: int = 0
    crop_w: int = 0
    crop_h: int = 0

    @property
    def region(self) -> tuple:
        """(width, height) of the rendered region."""
        if self.crop_w == 0 and self.crop_h == 0:
            return int(self.w), int(self.h)
        return int(self.crop_w), int(self.crop_h)


@dataclass
class Params:
    max_depth: int
    seed: int = SEED_RENDER
    env: tuple = (1.0, 1.0, 1.0)
    sun_dir: tuple = (0.0, 0.0, 1.0)
    sun_E: tuple = (0.0, 0.0, 0.0)
    # per-face textures, float [n_quads, R, R, 3] (the renderer's copy lives
    # on its device), and key lights, float [n, 12] (corner, edge1, edge2,
    # radiance per parallelogram); None = off
    tex: object = None
    lights: object = None

    @property
    def sun_on(self) -> bool:
        return any(e != 0.0 for e in self.sun_E)


# --------------------------------------------------------------------------
# mesh builders
# --------------------------------------------------------------------------

def grid_quads(nx: int, ny: int) -> np.ndarray:
    """Quads of an (nx+1)x(ny+1) vertex lattice, counter-clockwise seen from +z."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    v00 = (j * (nx + 1) + i).ravel()
    q = np.stack([v00, v00 + 1, v00 + nx + 2, v00 + nx + 1], axis=1)
    return q.astype(np.uint32)


def _value_noise(rng: np.random.Generator, octaves: int = 5, base: int = 4):
    """Returns f(x, y) -> fbm value noise in about [-1, 1]; x, y in [0, 1]."""
    tables = []
    for o in range(octaves):
        n = base * (2 ** o) + 1
        tables.append(rng.uniform(-1.0, 1.0, size=(n, n)))

    def f(x, y):
        out = np.zeros_like(x, dtype=np.float64)
        amp = 1.0
        for tab in tables:
            n = tab.shape[0] - 1
            gx = np.clip(x, 0.0, 1.0) * n
            gy = np.clip(y, 0.0, 1.0) * n
            ix = np.minimum(gx.astype(np.int64), n - 1)
            iy = np.minimum(gy.astype(np.int64), n - 1)
            fx = gx - ix
            fy = gy - iy
            sx = fx * fx * (3 - 2 * fx)
            sy = fy * fy * (3 - 2 * fy)
            a = tab[iy, ix] * (1 - sx) + tab[iy, ix + 1] * sx
            b = tab[iy + 1, ix] * (1 - sx) + tab[iy + 1, ix + 1] * sx
            out += amp * (a * (1 - sy) + b * sy)
            amp *= 0.5
        return out / 1.9375

    return f


def tiny_mesh(seed: int = SEED_GEOMETRY):
    """65x65 vertex grid over [-1,1]^2, z ~ U(-0.1, 0.1): 4096 quads."""
    rng = np.random.default_rng(seed)
    n = 64
    xs = np.linspace(-1.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    Z = rng.uniform(-0.1, 0.1, size=X.shape)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)
    return verts, grid_quads(n, n)


def displaced_grid(rng: np.random.Generator, nq: int):
    """Unit-size displaced grid in [-0.5,0.5]^2 with fbm height (a 'leaf' or 'frond')."""
    nx = max(2, int(round(math.sqrt(nq))))
    ny = max(2, int(round(nq / nx)))
    xs = np.linspace(-0.5, 0.5, nx + 1)
    ys = np.linspace(-0.5, 0.5, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    f = _value_noise(rng, octaves=4, base=3)
    Z = 0.15 * f(X + 0.5, Y + 0.5)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)
    return verts, grid_quads(nx, ny)


def noisy_blob(rng: np.random.Generator, nq: int):
    """Closed lat-long sphere of radius ~0.5 with radial noise.

    Rows touching a pole use the single pole vertex twice, so those quads are
    degenerate on one edge (a triangle), as real production meshes have.
    """
    nlon = max(4, int(round(math.sqrt(2 * nq))))
    nlat = max(3, int(round(nq / nlon)))
    theta = np.linspace(0.0, math.pi, nlat + 1)[1:-1]  # interior rings
    phi = np.linspace(0.0, 2 * math.pi, nlon, endpoint=False)
    T, P = np.meshgrid(theta, phi, indexing="ij")
    f = _value_noise(rng, octaves=3, base=3)
    r = 0.5 * (1.0 + 0.25 * f(T / math.pi, P / (2 * math.pi)))
    ring = np.stack([r * np.sin(T) * np.cos(P), r * np.sin(T) * np.sin(P), r * np.cos(T)], axis=-1)
    ring = ring.reshape(-1, 3)
    north = np.array([[0.0, 0.0, 0.5]])
    south = np.array([[0.0, 0.0, -0.5]])
    verts = np.concatenate([ring, north, south]).astype(np.float32)
    nr = nlat - 1  # number of interior rings
    iN = nr * nlon
    iS = iN + 1
    quads = []
    j = np.arange(nlon)
    jn = (j + 1) % nlon
    # north cap: pole, ring0[j], ring0[j+1] (pole repeated -> triangle)
    quads.append(np.stack([np.full(nlon, iN), j, jn, np.full(nlon, iN)], axis=1))
    for a in range(nr - 1):
        r0 = a * nlon
        r1 = (a + 1) * nlon
        quads.append(np.stack([r0 + j, r1 + j, r1 + jn, r0 + jn], axis=1))
    r0 = (nr - 1) * nlon
    quads.append(np.stack([r0 + j, np.full(nlon, iS), np.full(nlon, iS), r0 + jn], axis=1))
    return verts, np.concatenate(quads).astype(np.uint32)


# --------------------------------------------------------------------------
# transforms
# --------------------------------------------------------------------------

def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform rotations on SO(3) from normalised Gaussian quaternions, [n,3,3]."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def pack_xforms(L: np.ndarray, t: np.ndarray) -> np.ndarray:
    """[n,3,3] linear part and [n,3] translation -> float32 [n,12] row-major 3x4."""
    n = L.shape[0]
    M = np.zeros((n, 3, 4))
    M[:, :, :3] = L
    M[:, :, 3] = t
    return M.reshape(n, 12).astype(np.float32)


IDENTITY_XFORM = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], dtype=np.float32)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def tiny_scene(seed_geom: int = SEED_GEOMETRY, seed_inst: int = SEED_INSTANCES,
               n_inst: int = 256) -> Scene:
    verts, quads = tiny_mesh(seed_geom)
    rng = np.random.default_rng(seed_inst)
    R = random_rotations(rng, n_inst)
    s = rng.uniform(0.5, 2.0, size=n_inst)
    t = rng.uniform(0.0, 100.0, size=(n_inst, 3))
    xf = pack_xforms(R * s[:, None, None], t)
    return Scene([(verts, quads)], xf, np.zeros(n_inst, dtype=np.uint32), name="tiny")


def tiny_view() -> View:
    return View(eye=(50.0, -120.0, 50.0), look=(50.0, 50.0, 50.0), up=(0.0, 0.0, 1.0),
                vfov_deg=40.0, w=256, h=256, spp=1)


def tiny_params() -> Params:
    return Params(max_depth=2, env=(1.0, 1.0, 1.0), sun_E=(0.0, 0.0, 0.0))


def albedo(n_quads: int, seed: int = SEED_ALBEDO, lo: float = 0.2, hi: float = 0.8) -> np.ndarray:
    """Per-unique-quad RGB albedo, float32 [n_quads, 3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n_quads, 3)).astype(np.float32)


MID_TERRAIN_EXTENT = 4096.0
MID_TERRAIN_QUADS = 2048
MID_TERRAIN_AMPLITUDE = 150.0


def terrain_heights(seed: int, nq: int = MID_TERRAIN_QUADS,
                    amplitude: float = MID_TERRAIN_AMPLITUDE) -> np.ndarray:
    rng = np.random.default_rng(seed + 1000)
    f = _value_noise(rng, octaves=6, base=4)
    u = np.linspace(0.0, 1.0, nq + 1)
    U, V = np.meshgrid(u, u, indexing="xy")
    return amplitude * f(U, V)


def terrain_mesh(heights: np.ndarray, extent: float):
    n = heights.shape[0] - 1
    xs = np.linspace(0.0, extent, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel(), heights.ravel()], axis=1).astype(np.float32)
    return verts, grid_quads(n, n)


def terrain_tiles(heights: np.ndarray, extent: float, tiles: int = 8):
    """The heightfield as tiles x tiles meshes, each in coordinates local to
    its tile centre, with the instance translations that put them back.  The
    grid spacing and tile size are powers of two, so every local coordinate
    and translation is exact and the world-space vertices equal those of
    terrain_mesh() bit for bit."""
    n = heights.shape[0] - 1
    assert n % tiles == 0
    k = n // tiles
    step = extent / n
    meshes, trans = [], []
    for j in range(tiles):
        for i in range(tiles):
            h = heights[j * k:(j + 1) * k + 1, i * k:(i + 1) * k + 1]
            cx = (i + 0.5) * k * step
            cy = (j + 0.5) * k * step
            xs = (np.arange(k + 1) - 0.5 * k) * step
            X, Y = np.meshgrid(xs, xs, indexing="xy")
            verts = np.stack([X.ravel(), Y.ravel(), h.ravel()], axis=1).astype(np.float32)
            meshes.append((verts, grid_quads(k, k)))
            trans.append((cx, cy, 0.0))
    return meshes, np.asarray(trans)


def _terrain_height_at(heights: np.ndarray, extent: float, x, y):
    n = heights.shape[0] - 1
    gx = np.clip(x / extent * n, 0, n - 1e-9)
    gy = np.clip(y / extent * n, 0, n - 1e-9)
    ix = gx.astype(np.int64)
    iy = gy.astype(np.int64)
    fx = gx - ix
    fy = gy - iy
    h = heights
    return ((h[iy, ix] * (1 - fx) + h[iy, ix + 1] * fx) * (1 - fy)
            + (h[iy + 1, ix] * (1 - fx) + h[iy + 1, ix + 1] * fx) * fy)


def mid_scene(seed_geom: int = SEED_GEOMETRY, seed_inst: int = SEED_INSTANCES,
              n_proto: int = 64, n_inst: int = 100_000,
              terrain_quads: int = MID_TERRAIN_QUADS,
              extent: float = MID_TERRAIN_EXTENT) -> Scene:
    """64 prototypes + terrain, 100k instances + 1 terrain instance (identity)."""
    rng = np.random.default_rng(seed_geom)
    meshes = []
    for p in range(n_proto):
        nq = int(round(2.0 ** rng.uniform(12.0, 16.0)))
        meshes.append(displaced_grid(rng, nq) if p % 2 == 0 else noisy_blob(rng, nq))
    heights = terrain_heights(seed_geom, terrain_quads)
    tiles, tile_t = terrain_tiles(heights, extent)
    terrain_first = len(meshes)
    meshes.extend(tiles)

    rng = np.random.default_rng(seed_inst)
    R = random_rotations(rng, n_inst)
    s = rng.uniform(0.5, 2.0, size=(n_inst, 3))
    base = np.exp(rng.uniform(math.log(4.0), math.log(40.0), size=n_inst))
    L = R * (s * base[:, None])[:, None, :]          # R @ diag(s * base)
    x = rng.uniform(0.0, extent, size=n_inst)
    y = rng.uniform(0.0, extent, size=n_inst)
    z = _terrain_height_at(heights, extent, x, y)
    xf = pack_xforms(L, np.stack([x, y, z], axis=1))
    ids = rng.integers(0, n_proto, size=n_inst).astype(np.uint32)
    nt = len(tiles)
    xf = np.concatenate([xf, pack_xforms(np.broadcast_to(np.eye(3), (nt, 3, 3)), tile_t)], axis=0)
    ids = np.concatenate([ids, np.arange(terrain_first, terrain_first + nt, dtype=np.uint32)])
    return Scene(meshes, xf, ids, name="mid",
                 meta={"n_proto": n_proto, "terrain_meshes": (terrain_first, nt), "extent": extent})


def mid_view(w: int = 1024, h: int = 1024, spp: int = 4) -> View:
    return View(eye=(2048.0, -300.0, 450.0), look=(2048.0, 1800.0, 0.0), up=(0.0, 0.0, 1.0),
                vfov_deg=50.0, w=w, h=h, spp=spp)


def _normalize(v):
    v = np.asarray(v, dtype=np.float64)
    return tuple(float(c) for c in v / np.linalg.norm(v))


MID_SUN_DIR = _normalize((0.4, 0.3, 1.0))


def mid_params(max_depth: int = 5) -> Params:
    return Params(max_depth=max_depth, env=(1.0, 1.0, 1.0), sun_dir=MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))


def batched_views(n_views: int = 32, seed: int = SEED_VIEWS, min_log2: float = 8.0,
                  max_log2: float = 11.0, max_spp: int = 16) -> list:
    """Uneven views around the mid vista: side = 32*round(2^U(8,11)/32), spp ~ U{1..16}.

    pixel_base is the running pixel count, so every (view, pixel) has a unique
    global pixel index and therefore its own random stream.
    """
    rng = np.random.default_rng(seed)
    views = []
    base = 0
    for _ in range(n_views):
        side = int(32 * round(2.0 ** rng.uniform(min_log2, max_log2) / 32))
        side = max(32, side)
        spp = int(rng.integers(1, max_spp + 1))
        ex = 2048.0 + rng.uniform(-1200.0, 1200.0)
        ey = rng.uniform(-600.0, 600.0)
        ez = rng.uniform(250.0, 700.0)
        lx = ex + rng.uniform(-800.0, 800.0)
        ly = ey + rng.uniform(1200.0, 2400.0)
        views.append(View(eye=(ex, ey, ez), look=(lx, ly, 0.0), up=(0.0, 0.0, 1.0),
                          vfov_deg=float(rng.uniform(35.0, 60.0)), w=side, h=side, spp=spp,
                          pixel_base=base))
        base += side * side
    return views


def adjoint_view() -> View:
    return mid_view(512, 512, 8)


def adjoint_params() -> Params:
    return mid_params(max_depth=4)


def face_textures(n_quads: int, res: int = 4, seed: int = SEED_TEXTURE, lo: float = 0.4,
                  hi: float = 1.0) -> np.ndarray:
    """Per-face texel grids standing in for Ptex textures (a texture baked on
    each face, modulating the diffuse albedo): res x res RGB texels per quad,
    U(lo, hi), float [n_quads, res, res, 3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n_quads, res, res, 3)).astype(np.float32)


def key_lights(n: int, lo, hi, size, height: float, radiance, seed: int = SEED_LIGHTS) -> np.ndarray:
    """n square key lights facing down (parallelograms emitting toward -z),
    side `size`, centres uniform over the box [lo, hi] of xy at z = height,
    spun about z; radiance RGB scaled by U(0.5, 1.5).  float [n, 12]:
    corner, edge1, edge2, radiance."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 12), dtype=np.float32)
    for k in range(n):
        cx, cy = rng.uniform(lo[0], hi[0]), rng.uniform(lo[1], hi[1])
        phi = rng.uniform(0.0, 2.0 * math.pi)
        e1 = size * np.array([math.cos(phi), math.sin(phi), 0.0])
        e2 = size * np.array([math.sin(phi), -math.cos(phi), 0.0])   # e1 x e2 points down
        c = np.array([cx, cy, height]) - 0.5 * (e1 + e2)
        out[k, 0:3], out[k, 3:6], out[k, 6:9] = c, e1, e2
        out[k, 9:12] = np.asarray(radiance, dtype=np.float64) * rng.uniform(0.5, 1.5)
    return out


def tiny_lights() -> np.ndarray:
    """Four key lights above the tiny scene's 100^3 box."""
    return key_lights(4, (10.0, 10.0), (90.0, 90.0), 15.0, 130.0, (30.0, 27.0, 22.0))


def mid_lights() -> np.ndarray:
    """The 23 key lights of the paper's Moana scene (Section 4.1), as squares
    of side 120 at height 600 over the mid terrain."""
    return key_lights(23, (300.0, 300.0), (3800.0, 3800.0), 120.0, 600.0, (60.0, 55.0, 45.0))


def perturbed_albedo(a: np.ndarray, seed: int = SEED_TARGET, sigma: float = 0.05) -> np.ndarray:
    """Target albedo a* + N(0, sigma), clamped to [0.01, 0.99]."""
    rng = np.random.default_rng(seed)
    return np.clip(a + rng.normal(0.0, sigma, size=a.shape), 0.01, 0.99).astype(np.float32)


# --------------------------------------------------------------------------
# ray sets for the trace entry points (independent of any renderer)
# --------------------------------------------------------------------------

def ray_array(o: np.ndarray, d: np.ndarray, tmin: float = 0.0, tmax: float = np.inf) -> np.ndarray:
    """Pack origins/directions into float32 [n,8] = (o, tmin, d, tmax)."""
    n = o.shape[0]
    r = np.empty((n, 8), dtype=np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


def scene_box(scene: Scene) -> tuple:
    """Loose world box from instance translations (inputs only, not a bound)."""
    t = scene.xforms.reshape(-1, 3, 4)[:, :, 3].astype(np.float64)
    return t.min(axis=0), t.max(axis=0)


def rays_focused(n: int, eye, lo, hi, seed: int) -> np.ndarray:
    """Coherent bundle: from one eye toward uniform points in [lo, hi]."""
    rng = np.random.default_rng(seed)
    tgt = rng.uniform(lo, hi, size=(n, 3))
    o = np.broadcast_to(np.asarray(eye, dtype=np.float64), (n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return ray_array(o, d)


def rays_random(n: int, lo, hi, seed: int, tmax: float = np.inf) -> np.ndarray:
    """Incoherent: uniform origins in [lo, hi], uniform directions on the sphere."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return ray_array(o, d, 0.0, tmax)


def rays_parallel(n: int, lo, hi, direction, seed: int) -> np.ndarray:
    """Shadow-like: uniform origins in [lo, hi], one shared direction."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(lo, hi, size=(n, 3))
    d = np.broadcast_to(np.asarray(direction, dtype=np.float64), (n, 3))
    return ray_array(o, d)


def rays_toward(n: int, lo, hi, targets: np.ndarray, jitter: float, seed: int) -> np.ndarray:
    """Origins uniform in [lo, hi], each aimed at a random target point
    (plus a uniform jitter of +-jitter per axis) -- a high hit-rate ray set."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(lo, hi, size=(n, 3))
    k = rng.integers(0, targets.shape[0], size=n)
    tgt = targets[k] + rng.uniform(-jitter, jitter, size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return ray_array(o, d)


def instance_origins(scene: Scene) -> np.ndarray:
    """Translation column of each instance transform (where its object sits)."""
    return scene.xforms.reshape(-1, 3, 4)[:, :, 3].astype(np.float64)


def sphere_mesh(n_lat: int = 24, n_lon: int = 48, radius: float = 1.0):
    """Noise-free lat-long sphere (a convex polyhedron), pole rows degenerate."""
    theta = np.linspace(0.0, math.pi, n_lat + 1)[1:-1]
    phi = np.linspace(0.0, 2 * math.pi, n_lon, endpoint=False)
    T, P = np.meshgrid(theta, phi, indexing="ij")
    ring = radius * np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    verts = np.concatenate([ring.reshape(-1, 3), [[0, 0, radius]], [[0, 0, -radius]]]).astype(np.float32)
    nr = n_lat - 1
    iN, iS = nr * n_lon, nr * n_lon + 1
    j = np.arange(n_lon)
    jn = (j + 1) % n_lon
    quads = [np.stack([np.full(n_lon, iN), j, jn, np.full(n_lon, iN)], axis=1)]
    for a in range(nr - 1):
        quads.append(np.stack([a * n_lon + j, (a + 1) * n_lon + j, (a + 1) * n_lon + jn, a * n_lon + jn], axis=1))
    r0 = (nr - 1) * n_lon
    quads.append(np.stack([r0 + j, np.full(n_lon, iS), np.full(n_lon, iS), r0 + jn], axis=1))
    return verts, np.concatenate(quads).astype(np.uint32)


def plane_mesh(n: int = 8):
    """Flat n x n quad grid over [-1,1]^2 at z = 0."""
    xs = np.linspace(-1.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1).astype(np.float32)
    return verts, grid_quads(n, n)


# --------------------------------------------------------------------------
# Moana-scale workload
# --------------------------------------------------------------------------

MOANA_QUADS = 261_100_000          # unique quads (Section 1)
MOANA_INSTANCES = 39_300_000       # instances (Section 1)
MOANA_INSTANCED_QUADS = 82.4e9     # quads after instancing (Section 1)
MOANA_PROTOS = 5000
MOANA_NMAX = 8_000_000             # multi-million-quad trees (Section 4.2)
MOANA_EXTENT = 8192.0
MOANA_TERRAIN_QUADS = 2048


def _solve_bisect(f, lo, hi, iters=100):
    flo = f(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def moana_sizes(scale: float = 1.0, seed: int = SEED_GEOMETRY):
    """Prototype quad counts and instance counts of the Moana-scale workload.

    Two populations, as the island has (Section 4.2): 1000 large objects with
    quad counts n_p = n_max p^-gamma (trees of millions of quads down to
    rocks and bushes), gamma solved so that all unique quads total 261 M; and
    4000 small objects of 2^U(4, 9) quads (leaves, buds, pebbles).  Instance
    counts: large objects c_p proportional to n_p^-1/2, small ones uniform;
    the split between the two is solved so that the instances total 39.3 M
    and the instanced quads 82.4 G.  scale < 1 shrinks every total."""
    s1 = min(1.0, scale ** 0.5)
    PL = max(4, int(round(1000 * s1)))
    PS = max(4, int(round(4000 * s1)))
    rng = np.random.default_rng(seed + 77)
    ns = np.round(2.0 ** rng.uniform(4.0, 9.0, size=PS)).astype(np.int64)
    terrain = MOANA_TERRAIN_QUADS ** 2 if scale >= 0.5 else int(MOANA_TERRAIN_QUADS * scale ** 0.5) ** 2
    QL = MOANA_QUADS * scale - terrain - ns.sum()
    nmax = max(256.0, MOANA_NMAX * scale)
    p = np.arange(1, PL + 1, dtype=np.float64)
    gamma = _solve_bisect(lambda g: np.maximum(16.0, nmax * p ** -g).sum() - QL, 0.01, 6.0)
    nl = np.maximum(16, np.round(nmax * p ** -gamma)).astype(np.int64)
    N = MOANA_INSTANCES * scale
    QI = MOANA_INSTANCED_QUADS * scale
    wl = nl.astype(np.float64) ** -0.5
    mL = (wl * nl).sum() / wl.sum()
    mS = float(ns.mean())
    NL = (QI - N * mS) / (mL - mS)
    NL = float(np.clip(NL, PL, N - PS))
    cl = np.maximum(1, np.round(NL * wl / wl.sum())).astype(np.int64)
    ws = rng.uniform(0.5, 1.5, size=PS)
    cs = np.maximum(1, np.round((N - NL) * ws / ws.sum())).astype(np.int64)
    return np.concatenate([nl, ns]), np.concatenate([cl, cs]), terrain


def moana_scene(scale: float = 1.0, seed_geom: int = SEED_GEOMETRY,
                seed_inst: int = SEED_INSTANCES) -> Scene:
    """Synthetic Moana-scale island: Zipf-sized prototypes (displaced grids and
    closed blobs) instanced as clustered vegetation over a heightfield terrain
    (Thomas cluster process), rotation about z with up to 15 degrees of tilt,
    isotropic scale U(0.5, 2) times a size that grows with the prototype's
    quad count.  scale < 1 shrinks every total proportionally."""
    n, c, terrain_q = moana_sizes(scale, seed_geom)
    extent = MOANA_EXTENT * (scale ** 0.5 if scale < 1.0 else 1.0)
    rng = np.random.default_rng(seed_geom)
    meshes = []
    for k, nq in enumerate(n):
        meshes.append(displaced_grid(rng, int(nq)) if k % 2 == 0 else noisy_blob(rng, int(nq)))
    tq = int(round(terrain_q ** 0.5))
    heights = terrain_heights(seed_geom + 7, tq, amplitude=220.0)
    ntile = 8 if tq % 8 == 0 else 1
    tiles, tile_t = terrain_tiles(heights, extent, ntile)
    terrain_first = len(meshes)
    meshes.extend(tiles)

    rng = np.random.default_rng(seed_inst)
    ids = np.repeat(np.arange(len(n), dtype=np.uint32), c)
    rng.shuffle(ids)
    N = ids.shape[0]
    # Thomas cluster process: parents uniform, children Gaussian around them
    n_par = max(1, N // 300)
    par = rng.uniform(0.0, extent, size=(n_par, 2))
    which = rng.integers(0, n_par, size=N)
    xy = par[which] + rng.normal(0.0, extent / 400.0, size=(N, 2))
    xy = np.clip(xy, 0.0, extent)
    z = _terrain_height_at(heights, extent, xy[:, 0], xy[:, 1])
    # rotation: tilt <= 15 degrees about a horizontal axis, then spin about z
    phi = rng.uniform(0.0, 2 * math.pi, size=N)
    tilt = np.radians(rng.uniform(0.0, 15.0, size=N))
    ax = rng.uniform(0.0, 2 * math.pi, size=N)
    size = 0.5 * (n[ids].astype(np.float64) / 16.0) ** 0.3 * rng.uniform(0.5, 2.0, size=N)
    cz, sz = np.cos(phi), np.sin(phi)
    ux, uy = np.cos(ax), np.sin(ax)
    ct, st = np.cos(tilt), np.sin(tilt)
    # Rodrigues rotation about (ux, uy, 0) by tilt
    T = np.empty((N, 3, 3))
    T[:, 0, 0] = ct + ux * ux * (1 - ct)
    T[:, 0, 1] = ux * uy * (1 - ct)
    T[:, 0, 2] = uy * st
    T[:, 1, 0] = ux * uy * (1 - ct)
    T[:, 1, 1] = ct + uy * uy * (1 - ct)
    T[:, 1, 2] = -ux * st
    T[:, 2, 0] = -uy * st
    T[:, 2, 1] = ux * st
    T[:, 2, 2] = ct
    Z = np.zeros((N, 3, 3))
    Z[:, 0, 0] = cz
    Z[:, 0, 1] = -sz
    Z[:, 1, 0] = sz
    Z[:, 1, 1] = cz
    Z[:, 2, 2] = 1.0
    L = np.einsum("nij,njk->nik", T, Z) * size[:, None, None]
    xf = pack_xforms(L, np.stack([xy[:, 0], xy[:, 1], z], axis=1))
    nt = len(tiles)
    inst_q = int(n[ids].sum()) + terrain_q
    xf = np.concatenate([xf, pack_xforms(np.broadcast_to(np.eye(3), (nt, 3, 3)), tile_t)], axis=0)
    ids = np.concatenate([ids, np.arange(terrain_first, terrain_first + nt, dtype=np.uint32)])
    return Scene(meshes, xf, ids, name="moana",
                 meta={"n_proto": int(len(n)), "terrain_meshes": (terrain_first, nt),
                       "extent": extent, "instanced_quads": inst_q})


def moana_view(extent: float = MOANA_EXTENT, w: int = 1920, h: int = 1080, spp: int = 16) -> View:
    return View(eye=(0.5 * extent, -0.07 * extent, 0.11 * extent),
                look=(0.5 * extent, 0.45 * extent, 0.0), up=(0.0, 0.0, 1.0),
                vfov_deg=50.0, w=w, h=h, spp=spp)


def moana_params() -> Params:
    return mid_params(max_depth=8)
