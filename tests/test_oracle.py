"""Pins for the FP64 oracle: each check ties the oracle to something other than
itself (a closed form, an external implementation, brute force, or an
invariant of the method) so that a dropped term, a wrong sign or index, or a
transposed operand fails at least one of them.  CPU only.
"""
import dataclasses
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle as O
from paper_2001_02620_gb300 import inputs as I

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


# ---------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------

def test_philox_zero_vector_known_answer():
    # Counter 0, key 0: the first output word of Philox4x32-10 is 0x6627e8d5
    # (the all-zero known-answer vector of the generator's authors).
    out = O.philox([0, 0, 0, 0], [0, 0])
    assert int(out[0]) == 0x6627E8D5


def test_philox_matches_triton_interpreter():
    """Cross-check against an independent Philox4x32-10: Triton's, run by its
    CPU interpreter in a child process (the interpreter mode must be chosen
    before triton is imported)."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    n = 64
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    seeds = rng.integers(0, 2**63, size=n, dtype=np.uint64)
    seeds[0] = 0
    ctr[0] = 0
    prog = textwrap.dedent("""
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl
        from triton.language.random import philox

        @triton.jit
        def k(out, seed, c0, c1, c2, c3):
            a, b, c, d = philox(seed, tl.load(c0), tl.load(c1), tl.load(c2), tl.load(c3), 10)
            tl.store(out + 0, a); tl.store(out + 1, b); tl.store(out + 2, c); tl.store(out + 3, d)

        data = json.loads(sys.stdin.read())
        res = []
        for seed, c in zip(data["seeds"], data["ctr"]):
            cs = [torch.tensor([x], dtype=torch.uint32) for x in c]
            out = torch.zeros(4, dtype=torch.uint32)
            k[(1,)](out, seed, *cs)
            res.append([int(x) & 0xFFFFFFFF for x in out.tolist()])
        print(json.dumps(res))
    """)
    import json
    payload = json.dumps({"seeds": [int(s) for s in seeds], "ctr": ctr.tolist()})
    r = subprocess.run([sys.executable, "-c", prog], input=payload, capture_output=True,
                       text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint64)
    for i in range(n):
        s = int(seeds[i])
        got = O.philox(ctr[i], [s & 0xFFFFFFFF, s >> 32])
        assert got.tolist() == ref[i].tolist(), (i, ctr[i], s)


# ---------------------------------------------------------------------------
# Ray / quad
# ---------------------------------------------------------------------------

UNIT_Z5 = np.array([[0, 0, 5], [1, 0, 5], [1, 1, 5], [0, 1, 5]], dtype=np.float64)


def test_quad_axis_aligned_closed_form():
    hit, t, u, v = O.intersect_quad([0.25, 0.5, 0.0], [0, 0, 1], UNIT_Z5)
    assert hit and t == 5.0
    # unit square: quad-space (u, v) is the (x, y) position of the hit
    assert abs(u - 0.25) < 1e-15 and abs(v - 0.5) < 1e-15
    hit, t, u, v = O.intersect_quad([0.75, 0.2, 0.0], [0, 0, 1], UNIT_Z5)
    assert hit and abs(u - 0.75) < 1e-15 and abs(v - 0.2) < 1e-15
    # from the other side (double-sided), scaled direction: t scales with 1/|d|
    hit, t, u, v = O.intersect_quad([0.3, 0.6, 9.0], [0, 0, -2.0], UNIT_Z5)
    assert hit and abs(t - 2.0) < 1e-15


def test_quad_skew_ray_closed_form():
    d = np.array([0.05, 0.1, 1.0])   # lands at (0.4, 0.7) on z = 5
    d /= np.linalg.norm(d)
    o = np.array([0.1, 0.1, -1.0])
    hit, t, u, v = O.intersect_quad(o, d, UNIT_Z5)
    t_exact = (5.0 - o[2]) / d[2]
    p = o + t_exact * d
    assert hit and abs(t - t_exact) < 1e-13 * t_exact
    assert abs(u - p[0]) < 1e-13 and abs(v - p[1]) < 1e-13


def test_quad_tilted_plane_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(200):
        c = rng.normal(size=3)
        e1 = rng.normal(size=3)
        e2 = rng.normal(size=3)
        q = np.array([c, c + e1, c + e1 + e2, c + e2])  # planar parallelogram
        n = np.cross(e1, e2)
        a, b = rng.uniform(0.05, 0.95, size=2)
        target = c + a * e1 + b * e2
        o = target + rng.normal(size=3) * 3
        d = target - o
        hit, t, u, v = O.intersect_quad(o, d, q)
        t_exact = np.dot(n, c - o) / np.dot(n, d)
        assert hit
        assert abs(t - t_exact) < 1e-10 * abs(t_exact)
        assert abs(t - 1.0) < 1e-10  # d reaches the target at t = 1


def test_quad_edges_vertices_and_misses():
    def hit_at(x, y):
        return O.intersect_quad([x, y, 0.0], [0, 0, 1], UNIT_Z5)[0]
    # edges, vertices and the shared diagonal are inclusive
    for x, y in [(0.5, 0.0), (1.0, 0.5), (0.5, 1.0), (0.0, 0.5), (0, 0), (1, 0), (1, 1), (0, 1),
                 (0.5, 0.5), (0.25, 0.25)]:
        assert hit_at(x, y), (x, y)
    for x, y in [(1 + 1e-9, 0.5), (-1e-9, 0.5), (0.5, -1e-9), (0.5, 1 + 1e-9), (2, 2)]:
        assert not hit_at(x, y), (x, y)
    # parallel, behind the origin, beyond tmax, at exactly tmax (open interval)
    assert not O.intersect_quad([0.5, 0.5, 5.0], [1, 0, 0], UNIT_Z5)[0]
    assert not O.intersect_quad([0.5, 0.5, 10.0], [0, 0, 1], UNIT_Z5)[0]
    assert not O.intersect_quad([0.5, 0.5, 0.0], [0, 0, 1], UNIT_Z5, 0.0, 4.9)[0]
    assert not O.intersect_quad([0.5, 0.5, 0.0], [0, 0, 1], UNIT_Z5, 0.0, 5.0)[0]
    assert not O.intersect_quad([0.5, 0.5, 0.0], [0, 0, 1], UNIT_Z5, 5.0, 9.0)[0]


def test_quad_nonplanar_picks_triangle_by_side_of_diagonal():
    # v2 lifted: triangle (v0,v1,v2) and (v0,v2,v3) are different planes
    q = UNIT_Z5.copy()
    q[2, 2] = 7.0
    # below the diagonal (y < x) -> triangle 0: plane through (0,0,5),(1,0,5),(1,1,7): z = 5 + 2y
    hit, t, u, v = O.intersect_quad([0.8, 0.3, 0.0], [0, 0, 1], q)
    assert hit and abs(t - (5 + 2 * 0.3)) < 1e-14
    # above (y > x) -> triangle 1: plane through (0,0,5),(1,1,7),(0,1,5): z = 5 + 2x
    hit, t, u, v = O.intersect_quad([0.3, 0.8, 0.0], [0, 0, 1], q)
    assert hit and abs(t - (5 + 2 * 0.3)) < 1e-14


def test_degenerate_quad_is_its_triangle():
    # v2 == v3: only triangle (v0,v1,v2) has area
    q = np.array([[0, 0, 1], [1, 0, 1], [1, 1, 1], [1, 1, 1]], dtype=np.float64)
    assert O.intersect_quad([0.7, 0.2, 0.0], [0, 0, 1], q)[0]
    assert not O.intersect_quad([0.2, 0.7, 0.0], [0, 0, 1], q)[0]


# ---------------------------------------------------------------------------
# Scene traversal
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_scene():
    return I.tiny_scene(n_inst=24)


@pytest.fixture(scope="module")
def small_rays(small_scene):
    lo, hi = I.scene_box(small_scene)
    tg = I.instance_origins(small_scene)
    return np.concatenate([
        I.rays_toward(300, lo - 20, hi + 20, tg, 1.5, seed=11),
        I.rays_random(100, lo, hi, seed=12),
        I.rays_focused(100, (50, -120, 50), lo, hi, seed=13),
    ])


def test_bvh_equals_brute_force_exactly(small_scene, small_rays):
    osc = O.OracleScene(small_scene)
    b = osc.trace_closest(small_rays, mode=0)
    f = osc.trace_closest(small_rays, mode=1)
    hits = (f[1] != NONE).mean()
    assert hits > 0.15
    np.testing.assert_array_equal(b[1], f[1])
    np.testing.assert_array_equal(b[2], f[2])
    np.testing.assert_array_equal(b[0], f[0])


def test_instanced_equals_flattened_world_space(small_scene, small_rays):
    """Moving the ray to object space must agree with moving the quads to
    world space: pins the instance transform, its inverse and t sharing."""
    osc = O.OracleScene(small_scene)
    f = osc.trace_closest(small_rays, mode=1)
    w = osc.trace_closest(small_rays, mode=2)
    np.testing.assert_array_equal(f[1], w[1])
    np.testing.assert_array_equal(f[2], w[2])
    m = f[1] != NONE
    np.testing.assert_allclose(f[0][m], w[0][m], rtol=1e-12)


def test_any_hit_is_nonempty_closest(small_scene, small_rays):
    osc = O.OracleScene(small_scene)
    rays = small_rays.copy()
    rays[::3, 7] = 30.0  # some finite tmax values
    c = osc.trace_closest(rays, mode=1)
    for mode in (0, 1):
        occ = osc.trace_any(rays, mode=mode)
        np.testing.assert_array_equal(occ, c[1] != NONE)


def test_closest_tie_break_prefers_smaller_instance():
    # two instances of the same quad at the same place: same t -> smaller id
    v, q = I.plane_mesh(2)
    xf = np.stack([I.IDENTITY_XFORM, I.IDENTITY_XFORM])
    sc = I.Scene([(v, q)], xf, np.zeros(2, dtype=np.uint32))
    osc = O.OracleScene(sc)
    rays = I.ray_array(np.array([[0.3, 0.4, 3.0]]), np.array([[0.0, 0.0, -1.0]]))
    t, inst, prim, _, _ = osc.trace_closest(rays)
    assert inst[0] == 0 and t[0] == 3.0 and prim[0] == 3


# ---------------------------------------------------------------------------
# Camera and sampling
# ---------------------------------------------------------------------------

def test_camera_center_and_corner_closed_form():
    v = I.View(eye=(1.0, 2.0, 3.0), look=(4.0, 6.0, 3.0), up=(0.0, 0.0, 1.0), vfov_deg=60.0,
               w=200, h=100, spp=1)
    o, d = O.camera_ray(v, 100, 50, 0.0, 0.0)
    f = np.array([3.0, 4.0, 0.0]) / 5.0
    assert np.allclose(o, v.eye) and np.allclose(d, f, atol=1e-15)
    o, d = O.camera_ray(v, 0, 0, 0.0, 0.0)
    th = math.tan(math.radians(30.0))
    r = np.cross(f, [0, 0, 1])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    e = f - 2.0 * th * r + th * u
    assert np.allclose(d, e / np.linalg.norm(e), atol=1e-15)
    assert d[2] > 0  # row 0 is the top of the image


def test_cosine_sampling_closed_form_and_moments():
    xi = np.random.default_rng(9).uniform(size=(200000, 2))
    # n = +z: the basis is the identity, the sample is (r cos phi, r sin phi, sqrt(1-xi1))
    for x1, x2 in xi[:50]:
        s = O.sample_cosine([0, 0, 1], x1, x2)
        r = math.sqrt(x1)
        e = [r * math.cos(2 * math.pi * x2), r * math.sin(2 * math.pi * x2), math.sqrt(1 - x1)]
        assert np.allclose(s, e, atol=1e-15)
    rng = np.random.default_rng(10)
    cos1 = []
    for k in range(4000):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        x1, x2 = xi[k]
        s = O.sample_cosine(n, x1, x2)
        assert abs(np.linalg.norm(s) - 1) < 1e-12
        c = float(np.dot(s, n))
        assert abs(c - math.sqrt(1 - x1)) < 1e-12
        cos1.append(c)
    cos1 = np.array(cos1)
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2
    assert abs(cos1.mean() - 2 / 3) < 4 * math.sqrt(1 / 18 / cos1.size)
    assert abs((cos1 ** 2).mean() - 0.5) < 0.01


def test_cosine_sampling_azimuth_uniform():
    # azimuth about n must be uniform: chi-square over 16 bins
    rng = np.random.default_rng(11)
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    xi = rng.uniform(size=(8000, 2))
    ref = np.cross(n, [1.0, 0.0, 0.0])
    ref /= np.linalg.norm(ref)
    ref2 = np.cross(n, ref)
    ang = []
    for x1, x2 in xi:
        s = O.sample_cosine(n, x1, x2)
        ang.append(math.atan2(np.dot(s, ref2), np.dot(s, ref)))
    h, _ = np.histogram(ang, bins=16, range=(-math.pi, math.pi))
    e = len(ang) / 16
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4


# ---------------------------------------------------------------------------
# Path tracing: closed forms and invariants
# ---------------------------------------------------------------------------

def _rot(axis, ang):
    axis = np.asarray(axis, dtype=np.float64)
    axis /= np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _plane_scene():
    """One flat 128x128-quad plane under a sheared (rotate, anisotropic scale, rotate)
    transform, so the world normal needs the inverse transpose."""
    v, q = I.plane_mesh(128)
    A = _rot([0, 0, 1], 0.3) @ np.diag([400.0, 250.0, 3.0]) @ _rot([1, 0.2, 0], 0.7)
    xf = I.pack_xforms(A[None], np.array([[10.0, -5.0, 2.0]]))
    sc = I.Scene([(v, q)], xf, np.zeros(1, dtype=np.uint32))
    A32 = xf.reshape(3, 4)[:, :3].astype(np.float64)
    n_w = np.linalg.inv(A32).T @ np.array([0.0, 0.0, 1.0])
    n_w /= np.linalg.norm(n_w)
    eye = np.array([10.0, -5.0, 2.0]) + 40.0 * n_w
    view = I.View(eye=tuple(eye), look=(10.0, -5.0, 2.0), up=(0.0, 0.0, 1.0), vfov_deg=50.0,
                  w=48, h=40, spp=1)
    return sc, view, n_w


def test_flat_plane_env_and_sun_closed_form():
    sc, view, n_w = _plane_scene()
    osc = O.OracleScene(sc)
    alb = I.albedo(sc.n_quads, seed=21)
    l = np.array([0.2, -0.4, 1.0])
    l /= np.linalg.norm(l)
    cl = float(np.dot(n_w, l))
    assert cl > 0.1
    p = I.Params(max_depth=2, env=(1.0, 1.0, 1.0), sun_dir=tuple(l), sun_E=(3.0, 2.0, 1.0))
    r = osc.render(view, alb, p, log=True)
    q = r["prim"][:, 0]
    assert (r["inst"][:, 0] == 0).all()            # every camera ray hits the plane
    assert (r["inst"][:, 1] == NONE).all()         # every bounce escapes
    assert len(np.unique(q)) > 4
    E = np.array([3.0, 2.0, 1.0])
    expect = alb[q].astype(np.float64) * (1.0 + E * cl / math.pi)
    np.testing.assert_allclose(r["rgb"], expect, rtol=1e-6)  # FP32 sun_dir input
    # no sun: zero variance, exactly the albedo
    p0 = I.Params(max_depth=2, env=(1.0, 1.0, 1.0))
    r0 = osc.render(view, alb, p0, log=True)
    np.testing.assert_array_equal(r0["rgb"], alb[r0["prim"][:, 0]].astype(np.float64))
    # depth 1: only the sun term remains
    p1 = I.Params(max_depth=1, env=(1.0, 1.0, 1.0), sun_dir=tuple(l), sun_E=(3.0, 2.0, 1.0))
    r1 = osc.render(view, alb, p1, log=True)
    np.testing.assert_allclose(r1["rgb"], alb[r1["prim"][:, 0]] * E * cl / math.pi, rtol=1e-6)


def test_sun_below_horizon_gives_no_nee():
    sc, view, n_w = _plane_scene()
    osc = O.OracleScene(sc)
    alb = I.albedo(sc.n_quads, seed=21)
    l = -n_w
    p = I.Params(max_depth=2, env=(1.0, 1.0, 1.0), sun_dir=tuple(l), sun_E=(3.0, 3.0, 3.0))
    r = osc.render(view, alb, p, log=True)
    np.testing.assert_array_equal(r["rgb"], alb[r["prim"][:, 0]].astype(np.float64))
    assert (r["shadow"] == 0).all()


def test_white_furnace_convex_object_is_invisible():
    v, q = I.sphere_mesh(24, 48, 5.0)
    sc = I.Scene([(v, q)], I.IDENTITY_XFORM[None].copy(), np.zeros(1, dtype=np.uint32))
    osc = O.OracleScene(sc)
    view = I.View(eye=(0.0, -30.0, 4.0), look=(0.0, 0.0, 0.0), up=(0, 0, 1), vfov_deg=30.0,
                  w=64, h=64, spp=4)
    ones = np.ones((sc.n_quads, 3), dtype=np.float32)
    p = I.Params(max_depth=256, env=(1.0, 1.0, 1.0))
    r = osc.render(view, ones, p)
    assert r["truncated"] == 0
    np.testing.assert_array_equal(r["rgb"], 1.0)


def test_white_furnace_tiny_scene_counts_truncation():
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w = view.h = 96
    ones = np.ones((sc.n_quads, 3), dtype=np.float32)
    for depth in (3, 64):
        r = osc.render(view, ones, I.Params(max_depth=depth, env=(1.0, 1.0, 1.0)), log=True)
        rgb = r["rgb"][:, 0]
        assert set(np.unique(rgb)) <= {0.0, 1.0}
        assert int((rgb == 0).sum()) == r["truncated"]
        assert int((rgb == 1).sum()) == r["escaped"]
        trunc = (r["inst"][:, -1] != NONE)
        np.testing.assert_array_equal(trunc, rgb == 0)


def test_value_set_invariant_env_only():
    """Env only: each sample is env * prod(albedo of the quads on its path), or 0."""
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w = view.h = 128
    alb = I.albedo(sc.n_quads)
    env = (0.5, 1.0, 2.0)
    r = osc.render(view, alb, I.Params(max_depth=3, env=env), log=True)
    offs = sc.quad_offsets
    expect = np.zeros_like(r["rgb"])
    for k in range(r["rgb"].shape[0]):
        prod = np.ones(3)
        escaped = False
        for i in range(3):
            if r["inst"][k, i] == NONE:
                escaped = True
                break
            row = offs[sc.mesh_ids[r["inst"][k, i]]] + r["prim"][k, i]
            prod *= alb[row]
        if escaped:
            expect[k] = prod * np.array(env)
    np.testing.assert_allclose(r["rgb"], expect, rtol=1e-12, atol=0)
    assert (expect[:, 0] > 0).mean() > 0.5 and (expect[:, 0] < 0.99 * 0.5).any()


def test_render_pixel_subset_matches_full_image():
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w = view.h = 64
    alb = I.albedo(sc.n_quads)
    p = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    full = osc.render(view, alb, p)["rgb"]
    px = np.array([5, 77, 1000, 4095, 2222])
    sub = osc.render(view, alb, p, pixels=px)["rgb"]
    np.testing.assert_array_equal(sub, full[px])


def test_ray_log_follows_the_paths():
    """The oracle's ray log (used to explain divergent GPU paths) records the
    rays its paths trace: depth 1 is the camera ray from the eye; each
    logged hit lies on its logged ray (the quad's FP64 intersection); the
    spawn point of that hit, p + (1e-4 + 1e-5 max|p|) n with n the quad's
    world normal faced against the ray, is logged and starts the next ray;
    a key-light shadow ray leaves it toward a point of one of the lights;
    rays not traced are left zero."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from parity import NONE, world_normal, world_quad
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w, view.h, view.spp = 40, 30, 2
    lights = I.tiny_lights()
    p = I.Params(max_depth=4, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0), lights=lights)
    r = osc.render(view, I.albedo(sc.n_quads), p, log=True, rays=True)
    R = r["rays"]
    assert R.shape == (40 * 30 * 2, 4, 13)
    np.testing.assert_array_equal(R[:, 0, 0:3], np.broadcast_to(np.array(view.eye, float), (2400, 3)))
    np.testing.assert_allclose(np.linalg.norm(R[:, 0, 3:6], axis=1), 1.0, rtol=1e-14)
    l = np.array(I.MID_SUN_DIR, float) / np.linalg.norm(I.MID_SUN_DIR)
    L64 = lights.astype(np.float64)
    checked = shadows = lit = 0
    for k in range(2400):
        for i in range(4):
            inst, prim = r["inst"][k, i], r["prim"][k, i]
            if inst == NONE:
                assert (R[k, i + 1:] == 0).all()
                break
            o, d = R[k, i, 0:3], R[k, i, 3:6]
            hit, t, _, _ = O.intersect_quad(o, d, world_quad(sc, inst, prim))
            assert hit and t > 0
            n = world_normal(sc, inst, prim)
            if n @ d > 0:
                n = -n
            hp = o + t * d
            sp = hp + (1e-4 + 1e-5 * np.abs(hp).max()) * n
            np.testing.assert_allclose(R[k, i, 6:9], sp, rtol=1e-12, atol=1e-12)
            if (r["shadow"][k] >> (2 * i)) & 1:
                assert n @ l > 0
                shadows += 1
            if (r["light"][k] >> (2 * i)) & 1:
                ld, dist = R[k, i, 9:12], R[k, i, 12]
                assert abs(np.linalg.norm(ld) - 1.0) < 1e-12 and dist > 0 and ld @ n > 0
                y = sp + dist * ld
                on = False
                for L in L64:
                    A = np.stack([L[3:6], L[6:9]], 1)
                    st, res, _, _ = np.linalg.lstsq(A, y - L[0:3], rcond=None)
                    if np.abs(A @ st - (y - L[0:3])).max() < 1e-9 and (st > -1e-9).all() and (st < 1 + 1e-9).all():
                        on = True
                assert on
                lit += 1
            else:
                assert (R[k, i, 9:13] == 0).all()
            if i + 1 < 4:
                np.testing.assert_allclose(R[k, i + 1, 0:3], sp, rtol=1e-12, atol=1e-12)
                np.testing.assert_allclose(np.linalg.norm(R[k, i + 1, 3:6]), 1.0, rtol=1e-12)
                assert R[k, i + 1, 3:6] @ n > 0  # leaves on the faced side
            checked += 1
    assert checked > 200 and shadows > 20 and lit > 20


# --------------------------------------------------------------------------
# Per-face textures and key lights (the richer shading of the paper's scene:
# Ptex textures modulating the diffuse albedo, Section 5.3; quad-shaped key
# lights, Section 4.1)
# --------------------------------------------------------------------------
def test_tex_lookup_closed_forms():
    """Bilinear lookup between texel centres, clamped to the face: constant
    and linear texel grids are reproduced exactly; texel centres return the
    texel; outside the centre square the value is the edge's."""
    R = 4
    rng = np.random.default_rng(61)
    tex = rng.uniform(0.2, 1.0, size=(5, R, R, 3)).astype(np.float32)
    # constant grid on quad 2
    tex[2] = np.float32(0.625)
    for u, v in rng.uniform(0.0, 1.0, size=(20, 2)):
        np.testing.assert_allclose(O.tex_lookup(tex, 2, u, v), 0.625, rtol=1e-15)
    # texel centres of quad 3
    for j in range(R):
        for i in range(R):
            np.testing.assert_allclose(O.tex_lookup(tex, 3, (i + 0.5) / R, (j + 0.5) / R),
                                       tex[3, j, i].astype(np.float64), rtol=1e-15)
    # linear grid on quad 4: a + b u + c v at the texel centres
    a, b, c = 0.25, 0.5, 0.125     # exact in FP32
    cu = (np.arange(R) + 0.5) / R
    tex[4] = (a + b * cu[None, :, None] + c * cu[:, None, None]).astype(np.float32)
    for u, v in rng.uniform(0.5 / R, 1.0 - 0.5 / R, size=(20, 2)):
        np.testing.assert_allclose(O.tex_lookup(tex, 4, u, v), a + b * u + c * v, rtol=1e-12)
    # clamped outside the centres: the value at the nearest centre line
    np.testing.assert_allclose(O.tex_lookup(tex, 4, 0.0, 0.5), a + b * 0.5 / R + c * 0.5, rtol=1e-12)
    np.testing.assert_allclose(O.tex_lookup(tex, 4, 1.0, 1.0), a + (b + c) * (1 - 0.5 / R), rtol=1e-12)
    # one texel per face: constant
    np.testing.assert_allclose(O.tex_lookup(tex[:, :1, :1], 1, 0.3, 0.9), tex[1, 0, 0], rtol=1e-15)


def _polygon_irradiance(x, n, verts, L):
    """Irradiance at x (unit normal n) from a uniform Lambertian polygon of
    radiance L lying above x's horizon (Lambert's polygon formula)."""
    r = [(p - x) / np.linalg.norm(p - x) for p in verts]
    tot = 0.0
    for k in range(len(r)):
        a, b = r[k], r[(k + 1) % len(r)]
        g = np.cross(a, b)
        tot += math.acos(np.clip(np.dot(a, b), -1.0, 1.0)) * np.dot(n, g / np.linalg.norm(g))
    return 0.5 * abs(tot) * np.asarray(L, dtype=np.float64)


def test_light_sample_mean_is_the_polygon_irradiance():
    """The key-light estimator Le cos_x cos_l A n / d^2, sampled uniformly
    over the lights, averages to the closed-form irradiance of the
    parallelograms (Lambert's formula), for a light straight above a point,
    a tilted one off to the side, and two lights together (n = 2)."""
    x = np.array([0.3, -0.2, 0.1])
    nx = np.array([0.0, 0.0, 1.0])
    # light 1: square of side 2 at height 3, facing down
    c1, e1, f1 = np.array([-0.7, -1.2, 3.1]), np.array([2.0, 0.0, 0.0]), np.array([0.0, 2.0, 0.0])
    f1, e1 = e1, f1   # e1 x f1 points down
    # light 2: a tilted parallelogram off to the side, facing x
    c2 = np.array([2.0, 1.0, 1.5])
    e2, f2 = np.array([0.0, 1.5, 0.0]), np.array([0.8, 0.0, 0.9])
    if np.dot(np.cross(e2, f2), x - (c2 + 0.5 * e2 + 0.5 * f2)) < 0:
        e2, f2 = f2, e2
    L1, L2 = np.array([4.0, 2.0, 1.0]), np.array([1.0, 3.0, 2.0])
    lights = np.array([np.concatenate([c1, e1, f1, L1]), np.concatenate([c2, e2, f2, L2])], dtype=np.float32)
    l64 = lights.astype(np.float64)
    quad = lambda l: [l[0:3], l[0:3] + l[3:6], l[0:3] + l[3:6] + l[6:9], l[0:3] + l[6:9]]
    E1 = _polygon_irradiance(x, nx, quad(l64[0]), l64[0, 9:12])
    E2 = _polygon_irradiance(x, nx, quad(l64[1]), l64[1, 9:12])
    rng = np.random.default_rng(71)
    xi = rng.uniform(size=(60000, 3))
    for lt, expect in ((lights[:1], E1), (lights[1:], E2), (lights, E1 + E2)):
        acc = np.zeros(3)
        acc2 = np.zeros(3)
        for z in xi:
            ok, d, dist, w = O.light_sample(lt, z, x, nx)
            acc += w
            acc2 += w * w
        m = acc / len(xi)
        se = np.sqrt(np.maximum(acc2 / len(xi) - m * m, 0.0) / len(xi))
        assert (np.abs(m - expect) <= 4 * se + 1e-12).all(), (m, expect, se)
        assert (se < 0.02 * expect).all()


def test_light_sample_facing_away_or_below_horizon_gives_nothing():
    x, nx = np.zeros(3), np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(72)
    up = np.array([[-1.0, -1.0, 2.0, 2.0, 0.0, 0.0, 0.0, 2.0, 0.0, 1.0, 1.0, 1.0]], dtype=np.float32)
    below = np.array([[-1.0, -1.0, -2.0, 2.0, 0.0, 0.0, 0.0, 2.0, 0.0, 1.0, 1.0, 1.0]], dtype=np.float32)
    for z in rng.uniform(size=(200, 3)):
        assert not O.light_sample(up, z, x, nx)[0]      # emits upward, away from x
        assert not O.light_sample(below, z, x, nx)[0]   # under x's horizon
        ok, d, dist, w = O.light_sample(up[:, [0, 1, 2, 6, 7, 8, 3, 4, 5, 9, 10, 11]], z, x, nx)
        assert ok and np.isclose(np.linalg.norm(d), 1.0) and dist > 0  # flipped: faces x


def test_render_constant_face_textures_equal_scaled_albedo():
    """A texture constant over each face multiplies that face's albedo:
    rendering with it equals rendering with the product albedo (paths do not
    depend on albedo), with the sun and several bounces."""
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w, view.h, view.spp = 48, 40, 2
    alb = I.albedo(sc.n_quads)
    k = np.random.default_rng(62).uniform(0.3, 1.0, size=(sc.n_quads, 3)).astype(np.float32)
    tex = np.repeat(np.repeat(k[:, None, None, :], 4, axis=1), 4, axis=2)
    p = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    r_tex = osc.render(view, alb, dataclasses.replace(p, tex=tex))["rgb"]
    r_mul = osc.render(view, (alb.astype(np.float64) * k).astype(np.float32), p)["rgb"]
    ok = r_mul > 0
    assert ok.mean() > 0.2
    np.testing.assert_allclose(r_tex, r_mul, rtol=2e-7)   # the FP32 rounding of the product


def test_render_texture_follows_the_hit_position():
    """A face texture bright on its u < 1/2 texels and dark on the others: on
    the flat plane (env only, depth 2: the bounce always escapes) a pixel's
    radiance is the albedo times the bilinear texture at the hit's
    quad-space u, which the logged hit position reproduces."""
    sc, view, n_w = _plane_scene()
    osc = O.OracleScene(sc)
    alb = np.ones((sc.n_quads, 3), dtype=np.float32)
    tex = np.zeros((sc.n_quads, 2, 2, 3), dtype=np.float32)
    tex[:, :, 0, :] = 1.0          # texels with i = 0 (u < 1/2)
    p = I.Params(max_depth=2, env=(1.0, 1.0, 1.0), tex=tex)
    r = osc.render(view, alb, p, log=True, rays=True)
    assert (r["inst"][:, 1] == NONE).all()
    vals = r["rgb"][:, 0]
    assert (vals > 0.99).mean() > 0.15 and (vals < 0.01).mean() > 0.15   # both halves seen
    # expected value from the hit position in the quad's own parameters
    v, q = I.plane_mesh(128)
    M = sc.xforms[0].reshape(3, 4).astype(np.float64)
    for k in range(0, len(vals), 37):
        o, d = r["rays"][k, 0, 0:3], r["rays"][k, 0, 3:6]
        P = v[q[r["prim"][k, 0]]].astype(np.float64) @ M[:, :3].T + M[:, 3]
        hit, t, u, w = O.intersect_quad(o, d, P)
        assert hit
        s_ = min(max(u * 2 - 0.5, 0.0), 1.0)
        assert abs(vals[k] - (1.0 - s_)) < 1e-9


def test_render_key_light_on_a_plane_is_the_polygon_irradiance():
    """Depth 1 on a flat plane lit only by one key light above the pixel's
    point (no environment, no sun): the radiance is a/pi times the light's
    irradiance there (Lambert's polygon formula), to the Monte Carlo error
    of its samples."""
    v, q = I.plane_mesh(1)
    xf = I.pack_xforms((np.eye(3) * 50.0)[None], np.zeros((1, 3)))
    sc = I.Scene([(v, q)], xf, np.zeros(1, dtype=np.uint32))
    osc = O.OracleScene(sc)
    # a narrow camera straight down at the origin: every sample hits within
    # 1e-3 of it
    view = I.View(eye=(0.0, 0.0, 20.0), look=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), vfov_deg=0.005,
                  w=1, h=1, spp=4096)
    light = np.array([[-1.5, -1.0, 6.0, 0.0, 2.0, 0.0, 3.0, 0.0, 0.0, 8.0, 5.0, 3.0]], dtype=np.float32)
    alb = np.full((1, 3), 0.5, dtype=np.float32)
    p = I.Params(max_depth=1, env=(0.0, 0.0, 0.0), lights=light)
    rgb = osc.render(view, alb, p)["rgb"][0]
    l64 = light[0].astype(np.float64)
    quad = [l64[0:3], l64[0:3] + l64[3:6], l64[0:3] + l64[3:6] + l64[6:9], l64[0:3] + l64[6:9]]
    x = np.array([0.0, 0.0, 1e-4 + 0.0])   # the spawn point above the hit
    E = _polygon_irradiance(x, np.array([0.0, 0.0, 1.0]), quad, l64[9:12])
    np.testing.assert_allclose(rgb, 0.5 / math.pi * E, rtol=3e-3)


def test_gradient_with_textures_and_key_lights_matches_central_differences():
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w = view.h = 48
    view.spp = 2
    alb = I.albedo(sc.n_quads).astype(np.float64)
    p = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(2.0, 2.0, 2.0),
                 tex=I.face_textures(sc.n_quads), lights=I.tiny_lights())
    dimg = np.random.default_rng(6).normal(size=(view.w * view.h, 3))
    g = osc.grad(view, alb.astype(np.float32), p, dimg)
    nz = np.argwhere(np.abs(g) > 1e-3 * np.abs(g).max())
    assert nz.shape[0] > 20
    pick = nz[np.random.default_rng(7).choice(nz.shape[0], 12, replace=False)]
    h = 1.0 / 1024

    def F(a):
        return float((osc.render(view, a.astype(np.float32), p)["rgb"] * dimg).sum())

    a32 = alb.astype(np.float32).astype(np.float64)
    for qq, c in pick:
        ap = a32.copy()
        am = a32.copy()
        ap[qq, c] = np.float32(a32[qq, c] + h)
        am[qq, c] = np.float32(a32[qq, c] - h)
        fd = (F(ap) - F(am)) / (ap[qq, c] - am[qq, c])
        assert abs(fd - g[qq, c]) <= 1e-7 * max(1.0, abs(g[qq, c])), (qq, c, fd, g[qq, c])


def test_progressive_samples_compose_to_one_render():
    """Section 5.4 renders one sample per pixel per frame.  A view's samples
    are drawn at sample_base + k: the mean of frames with spp = 1 and
    sample_base = 0, 1, 2 is the 3-spp render, and a frame is the matching
    sample of it (its path log rows)."""
    import dataclasses
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w = view.h = 32
    view.spp = 3
    alb = I.albedo(sc.n_quads)
    p = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    full = osc.render(view, alb, p, log=True)
    frames = [osc.render(dataclasses.replace(view, spp=1, sample_base=k), alb, p, log=True)
              for k in range(3)]
    acc = (frames[0]["rgb"] + frames[1]["rgb"]) + frames[2]["rgb"]
    np.testing.assert_array_equal(acc / 3.0, full["rgb"])
    for k in range(3):
        np.testing.assert_array_equal(frames[k]["inst"], full["inst"][k::3])
        np.testing.assert_array_equal(frames[k]["prim"], full["prim"][k::3])
    # a different sample index draws a different path somewhere
    assert not np.array_equal(frames[0]["inst"], frames[1]["inst"])


# ---------------------------------------------------------------------------
# Gradient
# ---------------------------------------------------------------------------

def test_gradient_flat_plane_closed_form():
    """On the plane with depth 2, I = a_q (1 + E cos / pi) per sample, so
    dI/da_q = 1 + E cos / pi for the quad each pixel sees."""
    sc, view, n_w = _plane_scene()
    view.spp = 3
    osc = O.OracleScene(sc)
    alb = I.albedo(sc.n_quads, seed=21)
    l = np.array([0.2, -0.4, 1.0])
    l /= np.linalg.norm(l)
    p = I.Params(max_depth=2, env=(1.0, 1.0, 1.0), sun_dir=tuple(l), sun_E=(3.0, 2.0, 1.0))
    r = osc.render(view, alb, p, log=True)
    dimg = np.random.default_rng(3).normal(size=r["rgb"].shape)
    g = osc.grad(view, alb, p, dimg)
    cl = float(np.dot(n_w, l))
    fac = 1.0 + np.array([3.0, 2.0, 1.0]) * cl / math.pi
    expect = np.zeros_like(g)
    q = r["prim"][:, 0].reshape(-1, view.spp)
    for k in range(q.shape[0]):
        for s in range(view.spp):
            expect[q[k, s]] += dimg[k] * fac / view.spp
    np.testing.assert_allclose(g, expect, rtol=1e-6, atol=1e-12)


def test_gradient_matches_central_differences():
    sc = I.tiny_scene()
    osc = O.OracleScene(sc)
    view = I.tiny_view()
    view.w = view.h = 64
    view.spp = 2
    alb = I.albedo(sc.n_quads).astype(np.float64)
    p = I.Params(max_depth=3, sun_dir=I.MID_SUN_DIR, sun_E=(3.0, 3.0, 3.0))
    dimg = np.random.default_rng(4).normal(size=(view.w * view.h, 3))
    g = osc.grad(view, alb.astype(np.float32), p, dimg)
    nz = np.argwhere(np.abs(g) > 1e-3 * np.abs(g).max())
    assert nz.shape[0] > 20
    pick = nz[np.random.default_rng(5).choice(nz.shape[0], 12, replace=False)]
    h = 1.0 / 1024  # the step actually taken is measured after rounding to FP32

    def F(a):
        return float((osc.render(view, a.astype(np.float32), p)["rgb"] * dimg).sum())

    a32 = alb.astype(np.float32).astype(np.float64)
    for q, c in pick:
        ap = a32.copy()
        am = a32.copy()
        ap[q, c] = np.float32(a32[q, c] + h)
        am[q, c] = np.float32(a32[q, c] - h)
        fd = (F(ap) - F(am)) / (ap[q, c] - am[q, c])
        assert abs(fd - g[q, c]) <= 1e-7 * max(1.0, abs(g[q, c])), (q, c, fd, g[q, c])
