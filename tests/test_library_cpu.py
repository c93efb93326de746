"""CPU-only checks of the C ABI library: it loads, exports every symbol the
header declares, rejects bad arguments on the host, and its BVH builder keeps
its invariants.  No GPU call is made here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2001_02620_gb300 import build as B
from paper_2001_02620_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    B.build()
    from paper_2001_02620_gb300 import _native as N
    return N


def _declared():
    src = open(os.path.join(ROOT, "include", "qrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qrt_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for f in ["qrt_scene_create", "qrt_scene_destroy", "qrt_trace_closest", "qrt_trace_any",
              "qrt_render_spp", "qrt_render_adjoint", "qrt_check"]:
        assert f in names


def test_library_exports_every_declared_symbol(native):
    L = C.CDLL(native.LIB_PATH)
    for name in _declared():
        assert hasattr(L, name), name
    # and the binding declares a signature for each of them
    assert sorted(native.SIGNATURES) == _declared()


def test_version_and_error_string(native):
    L = native.lib()
    assert L.qrt_version() == 1
    assert isinstance(L.qrt_last_error(), bytes)


def test_host_side_argument_errors(native):
    L = native.lib()
    # NULL scene handles are rejected before any CUDA call
    assert L.qrt_trace_closest(None, None, 10, None, None, None) == native.QRT_ERR_INVALID_ARG
    assert b"scene" in L.qrt_last_error()
    assert L.qrt_trace_any(None, None, 0, None, None, None) == native.QRT_ERR_INVALID_ARG
    assert L.qrt_render_spp(None, None, 0, None, None, None) == native.QRT_ERR_INVALID_ARG
    assert L.qrt_check(None, None) == native.QRT_ERR_INVALID_ARG
    assert L.qrt_scene_destroy(None) == native.QRT_ERR_INVALID_ARG
    assert L.qrt_graph_launch(None, None) == native.QRT_ERR_INVALID_ARG
    assert L.qrt_l2_loss(None, None, 0, None, None, None) == native.QRT_ERR_INVALID_ARG
    out = C.c_void_p()
    assert L.qrt_scene_create(None, 0, None, None, 0, None, C.byref(out)) == native.QRT_ERR_INVALID_ARG
    # an instance naming a missing mesh is rejected before any device work
    v, q = I.plane_mesh(2)
    m = (native.qrt_mesh * 1)()
    m[0].verts = v.ctypes.data_as(C.POINTER(C.c_float))
    m[0].n_verts = v.shape[0]
    m[0].quads = q.ctypes.data_as(C.POINTER(C.c_uint32))
    m[0].n_quads = q.shape[0]
    xf = np.tile(I.IDENTITY_XFORM, 2)
    ids = np.array([0, 3], dtype=np.uint32)
    rc = L.qrt_scene_create(m, 1, xf.ctypes.data_as(C.POINTER(C.c_float)),
                            ids.ctypes.data_as(C.POINTER(C.c_uint32)), 2, None, C.byref(out))
    assert rc == native.QRT_ERR_INVALID_ARG and b"out of range" in L.qrt_last_error()
    # build options out of range
    ids = np.array([0, 0], dtype=np.uint32)
    o = native.qrt_build_opts()
    o.inst_boxes = 7
    rc = L.qrt_scene_create(m, 1, xf.ctypes.data_as(C.POINTER(C.c_float)),
                            ids.ctypes.data_as(C.POINTER(C.c_uint32)), 2, C.byref(o), C.byref(out))
    assert rc == native.QRT_ERR_INVALID_ARG and b"inst_boxes" in L.qrt_last_error()
    for field, val, word in (("tlas_builder", 3, b"tlas_builder"), ("blas_builder", 3, b"blas_builder")):
        o = native.qrt_build_opts()
        setattr(o, field, val)
        rc = L.qrt_scene_create(m, 1, xf.ctypes.data_as(C.POINTER(C.c_float)),
                                ids.ctypes.data_as(C.POINTER(C.c_uint32)), 2, C.byref(o), C.byref(out))
        assert rc == native.QRT_ERR_INVALID_ARG and word in L.qrt_last_error()
    o = native.qrt_build_opts()
    o.blas_builder, o.degenerate = 2, 1   # the chain-shaped test BLAS exists only on the host builder
    rc = L.qrt_scene_create(m, 1, xf.ctypes.data_as(C.POINTER(C.c_float)),
                            ids.ctypes.data_as(C.POINTER(C.c_uint32)), 2, C.byref(o), C.byref(out))
    assert rc == native.QRT_ERR_INVALID_ARG and b"degenerate" in L.qrt_last_error()
    # a singular instance transform is found by the host build (no GPU needed)
    xs = xf.copy()
    xs[12:24] = [1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0]
    rc = L.qrt_scene_create(m, 1, xs.ctypes.data_as(C.POINTER(C.c_float)),
                            ids.ctypes.data_as(C.POINTER(C.c_uint32)), 2, None, C.byref(out))
    assert rc == native.QRT_ERR_INVALID_ARG and b"instance 1" in L.qrt_last_error()
    assert b"singular" in L.qrt_last_error()


def _check_mesh(native, v, q, **opts):
    L = native.lib()
    m = native.qrt_mesh()
    v = np.ascontiguousarray(v, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.uint32)
    m.verts = v.ctypes.data_as(C.POINTER(C.c_float))
    m.n_verts = v.shape[0]
    m.quads = q.ctypes.data_as(C.POINTER(C.c_uint32))
    m.n_quads = q.shape[0]
    o = native.qrt_build_opts()
    for k, val in opts.items():
        setattr(o, k, val)
    n = C.c_uint64()
    d = C.c_uint32()
    rc = L.qrt_blas_build_check(C.byref(m), C.byref(o), C.byref(n), C.byref(d))
    return rc, n.value, d.value, L.qrt_last_error().decode()


@pytest.mark.parametrize("leaf", [1, 2, 4, 8])
def test_blas_invariants_tiny_mesh(native, leaf):
    v, q = I.tiny_mesh()
    rc, n, d, msg = _check_mesh(native, v, q, max_leaf=leaf)
    assert rc == 0, msg
    assert n >= q.shape[0] / (leaf * 4)
    assert d < 20


def test_blas_invariants_varied_meshes(native):
    rng = np.random.default_rng(3)
    meshes = [I.displaced_grid(rng, 5000), I.noisy_blob(rng, 3000), I.sphere_mesh(10, 20),
              I.plane_mesh(1), I.plane_mesh(3)]
    # extreme coordinates: far from the origin and tiny extents
    v, q = I.plane_mesh(16)
    meshes.append((v * np.float32(1e-6) + np.float32(3e4), q))
    meshes.append((v * np.float32(1e5), q))
    # all quads coincident (zero centroid extent)
    vv = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    meshes.append((vv, np.tile(np.array([[0, 1, 2, 3]], dtype=np.uint32), (50, 1))))
    for v, q in meshes:
        rc, n, d, msg = _check_mesh(native, v, q)
        assert rc == 0, msg


def test_parallel_build_gives_the_same_tree(native):
    """Large subtrees are built by helper threads; the tree must not depend
    on how many: node count and depth (and the invariant check) agree for 1
    and 8 threads on meshes large enough to fork."""
    rng = np.random.default_rng(5)
    for v, q in [I.displaced_grid(rng, 300_000), I.noisy_blob(rng, 200_000)]:
        r1 = _check_mesh(native, v, q, threads=1)
        r8 = _check_mesh(native, v, q, threads=8)
        assert r1[0] == 0 and r8[0] == 0, (r1[3], r8[3])
        assert r1[1:3] == r8[1:3]


def test_blas_degenerate_chain_is_deep(native):
    vv = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    q = np.tile(np.array([[0, 1, 2, 3]], dtype=np.uint32), (300, 1))
    rc, n, d, msg = _check_mesh(native, vv, q, degenerate=1)
    assert rc == 0, msg
    assert d >= 90


def test_blas_rejects_bad_meshes(native):
    v, q = I.plane_mesh(2)
    bad = q.copy()
    bad[0, 0] = 999
    rc, *_, msg = _check_mesh(native, v, bad)
    assert rc == native.QRT_ERR_INVALID_ARG and "out of range" in msg
    vn = v.copy()
    vn[0, 0] = np.nan
    rc, *_, msg = _check_mesh(native, vn, q)
    assert rc == native.QRT_ERR_INVALID_ARG and "non-finite" in msg


def _check_tlas(native, boxes, builder):
    L = native.lib()
    b = np.ascontiguousarray(boxes, dtype=np.float32)
    o = native.qrt_build_opts()
    o.tlas_builder = builder
    n = C.c_uint64()
    d = C.c_uint32()
    rc = L.qrt_tlas_build_check(b.ctypes.data, b.shape[0], C.byref(o), C.byref(n), C.byref(d))
    return rc, n.value, d.value, L.qrt_last_error().decode()


def _random_boxes(rng, n, spread=100.0, size=5.0):
    c = rng.uniform(-spread, spread, size=(n, 3))
    e = rng.uniform(0.1, size, size=(n, 3))
    return np.concatenate([c - e, c + e], axis=1)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 17, 1000, 100000])
def test_linear_tlas_invariants_on_host(native, n):
    """The linear-BVH TLAS steps (Morton order, radix-tree nodes, bottom-up
    boxes, four-wide collapse, quantisation), run on the host: every instance
    referenced once and every quantised child box containing its subtree."""
    boxes = _random_boxes(np.random.default_rng(n), n)
    rc, nodes, depth, msg = _check_tlas(native, boxes, 2)
    assert rc == 0, msg
    assert 1 <= nodes <= max(1, n - 1)
    assert depth >= int(np.ceil(np.log(max(n, 2)) / np.log(4)))
    assert depth <= 3 * int(np.ceil(np.log2(max(n, 2)))) + 2
    rc0, nodes0, _, msg0 = _check_tlas(native, boxes, 0)   # the SAH builder on the same boxes
    assert rc0 == 0, msg0


def test_linear_tlas_degenerate_inputs_on_host(native):
    rng = np.random.default_rng(7)
    cases = {
        # equal Morton keys everywhere: positions break the ties
        "identical": np.tile(np.array([[0, 0, 0, 1, 1, 1]], np.float32), (1000, 1)),
        # zero centre extent on two axes
        "line": np.stack([np.arange(5000.0), np.zeros(5000), np.zeros(5000),
                          np.arange(5000.0) + 0.5, np.zeros(5000), np.zeros(5000)], axis=1),
        # far from the origin, tiny extents
        "far": _random_boxes(rng, 1000) * 1e-6 + 3e4,
        # huge spread, heavy overlap
        "wide": _random_boxes(rng, 20000, spread=1e6, size=1e5),
        # points (zero-volume boxes)
        "points": np.repeat(rng.uniform(-10, 10, size=(3000, 3)), 2, axis=1).reshape(3000, 6)[:, [0, 2, 4, 1, 3, 5]],
    }
    for name, boxes in cases.items():
        rc, nodes, depth, msg = _check_tlas(native, boxes, 2)
        assert rc == 0, (name, msg)
        assert nodes <= boxes.shape[0] - 1, name


def test_linear_tlas_rejects_bad_input_on_host(native):
    boxes = _random_boxes(np.random.default_rng(1), 10)
    bad = boxes.copy()
    bad[3, 2] = np.nan
    assert _check_tlas(native, bad, 2)[0] == native.QRT_ERR_INVALID_ARG
    inverted = boxes.copy()
    inverted[4, 0], inverted[4, 3] = 5.0, -5.0
    assert _check_tlas(native, inverted, 2)[0] == native.QRT_ERR_INVALID_ARG
    assert _check_tlas(native, boxes, 3)[0] == native.QRT_ERR_INVALID_ARG
    rc, nodes, depth, _ = _check_tlas(native, boxes[:0], 2)
    assert rc == 0 and nodes == 0


def _varied_meshes():
    rng = np.random.default_rng(3)
    meshes = [I.tiny_mesh(), I.displaced_grid(rng, 5000), I.noisy_blob(rng, 3000),
              I.sphere_mesh(10, 20), I.plane_mesh(1), I.plane_mesh(3)]
    v, q = I.plane_mesh(16)
    meshes.append((v * np.float32(1e-6) + np.float32(3e4), q))   # far away, tiny
    meshes.append((v * np.float32(1e5), q))                       # huge
    vv = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    meshes.append((vv, np.tile(np.array([[0, 1, 2, 3]], dtype=np.uint32), (50, 1))))  # coincident
    return meshes


def _check_meshes(native, meshes, **opts):
    L = native.lib()
    arr = (native.qrt_mesh * len(meshes))()
    keep = []
    for k, (v, q) in enumerate(meshes):
        v = np.ascontiguousarray(v, dtype=np.float32)
        q = np.ascontiguousarray(q, dtype=np.uint32)
        keep += [v, q]
        arr[k].verts = v.ctypes.data_as(C.POINTER(C.c_float))
        arr[k].n_verts = v.shape[0]
        arr[k].quads = q.ctypes.data_as(C.POINTER(C.c_uint32))
        arr[k].n_quads = q.shape[0]
    o = native.qrt_build_opts()
    for k, val in opts.items():
        setattr(o, k, val)
    n = C.c_uint64()
    d = C.c_uint32()
    rc = L.qrt_blases_build_check(arr, len(meshes), C.byref(o), C.byref(n), C.byref(d))
    return rc, n.value, d.value, L.qrt_last_error().decode()


@pytest.mark.parametrize("leaf", [1, 4, 8])
def test_linear_blas_invariants_on_host(native, leaf):
    """The linear-BVH BLAS steps run on the host, one mesh at a time and all
    meshes in one pass (mesh subtrees of one radix tree): every quad in one
    slot, every quantised box containing its subtree, any leaf size."""
    for v, q in _varied_meshes():
        rc, n, d, msg = _check_mesh(native, v, q, max_leaf=leaf, blas_builder=2)
        assert rc == 0, msg
        assert n >= 1 and d >= 1
    rc, n, d, msg = _check_meshes(native, _varied_meshes(), max_leaf=leaf, blas_builder=2)
    assert rc == 0, msg


def test_linear_blas_many_meshes_on_host(native):
    """The mid scene's 128 prototype meshes in one pass: each mesh's subtree is
    found and checked; node counts stay close to the SAH builder's."""
    sc = I.mid_scene()
    rc, n, d, msg = _check_meshes(native, sc.meshes, blas_builder=2)
    assert rc == 0, msg
    rc0, n0, d0, msg0 = _check_meshes(native, sc.meshes)
    assert rc0 == 0, msg0
    assert 0.7 * n0 <= n <= 1.3 * n0


def test_linear_blas_rejects_bad_input_on_host(native):
    v, q = I.plane_mesh(2)
    bad = q.copy()
    bad[1, 2] = v.shape[0]
    assert _check_meshes(native, [(v, q), (v, bad)], blas_builder=2)[0] == native.QRT_ERR_INVALID_ARG
    vn = v.copy()
    vn[0, 1] = np.inf
    assert _check_meshes(native, [(vn, q)], blas_builder=2)[0] == native.QRT_ERR_INVALID_ARG
    assert _check_meshes(native, [(v, q)], blas_builder=3)[0] == native.QRT_ERR_INVALID_ARG
    assert _check_mesh(native, v, q[:0], blas_builder=2)[0] == native.QRT_ERR_INVALID_ARG


def test_linear_tlas_random_layouts_on_host(native):
    """Random counts, spreads, sizes and clustering (many equal Morton codes):
    the host-run linear TLAS always passes the invariant check."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(n=st.integers(1, 3000), spread=st.floats(1e-3, 1e6), size=st.floats(0.0, 10.0),
               clusters=st.integers(1, 8), seed=st.integers(0, 2**31 - 1))
    def run(n, spread, size, clusters, seed):
        rng = np.random.default_rng(seed)
        centres = rng.uniform(-spread, spread, size=(clusters, 3))
        c = centres[rng.integers(0, clusters, size=n)] + rng.normal(0, spread * 1e-3, size=(n, 3))
        e = rng.uniform(0, size * spread * 1e-3 + 1e-6, size=(n, 3))
        boxes = np.concatenate([c - e, c + e], axis=1)
        rc, nodes, depth, msg = _check_tlas(native, boxes, 2)
        assert rc == 0, msg
        assert nodes <= max(1, n - 1)

    run()


def test_linear_blas_random_meshes_on_host(native):
    """Random mesh sets (counts, sizes, vertex sharing, coincident quads): the
    host-run linear BLASes, all meshes in one pass, pass the invariant check."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None)
    @hyp.given(n_mesh=st.integers(1, 12), max_q=st.integers(1, 600), scale=st.floats(1e-3, 1e5),
               leaf=st.integers(1, 8), seed=st.integers(0, 2**31 - 1))
    def run(n_mesh, max_q, scale, leaf, seed):
        rng = np.random.default_rng(seed)
        meshes = []
        for _ in range(n_mesh):
            nq = int(rng.integers(1, max_q + 1))
            nv = int(rng.integers(1, 4 * nq + 1))
            v = (rng.normal(size=(nv, 3)) * scale).astype(np.float32)
            q = rng.integers(0, nv, size=(nq, 4)).astype(np.uint32)
            meshes.append((v, q))
        rc, n, d, msg = _check_meshes(native, meshes, blas_builder=2, max_leaf=leaf)
        assert rc == 0, msg

    run()
