"""The device radix sort behind the linear BVH builds (qrt_test_sort_pairs):
a stable sort of (64-bit key, 32-bit value) pairs by the key's low end_bit
bits.  numpy's stable argsort is the definition it is checked against,
bit for bit, on sizes around the 2048-item tile (empty, one item, a ragged
last tile, several tiles), on keys where every digit varies, where only a
few digits vary (passes skipped), where all keys are equal (no pass), with
many duplicates (stability), with bits at and above end_bit that must not
take part in the order, and on Morton codes like the builders' own."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_02620_gb300 import build as B
    B.build()
    from paper_2001_02620_gb300 import _native as N
    return N


def _morton3(x, y, z):
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
        out = np.zeros_like(v)
        for b in range(21):
            out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
        return out
    return spread(x) | (spread(y) << np.uint64(1)) | (spread(z) << np.uint64(2))


def _keys(kind, n, rng):
    if kind == "random":
        return rng.integers(0, 2**64 - 1, n, dtype=np.uint64, endpoint=True)
    if kind == "duplicates":
        return rng.integers(0, 5, n).astype(np.uint64) << np.uint64(37)
    if kind == "equal":
        return np.full(n, 0x123456789, dtype=np.uint64)
    if kind == "top_digit":
        return (rng.integers(0, 256, n).astype(np.uint64) << np.uint64(48)) | np.uint64(3)
    if kind == "morton":
        p = rng.integers(0, 2**21, (3, n))
        # clustered: half the points in a small corner, as instanced scenes are
        p[:, : n // 2] //= 1024
        return _morton3(p[0], p[1], p[2])
    raise ValueError(kind)


def _sort(N, keys, vals, end_bit):
    n = keys.shape[0]
    ko = np.empty_like(keys)
    vo = np.empty_like(vals)
    rc = N.lib().qrt_test_sort_pairs(keys.ctypes.data, vals.ctypes.data, n, end_bit,
                                     ko.ctypes.data, vo.ctypes.data)
    N.check(rc)
    return ko, vo


@pytest.mark.parametrize("n", [0, 1, 7, 2047, 2048, 2049, 100_003, 3_000_001])
@pytest.mark.parametrize("kind", ["random", "duplicates", "equal", "top_digit", "morton"])
@pytest.mark.parametrize("end_bit", [63, 64])
def test_sort_pairs_matches_stable_argsort(N, n, kind, end_bit):
    rng = np.random.default_rng(n * 7 + end_bit)
    keys = _keys(kind, n, rng)
    vals = rng.integers(0, 2**32 - 1, n, dtype=np.uint32, endpoint=True)
    mask = np.uint64(2**64 - 1) if end_bit == 64 else np.uint64((1 << end_bit) - 1)
    perm = np.argsort(keys & mask, kind="stable")
    ko, vo = _sort(N, keys.copy(), vals.copy(), end_bit)
    np.testing.assert_array_equal(ko, keys[perm])
    np.testing.assert_array_equal(vo, vals[perm])


@pytest.mark.parametrize("end_bit", [0, 5, 17, 40])
def test_sort_pairs_partial_key_bits(N, end_bit):
    """Only bits below end_bit order the pairs (a last digit narrower than
    eight bits included); the rest of each key is carried along."""
    rng = np.random.default_rng(end_bit)
    n = 50_000
    keys = rng.integers(0, 2**64 - 1, n, dtype=np.uint64, endpoint=True)
    vals = np.arange(n, dtype=np.uint32)
    mask = np.uint64((1 << end_bit) - 1)
    perm = np.argsort(keys & mask, kind="stable")
    ko, vo = _sort(N, keys.copy(), vals.copy(), end_bit)
    np.testing.assert_array_equal(ko, keys[perm])
    np.testing.assert_array_equal(vo, vals[perm])


def test_sort_pairs_rejects_bad_arguments(N):
    k = np.zeros(4, dtype=np.uint64)
    v = np.zeros(4, dtype=np.uint32)
    L = N.lib()
    assert L.qrt_test_sort_pairs(k.ctypes.data, v.ctypes.data, 4, 65, k.ctypes.data,
                                 v.ctypes.data) == N.QRT_ERR_INVALID_ARG
    assert L.qrt_test_sort_pairs(None, v.ctypes.data, 4, 63, k.ctypes.data,
                                 v.ctypes.data) == N.QRT_ERR_INVALID_ARG
    assert L.qrt_test_sort_pairs(k.ctypes.data, v.ctypes.data, 2**32, 63, k.ctypes.data,
                                 v.ctypes.data) == N.QRT_ERR_INVALID_ARG
