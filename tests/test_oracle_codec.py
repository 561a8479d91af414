"""Pins of the oracle codec (CPU only).

The paper stores checkpoints with a fixed-tolerance lossy compressor, an
absolute point-wise bound (Sec. 2.2 "Lossy Compression").  The oracle codec
is pinned by: hand-derived streams (tests/golden/codec_streams.txt), the
definition of negabinary, exact invertibility and the stated properties of
the lifting step, the bound |x - x_hat| <= tol on every value of every
block, exact round trips where the specification promises them, and error
reporting.
"""
import ctypes
import os

import numpy as np
import pytest

from oracle import codec as C
from oracle import propagator as O
from oracle._lib import lib

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "codec_streams.txt")


def _golden():
    out, cur = [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "name":
                cur = {"name": rest}
                out.append(cur)
            elif key == "values":
                cur["values"] = np.array([float(v) for v in rest.split()], dtype=np.float32)
            elif key == "tol":
                cur["tol"] = float(rest)
            elif key == "bits":
                cur["bits"] = [int(v) for v in rest.split()]
    return out


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_golden_stream(case):
    x = case["values"].reshape(4, 4)
    st, nf = C.compress(x, case["tol"])
    assert not nf
    # container: 16 header words, 1 chunk offset, 1 size word, payload
    assert st[0] == 0x31435442 and st[5] == 1 and st[6] == 1 and st[16] == 0
    nbits = int(st[17] & 0xFFFF)
    assert nbits == len(case["bits"])
    payload = st[18:]
    got = [(int(payload[k >> 5]) >> (k & 31)) & 1 for k in range(nbits)]
    assert got == case["bits"]
    # unused bits of the last word are zero
    assert int(payload[-1]) >> (nbits & 31) == 0 or nbits % 32 == 0
    y = C.decompress(st, (4, 4))
    assert np.all(np.abs(y - x) <= case["tol"])


def _nega(c):
    L = lib()
    L.codec_nega.argtypes = [ctypes.c_int32]
    L.codec_nega.restype = ctypes.c_uint32
    return L.codec_nega(int(c))


def test_negabinary_definition():
    rng = np.random.default_rng(1)
    for c in list(rng.integers(-2 ** 30, 2 ** 30, 300)) + [0, 1, -1, 2, -2, 2 ** 30, -2 ** 30]:
        n = _nega(int(c))
        val = sum(((n >> k) & 1) * (-2) ** k for k in range(32))
        assert val == c


def _lift(v, inverse):
    a = (ctypes.c_int32 * 4)(*[int(t) for t in v])
    lib().codec_lift4.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib().codec_lift4(ctypes.cast(a, ctypes.c_void_p), 1 if inverse else 0)
    return list(a)


def test_lifting_properties():
    # constant -> (c, 0, 0, 0); linear ramp -> residuals zero
    assert _lift([7, 7, 7, 7], False) == [7, 0, 0, 0]
    S, D, d1, d3 = _lift([10, 13, 16, 19], False)
    assert (D, d1, d3) == (6, 0, 0) and S == 13
    # quadratic: second differences show up in the residuals
    assert _lift([0, 1, 4, 9], False)[2:] == [1 - 2, 9 - 8 + 1]
    rng = np.random.default_rng(2)
    for _ in range(500):
        v = [int(t) for t in rng.integers(-2 ** 24 + 1, 2 ** 24, 4)]
        assert _lift(_lift(v, False), True) == v


@pytest.mark.parametrize("dims", [2, 3])
def test_block_transform_invertible_and_bounded(dims):
    V = 64 if dims == 3 else 16
    lib().codec_xform.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    rng = np.random.default_rng(3)
    for trial in range(200):
        if trial % 2:
            v = rng.integers(-2 ** 24 + 1, 2 ** 24, V).astype(np.int32)
        else:
            v = (rng.choice([-1, 1], V) * (2 ** 24 - 1)).astype(np.int32)
        b = v.copy()
        lib().codec_xform(b.ctypes.data_as(ctypes.c_void_p), dims, 0)
        assert np.abs(b.astype(np.int64)).max() < 2 ** 30
        lib().codec_xform(b.ctypes.data_as(ctypes.c_void_p), dims, 1)
        assert np.array_equal(b, v)


def test_sequency_order():
    perm = (ctypes.c_int * 64)()
    lib().codec_order.argtypes = [ctypes.c_int, ctypes.c_void_p]
    lib().codec_order(3, ctypes.cast(perm, ctypes.c_void_p))
    keys = [((i // 16) + (i // 4) % 4 + i % 4, i // 16, (i // 4) % 4, i % 4) for i in perm]
    assert keys == sorted(keys) and sorted(perm) == list(range(64))
    assert list(perm[:4]) == [0, 1, 4, 16]


def _fields():
    rng = np.random.default_rng(4)
    yield "noise3d", rng.standard_normal((9, 10, 11)).astype(np.float32)
    z, y, x = np.meshgrid(*[np.linspace(0, 3, n) for n in (13, 17, 21)], indexing="ij")
    yield "smooth3d", (np.sin(2 * z) * np.cos(3 * y) * np.exp(-x) * 1e-3).astype(np.float32)
    yield "noise2d", (rng.standard_normal((37, 29)) * 50).astype(np.float32)
    w = rng.standard_normal((16, 16, 16)).astype(np.float32)
    w *= np.float32(10.0) ** rng.integers(-20, 5, w.shape)
    yield "range3d", w.astype(np.float32)
    yield "tiny3d", np.full((3, 2, 5), 1e-30, np.float32)


@pytest.mark.parametrize("name,x", list(_fields()), ids=[n for n, _ in _fields()])
@pytest.mark.parametrize("rel", [1e-1, 1e-3, 1e-5, 1e-7])
def test_pointwise_bound_every_block(name, x, rel):
    tol = max(rel * float(np.abs(x).max()), 2.0 ** -80)
    st, nf = C.compress(x, tol)
    assert not nf
    y = C.decompress(st, x.shape)
    assert np.all(np.abs(y.astype(np.float64) - x.astype(np.float64)) <= tol)


def test_bound_on_wavefield_and_ratio_grows_with_tol():
    g = O.Grid(3, (40, 44, 48), 8, 15.0, 8, 1.0, 160, 4.5)
    vel = np.full(g.shape, 2.5)
    s = O.ricker(g.nt, 1.0, 0.02)
    _, u = O.forward(g, vel, [[60.0, 200.0, 230.0]], s, [[0.0, 0.0, 0.0]], want_final=True)
    u = u.astype(np.float32)
    ratios = []
    for rel in (1e-2, 1e-3, 1e-4, 1e-5):
        tol = rel * float(np.abs(u).max())
        st, _ = C.compress(u, tol)
        y = C.decompress(st, u.shape)
        assert np.all(np.abs(y.astype(np.float64) - u) <= tol)
        ratios.append(C.ratio(st, u.shape))
    assert all(a > b for a, b in zip(ratios, ratios[1:])), ratios
    assert ratios[0] > 4


def test_exact_when_lowest_plane_reached():
    # equal exponents and T = 3 -> start plane 0 -> integers exact -> x_hat == x
    rng = np.random.default_rng(7)
    x = (1.0 + rng.random((8, 8, 8))).astype(np.float32)          # all in [1, 2)
    tol = 3.5 * 2.0 ** -23
    st, _ = C.compress(x, tol)
    stats = C.block_stats(st, x.shape)
    assert np.all(stats[:, 1] == 1) and np.all(stats[:, 3] == 0)
    assert np.array_equal(C.decompress(st, x.shape), x)


def test_raw_blocks_are_bit_exact():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((5, 6, 7)).astype(np.float32)
    x[0, 0, 0] = -0.0
    st, _ = C.compress(x, 2.0 ** -85)
    stats = C.block_stats(st, x.shape)
    assert np.all(stats[:, 1] == 2)
    y = C.decompress(st, x.shape)
    assert np.array_equal(y.view(np.uint32), x.view(np.uint32))


def test_zero_field_and_nonfinite_flag():
    x = np.zeros((8, 8, 8), np.float32)
    st, nf = C.compress(x, 1e-6)
    assert not nf and np.all(C.block_stats(st, x.shape)[:, 0] == 1)
    assert np.array_equal(C.decompress(st, x.shape), x)
    x[3, 4, 5] = np.nan
    _, nf = C.compress(x, 1e-6)
    assert nf


def test_corrupt_stream_detected():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((8, 8, 12)).astype(np.float32)
    st, _ = C.compress(x, 1e-3)
    bad = st.copy()
    bad[0] ^= 1
    with pytest.raises(ValueError, match="CORRUPT"):
        C.decompress(bad, x.shape)
    bad = st.copy()
    bad[16 + int(st[6])] += 1          # first block size off by one
    with pytest.raises(ValueError, match="CORRUPT"):
        C.decompress(bad, x.shape)


def test_invalid_tolerance_rejected():
    with pytest.raises(ValueError):
        C.compress(np.ones((4, 4), np.float32), 0.0)
    with pytest.raises(ValueError):
        C.compress(np.ones((4, 4), np.float32), 2.0 ** -95)


def test_coded_stream_never_longer_than_raw():
    # a checkerboard of near-maximal values plus noise: the lifting grows the
    # highest-sequency coefficient to ~2^30, so with a tight tolerance the
    # coded form would need ~32 planes of 64 bits -- the block is stored raw
    rng = np.random.default_rng(12)
    z, y, x = np.meshgrid(*[np.arange(8)] * 3, indexing="ij")
    cb = np.where((z + y + x) % 2 == 0, 1.99, -1.99)
    xf = (cb + 1e-3 * rng.standard_normal(cb.shape)).astype(np.float32)
    st, _ = C.compress(xf, 4.0 * 2.0 ** -23)
    stats = C.block_stats(st, xf.shape)
    assert np.all(stats[:, 0] <= 2 + 32 * 64)
    assert np.any(stats[:, 1] == 2)
    y_ = C.decompress(st, xf.shape)
    assert np.all(np.abs(y_.astype(np.float64) - xf) <= 4.0 * 2.0 ** -23)
