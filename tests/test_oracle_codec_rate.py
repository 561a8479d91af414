"""Pins of the oracle codec's fixed-rate mode (CPU only).

Sec. 2.2 lists ZFP's fixed-rate mode (a guaranteed size, no error bound)
beside the fixed-tolerance mode the paper uses.  The codec's fixed-rate mode
codes the fixed-accuracy mode's integer coefficients plane by plane into a
budget of ceil(R 4^d / 32) words per block.  Facts that fix it:
  * the size is the formula's for any input;
  * a hand-derived stream of a constant block (tests/golden: none needed,
    the bits are derived below);
  * the code is embedded: a larger rate extends every block's bits;
  * after its header, a block's bits are the fixed-accuracy mode's plane
    coding (a different code path, pinned by its own golden streams);
  * with room for every plane the integers come back exactly;
  * the error falls with the rate.
"""
import numpy as np
import pytest

from oracle import codec as C


def _bits(words, n):
    w = np.asarray(words, dtype=np.uint64)
    return [int((w[k >> 5] >> np.uint64(k & 31)) & np.uint64(1)) for k in range(n)]


def _nblocks(shape):
    return int(np.prod([(n + 3) // 4 for n in shape]))


@pytest.mark.parametrize("shape", [(13, 18, 21), (4, 4, 4), (9, 1, 30), (17, 22)])
@pytest.mark.parametrize("rate", [1, 3, 8, 16, 32])
def test_size_is_fixed(shape, rate):
    dims = len(shape)
    V = 64 if dims == 3 else 16
    W = (rate * V + 31) // 32
    want = 16 + _nblocks(shape) * W
    rng = np.random.default_rng(rate)
    for x in (np.zeros(shape), rng.standard_normal(shape) * 1e3, np.full(shape, np.nan)):
        s, flag = C.compress_rate(x.astype(np.float32), rate)
        assert len(s) == want == C.rate_words(shape, dims, rate)
        assert flag == bool(np.isnan(x).any())


def test_constant_block_hand_derived():
    # 4x4x4 block of 1.0: Emax = 0, every integer 2^23; lifting leaves only
    # the first coefficient (2^23), whose negabinary form is 0x01800000
    # (planes 24 and 23).  Bits: 1 | 127 (8) | ptop 24 (5) | plane 24:
    # group test 1, coefficient bit 1 (s = 1), group test 0 | plane 23:
    # verbatim 1, group test 0 | planes 22..0: verbatim 0, group test 0.
    bits = [1] + [1, 1, 1, 1, 1, 1, 1, 0] + [0, 0, 0, 1, 1] + [1, 1, 0] + [1, 0] + [0, 0] * 23
    assert len(bits) == 65
    x = np.ones((4, 4, 4), np.float32)
    for rate, budget in ((1, 64), (2, 128)):
        s, _ = C.compress_rate(x, rate)
        got = _bits(s[16:], budget)
        want = (bits + [0] * budget)[:budget]
        assert got == want
        assert np.array_equal(C.decompress(s, x.shape), x)   # the dropped bit is a zero group test


def test_embedded_code():
    rng = np.random.default_rng(3)
    x = np.cumsum(rng.standard_normal((8, 12, 16)), axis=2).astype(np.float32)
    nb = _nblocks(x.shape)
    prev = None
    for rate in (1, 2, 5, 8, 13, 21, 32):
        s, _ = C.compress_rate(x, rate)
        W = 2 * rate
        blocks = s[16:].reshape(nb, W)
        if prev is not None:
            pr, pW = prev
            for b in range(nb):
                assert _bits(blocks[b], 32 * pW) == _bits(pr[b], 32 * pW)
        prev = (blocks, W)


def test_planes_are_the_fixed_accuracy_coding():
    # a block whose fixed-accuracy stream reaches plane 0 (tolerance below
    # the integer step) holds the same plane bits after its 20-bit header
    # (1, 0, Emax, ptop, pbot) as the fixed-rate block after its 14 bits
    # (1, Emax, ptop)
    rng = np.random.default_rng(5)
    for dims, shape in ((3, (4, 4, 4)), (2, (4, 4))):
        for k in range(20):
            x = (np.cumsum(rng.standard_normal(shape), axis=-1) * 2.0 ** rng.integers(-20, 20)).astype(np.float32)
            emax = int(np.floor(np.log2(np.abs(x).max())))
            fa, _ = C.compress(x, 2.0 ** (emax - 23) * 3.0)
            st = C.block_stats(fa, shape)
            if st[0, 1] != 1 or st[0, 3] != 0:
                continue
            nfa = int(st[0, 0])
            pay = fa[len(fa) - int(fa[7]):]
            fr, _ = C.compress_rate(x, 32)
            ab = _bits(pay, nfa)
            rb = _bits(fr[16:], 32 * len(fr[16:]))
            assert ab[0] == 1 and ab[1] == 0 and rb[0] == 1
            assert ab[2:15] == rb[1:14]                 # Emax and ptop
            L = nfa - 20
            if L <= len(rb) - 14:
                assert rb[14:14 + L] == ab[20:20 + L]


def test_exact_integers_with_room_for_every_plane():
    # a linear ramp leaves two non-zero coefficients: 32 bits per value
    # hold every plane, so the integers (and here the values) come back
    x = (np.arange(64, dtype=np.float32).reshape(4, 4, 4) * 0.25 + 3.0)
    s, _ = C.compress_rate(x, 32)
    assert np.array_equal(C.decompress(s, x.shape), x)


def test_error_falls_with_rate():
    rng = np.random.default_rng(11)
    x = np.cumsum(np.cumsum(rng.standard_normal((20, 24, 28)), 0), 2).astype(np.float32)
    errs = []
    for rate in (4, 8, 12, 16, 20, 24):
        s, _ = C.compress_rate(x, rate)
        errs.append(float(np.abs(C.decompress(s, x.shape) - x).max()))
    assert all(b < a / 4 for a, b in zip(errs, errs[1:])), errs


def test_zero_nonfinite_and_tiny_blocks():
    x = np.zeros((8, 8, 8), np.float32)
    x[0, 0, 0] = np.inf
    x[4:, 4:, 4:] = 2.0 ** -101          # below the flush level
    x[4:, :4, :4] = 1.5
    s, flag = C.compress_rate(x, 4)
    assert flag
    y = C.decompress(s, x.shape)
    assert np.all(y[:4, :4, :4] == 0) and np.all(y[4:, 4:, 4:] == 0)
    assert np.array_equal(y[4:, :4, :4], x[4:, :4, :4])
    blocks = s[16:].reshape(8, 8)
    for b in (0, 7):                     # zero-coded blocks: a single 0 bit, then zeros
        assert not blocks[b].any()


def test_invalid_rate_rejected():
    for r in (0, 33, -1):
        with pytest.raises(ValueError):
            C.compress_rate(np.zeros((4, 4, 4), np.float32), r)
