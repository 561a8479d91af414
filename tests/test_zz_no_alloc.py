"""The allocation-free compression entry point (collected last on purpose).

ckfwi_codec_compress_noalloc serves callers that cannot let the library
call cudaMalloc: it keeps its scratch in a fixed device array inside the
library.  Its streams must equal those of ckfwi_codec_compress bit for bit
(the codec's parity bar), on two calls in a row, so a second call sees the
scratch the first one left behind.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_1810_05268_gb300 import build
    build.build()
    from paper_1810_05268_gb300 import ckfwi
    return ckfwi


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    g = np.meshgrid(*[np.linspace(0, 2, n) for n in shape], indexing="ij")
    f = np.sin(3 * g[0] + 1) * np.cos(4 * g[-1]) + 0.05 * rng.standard_normal(shape)
    f[tuple(slice(0, n // 3) for n in shape)] = 0.0
    return torch.from_numpy((f * 1e-2).astype(np.float32)).cuda()


# the last case is exactly the largest field the static scratch accepts
# (16 x 64 x 64 = 65536 blocks)
@pytest.mark.parametrize("shape,tol", [((33, 41, 58), 1e-5), ((64, 48, 80), 1e-7), ((37, 130), 1e-6),
                                       ((64, 256, 256), 1e-5)])
def test_noalloc_matches_allocating_entry_point_twice(C, shape, tol):
    for call in range(2):
        x = _field(shape, seed=call + len(shape))
        ref, nf_ref = C.codec_compress(x, tol)
        dims = len(shape)
        nz, ny, nx = (shape if dims == 3 else (shape[0], 1, shape[1]))
        out = torch.zeros(C.codec_bound_words(dims, nz, ny, nx), dtype=torch.int32, device="cuda")
        used, nf = C.codec_compress_noalloc(x, out, tol)
        assert nf == nf_ref
        assert used == ref.numel()
        assert torch.equal(out[:used], ref)
        y = C.codec_decompress(out[:used].clone(), shape)
        assert float((y - x).abs().max()) <= tol


def test_noalloc_rejects_fields_beyond_its_scratch(C):
    x = torch.zeros((4 * 41, 4 * 40, 4 * 40), dtype=torch.float32, device="cuda")   # 65600 blocks
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(C.CkfwiError) as e:
        C.codec_compress_noalloc(x, out, 1e-3)
    assert e.value.status == C.EINVAL
