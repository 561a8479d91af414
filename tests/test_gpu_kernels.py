"""The generations of 3D stencil kernels agree bit for bit.

The TMA-fed kernels (stencil_tma.cu) and the vector-blocked kernels
(stencil_v3.cu) perform the same FP32 operations in the same order as the
register-queue kernels (kernels.cu), so receivers and gradients must be
identical, whatever the tile; all are also checked against the FP64 oracle
by test_gpu_parity.py through the autotuned choice.
"""
import os

import numpy as np
import pytest

from gpu_cases import make_case

torch = pytest.importorskip("torch")
C = pytest.importorskip("paper_1810_05268_gb300.ckfwi")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()


def _run(case, fwd_tile, adj_tile, dobs, slots, mode="fp32"):
    os.environ["CKFWI_TILE_FWD"] = fwd_tile
    os.environ["CKFWI_TILE_ADJ"] = adj_tile
    try:
        m = C.Model(case.pg)
        m.set_model(torch.from_numpy(case.vel).cuda())
        d = m.forward_shot(case.shot()).cpu().numpy()
        phi, g, st = m.adjoint_gradient(case.shot(), dobs, ckpt_slots=slots, store_mode=mode)
        out = (d, phi, g.cpu().numpy(), st)
        m.close()
        return out
    finally:
        del os.environ["CKFWI_TILE_FWD"]
        del os.environ["CKFWI_TILE_ADJ"]


@pytest.mark.parametrize("so,shape", [(2, (30, 37, 70)), (4, (33, 41, 131)), (8, (35, 43, 70)), (8, (26, 29, 200))])
@pytest.mark.parametrize("ty", [8, 16])
def test_tma_kernels_bitwise_equal_register_queue_kernels(so, shape, ty):
    case = make_case(3, so, shape, nbl=6, nt=80, seed=so + ty)
    rng = np.random.default_rng(so)
    dobs = torch.from_numpy((rng.standard_normal((81, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    k = so // 2
    by1 = max(8, k)
    ref = _run(case, "1,32,%d,9" % by1, "1,32,%d,9" % by1, dobs, 5)
    for per_sm in (1, 7):          # persistent grid: one or many z segments per CTA
        got = _run(case, "2,64,%d,%d" % (ty, per_sm), "2,64,%d,%d" % (ty, per_sm), dobs, 5)
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        assert np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("mode", ["bf16", "fp16"])
def test_tma_reverse_reads_half_slots_like_register_queue(mode):
    case = make_case(3, 8, (35, 43, 70), nbl=6, nt=60, seed=3)
    rng = np.random.default_rng(1)
    dobs = torch.from_numpy((rng.standard_normal((61, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    ref = _run(case, "1,32,8,9", "1,32,8,9", dobs, 4, mode)
    got = _run(case, "2,64,8,2", "2,64,8,2", dobs, 4, mode)
    assert got[1] == ref[1]
    assert np.array_equal(got[2], ref[2])


V3_TILES = ["3,32,16,%d,4", "3,32,16,%d,2"]


@pytest.mark.parametrize("so,shape", [(2, (30, 37, 70)), (4, (33, 41, 131)), (8, (35, 43, 70)), (8, (26, 29, 200)),
                                      (16, (36, 41, 77)), (4, (21, 19, 13))])
@pytest.mark.parametrize("tile", V3_TILES)
def test_vector_kernels_bitwise_equal_register_queue_kernels(so, shape, tile):
    case = make_case(3, so, shape, nbl=6, nt=70, seed=so + len(tile))
    rng = np.random.default_rng(so)
    dobs = torch.from_numpy((rng.standard_normal((71, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    k = so // 2
    by1 = max(8, k)
    ref = _run(case, "1,32,%d,9" % by1, "1,32,%d,9" % by1, dobs, 5)
    for zlen in (7, 64):           # several z runs per column, or one
        t = tile % zlen
        if int(t.split(",")[2]) < k:
            continue
        got = _run(case, t, t, dobs, 5)
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        assert np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("mode", ["bf16", "fp16"])
@pytest.mark.parametrize("vec", [2, 4])
def test_vector_kernels_half_slots_like_register_queue(mode, vec):
    case = make_case(3, 8, (35, 43, 70), nbl=6, nt=60, seed=3)
    rng = np.random.default_rng(1)
    dobs = torch.from_numpy((rng.standard_normal((61, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    ref = _run(case, "1,32,8,9", "1,32,8,9", dobs, 4, mode)
    got = _run(case, "3,32,16,11,%d" % vec, "3,32,16,11,%d" % vec, dobs, 4, mode)
    assert got[1] == ref[1]
    assert np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("so,shape", [(2, (30, 37, 70)), (4, (33, 41, 131)), (8, (35, 43, 70)), (8, (26, 29, 200)),
                                      (16, (36, 41, 77)), (4, (21, 19, 13))])
@pytest.mark.parametrize("vec", [2, 4])
@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_async_copy_forward_bitwise_equal_register_queue(so, shape, vec, mode):
    """The forward step fed by asynchronous copies (generation 4)."""
    case = make_case(3, so, shape, nbl=6, nt=70, seed=so + 3 * vec)
    rng = np.random.default_rng(so)
    dobs = torch.from_numpy((rng.standard_normal((71, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    k = so // 2
    by1 = max(8, k)
    ref = _run(case, "1,32,%d,9" % by1, "1,32,%d,9" % by1, dobs, 5, mode)
    tiles = [("4,32,16,%d,%d" % (z, vec), "4,32,16,%d,%d" % (z, vec)) for z in (7, 64)]
    tiles.append(("4,32,16,9,%d" % vec, "3,32,16,9,%d" % vec))   # mixed generations
    if vec == 4 and so <= 8:
        tiles.append(("4,32,16,9,4,1", "3,32,16,9,4"))            # one plane of prefetch
    for tf, ta in tiles:
        got = _run(case, tf, ta, dobs, 5, mode)
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        assert np.array_equal(got[2], ref[2])


# nx % 32 of the shapes: 6, 3, 6, 8, 13, 13 (a grid narrower than one tile),
# 16, 26 and 0 (no partial tile)
@pytest.mark.parametrize("so,shape", [(2, (30, 37, 70)), (4, (33, 41, 131)), (8, (35, 43, 70)), (8, (26, 29, 200)),
                                      (16, (36, 41, 77)), (4, (21, 19, 13)), (4, (27, 33, 80)), (8, (30, 35, 90)),
                                      (8, (25, 40, 64))])
@pytest.mark.parametrize("mode", ["fp32", "fp16"])
def test_tensor_copy_forward_bitwise_equal_register_queue(so, shape, mode):
    """Generation 8: the forward step fed by tensor copies and the reverse
    step split into its lam half (the same kernel with the adjoint
    injection) and its gradient half, one or two planes of prefetch, z runs
    of one plane, several planes and the whole column, alone and paired
    with other generations (with FP16 checkpoints the reverse step reads
    16-bit u^{j-1} through the lean kernel), on grids with and without a
    partial last x tile; the forced tiles must be the ones that ran."""
    case = make_case(3, so, shape, nbl=6, nt=70, seed=so + 11)
    rng = np.random.default_rng(so + 2)
    dobs = torch.from_numpy((rng.standard_normal((71, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    k = so // 2
    by1 = max(8, k)
    ref = _run(case, "1,32,%d,9" % by1, "1,32,%d,9" % by1, dobs, 5, mode)
    tiles = [("8,32,16,%d,4" % z, "3,32,16,9,4") for z in (1, 7, 64)]
    tiles.append(("8,32,16,9,4", "7,32,16,9,4,1"))
    tiles += [("8,32,16,%d,4,2" % z, "3,32,16,9,4") for z in (1, 2, 9)]   # two planes of prefetch
    # the reverse step split in two launches (lam half by the forward kernel, gradient half)
    tiles += [("3,32,16,9,4", "8,32,16,%d,4,%d" % (z, pf)) for z, pf in ((1, 1), (7, 1), (64, 1), (9, 2))]
    tiles.append(("8,32,16,7,4", "8,32,16,9,4"))
    for tf, ta in tiles:
        got = _run(case, tf, ta, dobs, 5, mode)
        assert got[3]["fwd_ver"] == int(tf[0]) and got[3]["adj_ver"] == int(ta[0]), (tf, ta)
        assert np.array_equal(got[0], ref[0]), (tf, ta)
        assert got[1] == ref[1], (tf, ta)
        assert np.array_equal(got[2], ref[2]), (tf, ta)


@pytest.mark.parametrize("so,shape", [(2, (30, 37, 70)), (4, (33, 41, 131)), (8, (35, 43, 70)), (8, (26, 29, 200)),
                                      (16, (36, 41, 77)), (4, (21, 19, 13))])
@pytest.mark.parametrize("np_", [1, 2])
@pytest.mark.parametrize("mode", ["fp32", "fp16"])
def test_lean_kernels_bitwise_equal_register_queue(so, shape, np_, mode):
    """The lean async-copy generation (Tile.ver 7) with one or two planes per
    step: forward and reverse steps, alone and mixed with other generations,
    with z runs of odd and even length (a two-plane step that ends with one
    plane) and a run covering the whole column."""
    case = make_case(3, so, shape, nbl=6, nt=70, seed=so + 5 * np_)
    rng = np.random.default_rng(so + 1)
    dobs = torch.from_numpy((rng.standard_normal((71, case.rec.shape[0])) * 1e-3).astype(np.float32)).cuda()
    k = so // 2
    by1 = max(8, k)
    ref = _run(case, "1,32,%d,9" % by1, "1,32,%d,9" % by1, dobs, 5, mode)
    tiles = [("7,32,16,%d,4,%d" % (z, np_), "7,32,16,%d,4,%d" % (z, np_)) for z in (7, 8, 64)]
    tiles.append(("7,32,16,9,4,%d" % np_, "3,32,16,9,4"))
    tiles.append(("4,32,16,9,4", "7,32,16,5,4,%d" % np_))
    for tf, ta in tiles:
        got = _run(case, tf, ta, dobs, 5, mode)
        assert np.array_equal(got[0], ref[0]), (tf, ta)
        assert got[1] == ref[1], (tf, ta)
        assert np.array_equal(got[2], ref[2]), (tf, ta)


@pytest.mark.parametrize("tf,ta,call", [("2,64,16,2", "2,64,16,2", "forward"),
                                        ("8,32,16,7,4,1", "3,32,16,9,4", "forward"),
                                        ("3,32,16,9,4", "8,32,16,7,4,1", "gradient")])
def test_tma_wait_that_runs_out_reports_timeout(tf, ta, call):
    """A TMA kernel whose plane waits run out (CKFWI_TMA_WAIT_LIMIT < 0: the
    waits give up at once, the copies in flight are still drained with the
    full bound) reports CKFWI_TIMEOUT, in the TMA-fed generation, the
    tensor-copy forward step and the split reverse step; the device stays
    usable and the next model is exact."""
    case = make_case(3, 8, (35, 43, 70), nbl=6, nt=40, seed=9)
    zeros = torch.zeros((41, case.rec.shape[0]), device="cuda")
    os.environ["CKFWI_TMA_WAIT_LIMIT"] = "-1"
    os.environ["CKFWI_TILE_FWD"] = tf
    os.environ["CKFWI_TILE_ADJ"] = ta
    try:
        m = C.Model(case.pg)
        m.set_model(torch.from_numpy(case.vel).cuda())
        with pytest.raises(C.CkfwiError) as e:
            if call == "forward":
                m.forward_shot(case.shot())
            else:
                m.adjoint_gradient(case.shot(), zeros, ckpt_slots=5)
        assert e.value.status == C.TIMEOUT
        m.close()
    finally:
        for k in ("CKFWI_TMA_WAIT_LIMIT", "CKFWI_TILE_FWD", "CKFWI_TILE_ADJ"):
            del os.environ[k]
    ref = _run(case, "1,32,8,9", "1,32,8,9", zeros, 5)
    got = _run(case, tf, ta, zeros, 5)
    assert np.array_equal(got[0], ref[0])
    assert np.array_equal(got[2], ref[2])
