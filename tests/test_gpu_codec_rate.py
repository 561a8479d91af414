"""GPU parity of the codec's fixed-rate mode (Sec. 2.2: ZFP's fixed-rate mode,
a guaranteed size without an error bound) against the oracle: streams
bitwise equal on identical float input (ragged shapes, zero, tiny and
non-finite blocks, every rate class), decoded fields bitwise equal, and the
fixed-rate checkpoint store: its pool is exactly the predicted size, its
gradient error falls with the rate, graph replay is bitwise."""
import numpy as np
import pytest

from oracle import codec as OC
from oracle import propagator as O

from gpu_cases import make_case, rel_l2

torch = pytest.importorskip("torch")
C = pytest.importorskip("paper_1810_05268_gb300.ckfwi")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _field(dims, shape, seed):
    rng = np.random.default_rng(seed)
    axes = [np.linspace(0, 2, n) for n in shape]
    g = np.meshgrid(*axes, indexing="ij")
    f = np.sin(3 * g[0] + 1) * np.cos(4 * g[-1]) + 0.05 * rng.standard_normal(shape)
    if dims == 3:
        f = f * np.cos(2 * g[1])
    f[tuple(slice(0, max(1, n // 3)) for n in shape)] = 0.0         # zero blocks
    f[tuple(slice(n - min(n, 4), n) for n in shape)] *= 2.0 ** -110  # blocks flushed to zero
    return (f * 1e-2).astype(np.float32)


SHAPES = [(3, (9, 10, 11)), (3, (32, 36, 40)), (3, (17, 70, 129)), (2, (37, 29)), (2, (64, 256)), (2, (101, 7))]


@pytest.mark.parametrize("dims,shape", SHAPES)
@pytest.mark.parametrize("rate", [1, 2, 3, 7, 8, 16, 32])
def test_rate_streams_bitwise_vs_oracle(dims, shape, rate):
    x = _field(dims, shape, seed=len(shape) * 11 + shape[0] + rate)
    ref, _ = OC.compress_rate(x, rate)
    words, nf = C.codec_compress_rate(torch.from_numpy(x).cuda(), rate)
    got = words.cpu().numpy().view(np.uint32)
    assert not nf
    assert got.size == ref.size == C.codec_rate_words(dims, *((shape) if dims == 3 else (shape[0], 1, shape[1])), rate)
    assert np.array_equal(got, ref)
    y = C.codec_decompress(words, shape).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), OC.decompress(ref, shape).view(np.uint32))


def test_rate_nonfinite_and_wavefield():
    case = make_case(3, 8, (40, 44, 48), nbl=8, nt=160, seed=3)
    _, u = O.forward(case.og, case.vel.astype(np.float64), [case.src], case.oracle_series(), case.rec,
                     want_final=True)
    x = u.astype(np.float32)
    for rate in (4, 12):
        ref, _ = OC.compress_rate(x, rate)
        words, _ = C.codec_compress_rate(torch.from_numpy(x).cuda(), rate)
        assert np.array_equal(words.cpu().numpy().view(np.uint32), ref)
    x[3, 5, 7] = np.nan
    ref, nf_ref = OC.compress_rate(x, 8)
    words, nf = C.codec_compress_rate(torch.from_numpy(x).cuda(), 8)
    assert nf and nf_ref
    assert np.array_equal(words.cpu().numpy().view(np.uint32), ref)


def test_rate_errors():
    x = torch.zeros((8, 8, 8), device="cuda")
    for r in (0, 33):
        with pytest.raises(Exception):
            C.codec_compress_rate(x, r)


CASE = dict(shape=(35, 43, 70), nbl=8, nt=120)


def _obs(case):
    true = case.vel.astype(np.float64) * 1.03
    return O.forward(case.og, true, [case.src], case.oracle_series(), case.rec).astype(np.float32)


def test_rate_checkpoints_predictable_pool_and_error_falls_with_rate():
    case = make_case(3, 8, **CASE, seed=5)
    dobs = _obs(case)
    _, g_ref, _ = O.gradient(case.og, case.vel.astype(np.float64), [case.src], case.oracle_series(), case.rec,
                             dobs.astype(np.float64))
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    dd = torch.from_numpy(dobs).cuda()
    M = 8
    words = C.codec_rate_words(3, *case.pg.shape, 8)
    errs = []
    for rate in (4, 8, 12, 16, 24):
        _, g, st = m.adjoint_gradient(case.shot(), dd, ckpt_slots=M, store_mode="rate", rate=rate)
        e = rel_l2(g.cpu().numpy(), g_ref)
        errs.append(e)
        words = C.codec_rate_words(3, *case.pg.shape, rate)
        assert st["pool_bytes_peak"] <= (M - 1) * 2 * words * 4
        assert abs(st["ratio_min"] - st["ratio_mean"]) < 1e-9          # every stream the same size
        print("rate %d: gradient rel-L2 %.3e, ratio %.2f" % (rate, e, st["ratio_mean"]))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3
    # a budget below the predicted size is refused up front
    with pytest.raises(C.CkfwiError):
        m.adjoint_gradient(case.shot(), dd, ckpt_slots=M, store_mode="rate", rate=8,
                           pool_bytes=(M - 1) * 2 * C.codec_rate_words(3, *case.pg.shape, 8) * 4 - 4)
    with pytest.raises(C.CkfwiError):
        m.adjoint_gradient(case.shot(), dd, ckpt_slots=M, store_mode="rate", rate=0)


def test_rate_graph_replay_bitwise():
    case = make_case(3, 4, (33, 37, 41), nbl=6, nt=110, seed=9)
    dd = torch.from_numpy(_obs(case)).cuda()
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    _, g0, _ = m.adjoint_gradient(case.shot(), dd, ckpt_slots=6, store_mode="rate", rate=10)
    g0 = g0.clone()
    _, g1, _ = m.adjoint_gradient(case.shot(), dd, ckpt_slots=6, store_mode="rate", rate=10, use_graph=True)
    g1 = g1.clone()
    _, g2, _ = m.adjoint_gradient(case.shot(), dd, ckpt_slots=6, store_mode="rate", rate=10, use_graph=True)
    assert torch.equal(g0, g1) and torch.equal(g1, g2)


def test_rate_batch_equals_single_shots():
    case = make_case(2, 8, (66, 131), nbl=12, nt=200, seed=13)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    shots, obs = [], []
    for k in range(3):
        c2 = make_case(2, 8, (66, 131), nbl=12, nt=200, seed=13)
        c2.src = (c2.src[0], 0.0, c2.src[2] * (0.6 + 0.3 * k))
        shots.append(c2.shot())
        obs.append(torch.from_numpy(_obs(c2)).cuda())
    phi, gs, _ = m.batch_gradient(shots, obs, ckpt_slots=9, store_mode="rate", rate=12)
    ref, phis = None, 0.0
    for s, o in zip(shots, obs):
        p1, g1, _ = m.adjoint_gradient(s, o, ckpt_slots=9, store_mode="rate", rate=12)
        phis += p1
        ref = g1.double() if ref is None else ref + g1.double()
    assert abs(phi - phis) <= 1e-12 * abs(phis)
    assert rel_l2(gs.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_stream_words_and_size_planning():
    """The stream sizes of a compressed-checkpoint gradient come back in
    schedule order; a plan from every state's size fits the pool it was made
    for, and (states compress better early) takes more slots than the
    worst-ratio rule."""
    from paper_1810_05268_gb300 import perfmodel as P
    case = make_case(3, 8, **CASE, seed=21)
    dd = torch.from_numpy(_obs(case)).cuda()
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    nt = case.pg.nt
    npts = int(np.prod(case.pg.shape))
    S = 2 * npts * 4
    _, _, st = m.adjoint_gradient(case.shot(), dd, ckpt_slots=6, store_mode="rate", rate=8)
    w = m.stream_words()
    assert len(w) == 2 * st["takeshots"]
    assert np.all(w == C.codec_rate_words(3, *case.pg.shape, 8))
    _, _, st = m.adjoint_gradient(case.shot(), dd, ckpt_slots=nt, store_mode="codec", tol=1e-5, pool_bytes=nt * S)
    w = m.stream_words()
    assert len(w) == 2 * (nt - 1)
    sizes = P.state_bytes(nt, nt, w)
    assert sorted(sizes) == list(range(1, nt))
    budget = 4 * S
    plan = P.slots_for_sizes(nt, budget, P.size_function(sizes))
    worst = int(budget / (S / st["ratio_min"] * 1.1))
    assert plan > worst
    _, _, st2 = m.adjoint_gradient(case.shot(), dd, ckpt_slots=plan, store_mode="codec", tol=1e-5,
                                   pool_bytes=budget)
    assert st2["pool_bytes_peak"] <= budget
