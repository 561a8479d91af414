"""Batched shots: one launch per stencil step over every lane of a batch.

A batch changes how the steps are launched, never a value: each lane runs
the single-shot arithmetic, so the batched sum over shots must be bitwise
the compensated FP64 sum of the single-shot gradients
(ckfwi_adjoint_gradient), in shot order.  Windows with uneven apertures
(ckfwi_batch_gradient_models) are checked the same way after placing each
window's gradient in the global grid, and the batched gradient is also
compared with the FP64 oracle (Sec. 1.2: shot gradients add up).
"""
import numpy as np
import pytest

from oracle import propagator as O

from gpu_cases import make_case, misfit_tol, rel_l2

torch = pytest.importorskip("torch")
C = pytest.importorskip("paper_1810_05268_gb300.ckfwi")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _neumaier(terms):
    """Compensated sum in the library's order: s, c over terms, then s + c."""
    s = np.zeros_like(np.asarray(terms[0], dtype=np.float64))
    c = np.zeros_like(s)
    for g in terms:
        v = np.asarray(g, dtype=np.float64)
        t = s + v
        c = c + np.where(np.abs(s) >= np.abs(v), (s - t) + v, (v - t) + s)
        s = t
    return s + c


def _shots(case, n, seed):
    """n shots on the case's grid: sources spread along x, shared receivers."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        src = list(case.src)
        src[-1] = case.src[-1] * (0.4 + 1.2 * i / max(1, n - 1))
        src[0] = case.src[0] + float(rng.uniform(0, 1)) * case.og.h
        out.append(C.ShotSpec(src=tuple(src), rec=case.rec, f0=case.f0, t0=case.t0))
    return out


def _observed(m, shots, scale=1.02):
    """Observed data: the model's own data, scaled (a nonzero residual)."""
    return [m.forward_shot(s) * scale for s in shots]


def _singles(m, shots, d_obs, M, mode, tol=0.0):
    grads, phis = [], []
    for s, d in zip(shots, d_obs):
        phi, g, _ = m.adjoint_gradient(s, d, M, store_mode=mode, tol=tol)
        grads.append(g.cpu().numpy())
        phis.append(phi)
    return grads, phis


def _misfit_sum(phis):
    ms = mc = 0.0
    for p in phis:
        t = ms + p
        mc += (ms - t) + p if abs(ms) >= abs(p) else (p - t) + ms
        ms = t
    return ms + mc


BATCH_CASES = [
    # dims, so, shape, nbl, nt, shots, lanes, M, mode
    (2, 8, (60, 83), 10, 150, 5, 2, 6, "fp32"),
    (2, 4, (47, 66), 8, 130, 3, 64, 130, "fp32"),       # store-all
    (2, 8, (52, 70), 8, 140, 4, 3, 5, "bf16"),
    (2, 8, (52, 70), 8, 140, 3, 64, 5, "fp16"),
    (2, 4, (44, 61), 8, 120, 3, 64, 6, "codec"),
    (3, 8, (30, 37, 45), 6, 70, 3, 2, 5, "fp32"),
    (3, 4, (27, 33, 36), 5, 70, 3, 64, 4, "bf16"),
    (3, 8, (29, 35, 38), 6, 60, 2, 64, 5, "codec"),
    (3, 16, (34, 38, 41), 8, 60, 2, 64, 4, "fp32"),
]


@pytest.mark.parametrize("dims,so,shape,nbl,nt,nshots,lanes,M,mode", BATCH_CASES)
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_shots(monkeypatch, dims, so, shape, nbl, nt, nshots, lanes, M, mode, use_graph):
    monkeypatch.setenv("CKFWI_MAX_LANES", str(lanes))
    case = make_case(dims, so, shape, nbl, nt, seed=7 * dims + so)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    shots = _shots(case, nshots, seed=so)
    d_obs = _observed(m, shots)
    tol = 1e-5 if mode == "codec" else 0.0
    grads, phis = _singles(m, shots, d_obs, M, mode, tol)
    phi_b, gsum, st = m.batch_gradient(shots, d_obs, M, store_mode=mode, tol=tol, use_graph=use_graph)
    ref = _neumaier(grads)
    got = gsum.cpu().numpy()
    assert got.dtype == np.float64
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))
    assert phi_b == _misfit_sum(phis)
    assert st["adj_steps"] == nshots * nt
    # a second call replays (graph) or re-runs; same result
    phi2, g2, _ = m.batch_gradient(shots, d_obs, M, store_mode=mode, tol=tol, use_graph=use_graph)
    assert np.array_equal(g2.cpu().numpy(), got) and phi2 == phi_b


@pytest.mark.parametrize("ver", [4, 7])
@pytest.mark.parametrize("dims,so,shape,nbl,nt,nshots,lanes,M,mode",
                         [c for c in BATCH_CASES if c[0] == 3] + [(3, 8, (29, 35, 38), 6, 60, 3, 64, 5, "fp16")])
def test_batch_async_copy_generations_equal_single_shots(monkeypatch, ver, dims, so, shape, nbl, nt, nshots, lanes,
                                                         M, mode):
    """The batched async-copy forward step (generation 4) and the batched lean
    forward and reverse steps (generation 7), forced by CKFWI_BATCH_VER."""
    monkeypatch.setenv("CKFWI_MAX_LANES", "64")          # one batch: its tiles are the stats'
    monkeypatch.setenv("CKFWI_BATCH_VER", str(ver))
    case = make_case(dims, so, shape, nbl, nt, seed=7 * dims + so + ver)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    shots = _shots(case, nshots, seed=so)
    d_obs = _observed(m, shots)
    tol = 1e-5 if mode == "codec" else 0.0
    grads, phis = _singles(m, shots, d_obs, M, mode, tol)
    phi_b, gsum, st = m.batch_gradient(shots, d_obs, M, store_mode=mode, tol=tol, use_graph=True, profile=False)
    _, _, sp = m.batch_gradient(shots, d_obs, M, store_mode=mode, tol=tol, profile=True)
    assert sp["fwd_ver"] == ver and sp["adj_ver"] == (7 if ver == 7 else 3)
    assert sp["u_absmax"] > 0
    ref = _neumaier(grads)
    assert np.array_equal(gsum.cpu().numpy(), ref)
    assert phi_b == _misfit_sum(phis)


def test_batch_launch_count(monkeypatch):
    """All lanes of a batch share each stencil launch."""
    monkeypatch.setenv("CKFWI_MAX_LANES", "4")
    case = make_case(2, 8, (50, 64), 8, 100, seed=3)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    shots = _shots(case, 4, seed=1)
    d_obs = _observed(m, shots)
    _, _, st = m.batch_gradient(shots, d_obs, 6, profile=True)
    _, _, one = m.adjoint_gradient(shots[0], d_obs[0], 6, profile=True)
    assert st["fwd_launches"] == one["fwd_launches"]
    assert st["adj_launches"] == one["adj_launches"] == case.og.nt
    assert st["fwd_steps"] == 4 * one["fwd_steps"]


def test_batch_shot_change_and_medium_change(monkeypatch):
    """Graphs are keyed by the lanes' shots; clones follow a new medium."""
    monkeypatch.setenv("CKFWI_MAX_LANES", "3")
    case = make_case(2, 4, (46, 60), 8, 120, seed=11)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    shots_a = _shots(case, 3, seed=2)
    shots_b = _shots(case, 3, seed=5)
    d_a = _observed(m, shots_a)
    d_b = _observed(m, shots_b)
    for shots, d in ((shots_a, d_a), (shots_b, d_b), (shots_a, d_a)):
        grads, _ = _singles(m, shots, d, 5, "fp32")
        _, g, _ = m.batch_gradient(shots, d, 5, use_graph=True)
        assert np.array_equal(g.cpu().numpy(), _neumaier(grads))
    vel2 = (case.vel * np.float32(1.03)).astype(np.float32)
    m.set_model(torch.from_numpy(vel2).cuda())
    grads, _ = _singles(m, shots_a, d_a, 5, "fp32")
    _, g, _ = m.batch_gradient(shots_a, d_a, 5, use_graph=True)
    assert np.array_equal(g.cpu().numpy(), _neumaier(grads))


def _windows(dims):
    """A global grid and uneven windows (shape, offset) inside it."""
    if dims == 2:
        gshape = (70, 120)
        wins = [((52, 60), (0, 0)), ((70, 74), (0, 40)), ((44, 51), (20, 69)), ((60, 88), (5, 16))]
    else:
        gshape = (40, 48, 60)
        wins = [((32, 36, 40), (0, 0, 0)), ((40, 44, 52), (0, 4, 8)), ((28, 33, 37), (10, 15, 23))]
    return gshape, wins


@pytest.mark.parametrize("dims,so,mode", [(2, 8, "fp32"), (2, 4, "bf16"), (3, 8, "fp32"), (3, 4, "codec")])
@pytest.mark.parametrize("use_graph", [False, True])
def test_windows_equal_single_models(dims, so, mode, use_graph):
    from paper_1810_05268_gb300 import synth
    gshape, wins = _windows(dims)
    nt, nbl, h = 90, 6, 10.0
    vel = synth.grf(gshape, 3.0, 41, 1.5, 3.0).astype(np.float32)
    models, shots, d_obs, offs, grads, phis = [], [], [], [], [], []
    tol = 1e-5 if mode == "codec" else 0.0
    for i, (wshape, off) in enumerate(wins):
        case = make_case(dims, so, wshape, nbl, nt, h=h, seed=i)
        sl = tuple(slice(o, o + n) for o, n in zip(off, wshape))
        wv = np.ascontiguousarray(vel[sl])
        m = C.Model(case.pg)
        m.set_model(torch.from_numpy(wv).cuda())
        s = C.ShotSpec(src=case.src, rec=case.rec, f0=case.f0, t0=case.t0)
        d = m.forward_shot(s) * 0.97
        phi, g, _ = m.adjoint_gradient(s, d, 5, store_mode=mode, tol=tol)
        models.append(m)
        shots.append(s)
        d_obs.append(d)
        offs.append(off)
        phis.append(phi)
        full = np.zeros(gshape, dtype=np.float64)
        full[sl] = g.cpu().numpy()
        grads.append(full)
    phi_b, gsum, _ = C.batch_gradient_models(models, shots, d_obs, offs, gshape, 5, store_mode=mode, tol=tol,
                                             use_graph=use_graph)
    ref = _neumaier(grads)
    got = gsum.cpu().numpy()
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))
    assert phi_b == _misfit_sum(phis)


def test_windows_errors():
    gshape, wins = _windows(2)
    case = make_case(2, 4, wins[0][0], 6, 40, seed=0)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    s = case.shot()
    d = m.forward_shot(s)
    with pytest.raises(C.CkfwiError) as e:
        C.batch_gradient_models([m], [s], [d], [(30, 0)], gshape, 4)        # window leaves the grid
    assert e.value.status == C.EINVAL
    with pytest.raises(C.CkfwiError) as e:
        C.batch_gradient_models([m, m], [s, s], [d, d], [(0, 0), (0, 0)], gshape, 4)   # repeated model
    assert e.value.status == C.EINVAL


def test_batch_matches_oracle(monkeypatch):
    """Batched gradient sum against the FP64 oracle's sum over shots."""
    monkeypatch.setenv("CKFWI_MAX_LANES", "3")
    case = make_case(2, 8, (58, 81), 10, 180, seed=23)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    shots = _shots(case, 3, seed=9)
    v0 = case.vel.astype(np.float64)
    # observed data from a faster medium (oracle), so the residual is a real one
    v_true = v0 * 1.03
    d_obs = []
    ref_g = np.zeros(case.pg.shape)
    ref_phi, tol = 0.0, 0.0
    series = case.oracle_series()
    for s in shots:
        d = O.forward(case.og, v_true, [s.src], series, case.rec).astype(np.float32)
        d_obs.append(torch.from_numpy(d).cuda())
        phi, g, dsim = O.gradient(case.og, v0, [s.src], series, case.rec, d.astype(np.float64))
        ref_g += g
        ref_phi += phi
        tol += misfit_tol(dsim, phi)
    phi_b, gsum, _ = m.batch_gradient(shots, d_obs, 8)
    err = rel_l2(gsum.cpu().numpy(), ref_g)
    print("batched gradient rel-L2 vs oracle %.3e, misfit %.9e vs %.9e" % (err, phi_b, ref_phi))
    assert err <= 1e-4, err
    assert abs(phi_b - ref_phi) <= tol
