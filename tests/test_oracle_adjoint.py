"""Pins of the oracle's adjoint and gradient (CPU only).

The adjoint-state gradient (Sec. 6, after Eq. "eqn:wave") is the exact
derivative of the discrete misfit.  Two independent facts fix it:
  * the dot-product test <F s, r> = <s, F^T r> for the linear source-to-data
    map F = P L^{-1} Q^T (to 1e-12 in FP64, 2D and 3D, every order);
  * the Taylor test: phi(m + e dm) - phi(m) - e <g, dm> = O(e^2).
The gradient must also not depend on how the forward states are
regenerated (the schedule changes cost, never values; Sec. 3).
"""
import numpy as np
import pytest

from oracle import propagator as O


def _setup(dims, so, nt, seed):
    rng = np.random.default_rng(seed)
    if dims == 2:
        shape = (26, 30)
        src = [[41.0, 0.0, 57.5], [10.0, 0.0, 120.0]]
        rec = [[22.5, 0.0, x] for x in np.linspace(0.0, 150.0, 7)]
    else:
        shape = (14, 15, 16)
        src = [[31.0, 40.0, 47.5]]
        rec = [[20.0, y, x] for y in (10.0, 52.5) for x in (5.0, 33.0, 71.0)]
    g = O.Grid(dims, shape, 4, 10.0, so, 1.0, nt, 3.0)
    vel = 1.5 + 1.5 * rng.random(shape)
    return g, vel, src, rec, rng


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_dot_product(dims, so):
    g, vel, src, rec, rng = _setup(dims, so, 45, 100 + so + dims)
    s = rng.standard_normal((len(src), g.nt))
    r = rng.standard_normal((g.nt + 1, len(rec)))
    d = O.forward(g, vel, src, s, rec)
    lhs = np.sum(d[1:] * r[1:])
    rhs = np.sum(s * O.adjoint(g, vel, src, None, rec, r, want_grad=False,
                               want_srcadj=True)["srcadj"])
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _taylor_problem(dims, seed=3):
    rng = np.random.default_rng(seed)
    if dims == 2:
        shape = (40, 56)
        g = O.Grid(2, shape, 8, 10.0, 4, 1.0, 220, 3.0)
        src = [[20.0, 0.0, 190.0]]
        rec = [[20.0, 0.0, x] for x in np.linspace(0.0, 390.0, 14)]
        true = np.full(shape, 2.0)
        true[25:, :] = 2.8
    else:
        shape = (20, 22, 24)
        g = O.Grid(3, shape, 5, 12.0, 8, 1.0, 120, 3.0)
        src = [[15.0, 70.0, 80.0]]
        rec = [[15.0, y, x] for y in (0.0, 70.0, 140.0) for x in (0.0, 80.0, 160.0)]
        true = np.full(shape, 2.0)
        true[12:, :, :] = 2.6
    from scipy.ndimage import gaussian_filter
    start = gaussian_filter(true, 3.0)
    s = O.ricker(g.nt, g.dt, 0.025 if dims == 2 else 0.03)
    dobs = O.forward(g, true, src, s, rec)
    dm = gaussian_filter(rng.standard_normal(shape), 2.0)
    dm *= 0.05 / np.abs(dm).max() / start.max() ** 2
    return g, start, src, s, rec, dobs, dm


@pytest.mark.parametrize("dims", [2, 3])
def test_taylor(dims):
    g, vel, src, s, rec, dobs, dm = _taylor_problem(dims)
    phi0, grad, _ = O.gradient(g, vel, src, s, rec, dobs)
    m0 = 1.0 / vel ** 2
    gdm = np.sum(grad * dm)
    assert abs(gdm) > 0
    e1, e2 = [], []
    eps = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]
    for e in eps:
        phi = O.misfit(g, 1.0 / np.sqrt(m0 + e * dm), src, s, rec, dobs)
        e1.append(abs(phi - phi0))
        e2.append(abs(phi - phi0 - e * gdm))
    r1 = [e1[i] / e1[i + 1] for i in range(2, 4)]
    r2 = [e2[i] / e2[i + 1] for i in range(4)]
    assert all(9 < v < 11 for v in r1), r1             # first order without the gradient
    assert all(90 < v < 110 for v in r2), r2           # second order with it


def test_gradient_independent_of_regeneration_segments():
    g, vel, src, s, rec, dobs, _ = _taylor_problem(2)
    _, ga, da = O.gradient(g, vel, src, s, rec, dobs, seg=1)
    _, gb, db = O.gradient(g, vel, src, s, rec, dobs, seg=7)
    _, gc, dc = O.gradient(g, vel, src, s, rec, dobs, seg=g.nt)
    assert np.array_equal(ga, gb) and np.array_equal(ga, gc)
    assert np.array_equal(da, db)


def test_misfit_matches_definition():
    g, vel, src, s, rec, dobs, _ = _taylor_problem(2)
    phi, _, dsim = O.gradient(g, vel, src, s, rec, dobs)
    assert abs(phi - 0.5 * np.sum((dsim[1:] - dobs[1:]) ** 2)) <= 1e-14 * phi
    assert np.all(dsim[0] == 0)
