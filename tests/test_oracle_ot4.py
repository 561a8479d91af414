"""Pins of the oracle's OT4 kernel (CPU only).

The OT4 kernel (Sec. 6) is fourth order in time: the leapfrog recursion
with lap replaced by A u = lap u + dt^2/12 lap(c^2 lap u).  Facts that fix it
without re-typing it:
  * on a sine eigenmode of the order-2 Dirichlet Laplacian (eigenvalue
    -lam) in a homogeneous, undamped medium one step multiplies the mode by
    1 - mu, mu = (c dt)^2 lam - (c dt)^4 lam^2 / 12 (the closed form of the
    symbol of the scheme);
  * over a fixed time T the error against the semi-discrete solution
    cos(c sqrt(lam) t) falls 16 times when dt is halved (4 times for OT2);
  * the dot-product and Taylor tests of the adjoint and the gradient, which
    exercise the extra c^4 lap u lap lam term of the exact gradient.
"""
import dataclasses

import numpy as np
import pytest

from oracle import propagator as O


def _mode(shape, h, p, q):
    nz, nx = shape
    z = np.arange(nz)[:, None]
    x = np.arange(nx)[None, :]
    phi = np.sin(np.pi * p * (z + 1) / (nz + 1)) * np.sin(np.pi * q * (x + 1) / (nx + 1))
    lam = 4.0 / h ** 2 * (np.sin(np.pi * p / (2 * (nz + 1))) ** 2 + np.sin(np.pi * q / (2 * (nx + 1))) ** 2)
    return phi, lam


@pytest.mark.parametrize("order", [2, 4])
def test_one_step_symbol(order):
    shape, h, c, dt = (19, 23), 10.0, 2.5, 1.7
    g = O.Grid(2, shape, 0, h, 2, dt, 1, 3.0, time_order=order)
    phi, lam = _mode(shape, h, 3, 5)
    vel = np.full(shape, c)
    out = O.step(g, vel, phi, phi)
    x = (c * dt) ** 2 * lam
    mu = x - (x * x / 12.0 if order == 4 else 0.0)
    assert np.max(np.abs(out - (1.0 - mu) * phi)) <= 1e-13


@pytest.mark.parametrize("order,rate", [(2, 4.0), (4, 16.0)])
def test_time_convergence_order(order, rate):
    shape, h, c, T = (21, 25), 10.0, 2.0, 240.0
    phi, lam = _mode(shape, h, 4, 3)
    om = c * np.sqrt(lam)
    vel = np.full(shape, c)
    errs = []
    for dt in (2.0, 1.0):
        g = O.Grid(2, shape, 0, h, 2, dt, 1, 3.0, time_order=order)
        prev, cur = np.cos(om * dt) * phi, phi.copy()
        n = int(round(T / dt))
        for _ in range(n):
            prev, cur = cur, O.step(g, vel, cur, prev)
        errs.append(np.max(np.abs(cur - np.cos(om * n * dt) * phi)))
    r = errs[0] / errs[1]
    assert 0.85 * rate < r < 1.15 * rate, (errs, r)


def _ot4(g):
    return dataclasses.replace(g, time_order=4)


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("so", [4, 8])
def test_dot_product_ot4(dims, so):
    from test_oracle_adjoint import _setup
    g, vel, src, rec, rng = _setup(dims, so, 45, 300 + so + dims)
    g = _ot4(g)
    s = rng.standard_normal((len(src), g.nt))
    r = rng.standard_normal((g.nt + 1, len(rec)))
    d = O.forward(g, vel, src, s, rec)
    lhs = np.sum(d[1:] * r[1:])
    rhs = np.sum(s * O.adjoint(g, vel, src, None, rec, r, want_grad=False,
                               want_srcadj=True)["srcadj"])
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("dims", [2, 3])
def test_taylor_ot4(dims):
    from test_oracle_adjoint import _taylor_problem
    g, vel, src, s, rec, _, dm = _taylor_problem(dims)
    g = _ot4(g)
    true = vel.copy()
    true[tuple(slice(n // 2, None) for n in vel.shape[:1])] *= 1.2
    dobs = O.forward(g, true, src, s, rec)
    phi0, grad, _ = O.gradient(g, vel, src, s, rec, dobs)
    m0 = 1.0 / vel ** 2
    gdm = np.sum(grad * dm)
    assert abs(gdm) > 0
    e2 = []
    for e in [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]:
        phi = O.misfit(g, 1.0 / np.sqrt(m0 + e * dm), src, s, rec, dobs)
        e2.append(abs(phi - phi0 - e * gdm))
    r2 = [e2[i] / e2[i + 1] for i in range(4)]
    assert all(90 < v < 110 for v in r2), r2


def test_ot4_gradient_independent_of_regeneration_segments():
    from test_oracle_adjoint import _taylor_problem
    g, vel, src, s, rec, dobs, _ = _taylor_problem(2)
    g = _ot4(g)
    _, ga, _ = O.gradient(g, vel, src, s, rec, dobs, seg=1)
    _, gb, _ = O.gradient(g, vel, src, s, rec, dobs, seg=9)
    assert np.array_equal(ga, gb)


def test_time_order_validated():
    g = O.Grid(2, (10, 12), 0, 10.0, 2, 1.0, 1, 3.0, time_order=3)
    with pytest.raises(ValueError):
        O.step(g, np.full((10, 12), 2.0), np.zeros((10, 12)), np.zeros((10, 12)))
