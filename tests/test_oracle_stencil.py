"""Pins of the oracle's spatial operators and physics (CPU only).

These check the oracle against facts fixed outside its own code: closed-form
stencil weights, polynomial exactness, symmetry, the exactly conserved
discrete energy of the undamped OT2 recursion (Sec. 6: 2nd order in time),
and the free-space Green's function of m u_tt - lap(u) = q (Eq. "eqn:wave").
"""
import math

import numpy as np
import pytest

from oracle import propagator as O


def test_fd_weights_closed_form_values():
    # k = 1: the three-point second difference; k = 2: (-5/2, 4/3, -1/12)
    assert np.allclose(O.fd_weights(1), [-2.0, 1.0], rtol=0, atol=1e-15)
    assert np.allclose(O.fd_weights(2), [-2.5, 4.0 / 3.0, -1.0 / 12.0], rtol=0, atol=1e-15)
    # k = 4 (8th order): the standard weights
    w8 = [-205.0 / 72, 8.0 / 5, -1.0 / 5, 8.0 / 315, -1.0 / 560]
    assert np.allclose(O.fd_weights(4), w8, rtol=1e-14, atol=0)


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_fd_weights_moments(k):
    # second-derivative conditions: sum_j c_j j^(2q) = 0 for q=0 (with c0), 1 for q=1
    # (weights act as c0 u + sum_j c_j (u_+j + u_-j)), and 0 for 2 <= q <= k
    c = O.fd_weights(k)
    j = np.arange(1, k + 1, dtype=np.float64)
    assert abs(c[0] + 2 * c[1:].sum()) < 1e-13
    assert abs(2 * np.sum(c[1:] * j ** 2) / 2 - 1.0) < 1e-12
    for q in range(2, k + 1):
        assert abs(np.sum(c[1:] * j ** (2 * q))) < 1e-9 * np.sum(np.abs(c[1:]) * j ** (2 * q))


@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_laplacian_exact_on_polynomials_3d(so):
    k = so // 2
    n = 2 * k + 6
    g = O.Grid(3, (n, n + 1, n + 2), 0, 0.5, so, 1.0, 1, 1.0)
    z, y, x = np.meshgrid(*[np.arange(s) * g.h for s in g.shape], indexing="ij")
    deg = so + 1
    xs, ys, zs = x / 3.0 - 1.0, y / 3.0 - 1.0, z / 3.0 - 1.0
    u = xs ** deg + 0.5 * ys ** (deg - 1) * xs + 0.25 * zs ** deg - ys * zs ** 2
    exact = (deg * (deg - 1) * xs ** (deg - 2)
             + 0.5 * (deg - 1) * (deg - 2) * ys ** (deg - 3) * xs
             + 0.25 * deg * (deg - 1) * zs ** (deg - 2) - 2 * ys) / 9.0
    lap = O.laplacian(g, u)
    inner = (slice(k, -k),) * 3
    err = np.abs(lap[inner] - exact[inner]).max()
    assert err < 1e-8 * np.abs(exact[inner]).max()


def test_laplacian_2d_exact_and_symmetric():
    g = O.Grid(2, (23, 31), 0, 1.3, 8, 1.0, 1, 1.0)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(g.shape)
    v = rng.standard_normal(g.shape)
    # symmetric with the zero Dirichlet values outside the grid
    a = np.sum(O.laplacian(g, u) * v)
    b = np.sum(u * O.laplacian(g, v))
    assert abs(a - b) < 1e-12 * abs(a)
    z, x = np.meshgrid(np.arange(23) * g.h, np.arange(31) * g.h, indexing="ij")
    w = (x / 10) ** 9 - 3 * (z / 10) ** 8 + (x / 10) * (z / 10) ** 7
    ex = (72 * (x / 10) ** 7 - 3 * 56 * (z / 10) ** 6 + (x / 10) * 42 * (z / 10) ** 5) / 100
    lap = O.laplacian(g, w)
    assert np.abs(lap[4:-4, 4:-4] - ex[4:-4, 4:-4]).max() < 1e-9 * np.abs(ex).max()


def test_laplacian_symmetric_3d():
    g = O.Grid(3, (11, 12, 13), 0, 1.0, 16, 1.0, 1, 1.0)
    rng = np.random.default_rng(6)
    u, v = rng.standard_normal((2,) + g.shape)
    a = np.sum(O.laplacian(g, u) * v)
    b = np.sum(u * O.laplacian(g, v))
    assert abs(a - b) < 1e-12 * abs(a)


def test_damping_profile():
    g = O.Grid(3, (30, 34, 38), 8, 12.5, 4, 1.0, 1, 3.0, 1e-3)
    eta = O.damping(g)
    L = g.nbl * g.h
    emax = 3 * g.vmax_damp / (2 * L) * math.log(1e3)
    # zero in the interior, eta_max on a face centre, 3 eta_max in a corner
    assert np.all(eta[8:-8, 8:-8, 8:-8] == 0)
    assert abs(eta[0, 17, 19] - emax) < 1e-12 * emax
    assert abs(eta[-1, -1, -1] - 3 * emax) < 1e-12 * emax
    # quadratic in the distance from the first interior point
    assert abs(eta[15, 17, 4] - emax * (4 / 8) ** 2) < 1e-12 * emax
    assert abs(eta[15, 17, 38 - 1 - 8 + 2] - emax * (2 / 8) ** 2) < 1e-12 * emax


def test_ricker_closed_form_properties():
    f0, dt = 0.010, 0.25
    t0 = 1.5 / f0
    nt = int(2 * t0 / dt) + 1
    s = O.ricker(nt, dt, f0, t0, amp=2.0)
    n0 = int(round(t0 / dt))
    assert abs(s[n0] - 2.0) < 1e-15                     # peak value A at t0
    assert np.argmax(s) == n0
    assert np.allclose(s[n0 - 40:n0], s[n0 + 40:n0:-1], atol=1e-14)   # even about t0
    tz = 1.0 / (math.sqrt(2) * math.pi * f0)           # zero crossings at t0 +- tz
    sz = O.ricker(1, 1.0, f0, -tz, 1.0)
    assert abs(sz[0]) < 1e-14
    assert abs(np.sum(s) * dt) < 1e-6                   # zero mean


def test_interp_weights():
    g = O.Grid(3, (20, 21, 22), 5, 10.0, 4, 1.0, 1, 2.0)
    pos = np.array([13.0, 47.5, 101.25])
    idx, wt = O.interp(g, pos)
    assert len(idx) == 8 and abs(wt.sum() - 1) < 1e-15 and np.all(wt >= 0)
    z, y, x = np.meshgrid(*[np.arange(s) for s in g.shape], indexing="ij")
    lin = 2.0 * z - 3.0 * y + 0.5 * x + 7.0
    gc = g.nbl + pos / g.h
    assert abs(np.sum(wt * lin.ravel()[idx]) - (2 * gc[0] - 3 * gc[1] + 0.5 * gc[2] + 7)) < 1e-12
    # on-grid point: weight 1 on that point
    idx, wt = O.interp(g, np.array([0.0, 0.0, 0.0]))
    assert wt.max() == 1.0 and idx[np.argmax(wt)] == (5 * 21 + 5) * 22 + 5
    with pytest.raises(ValueError):
        O.interp(g, np.array([-60.0, 0.0, 0.0]))


def _energy(g, vel, u1, u0):
    """Conserved discrete energy of the undamped OT2 recursion:
    (u1-u0)^T m (u1-u0)/dt^2 - u1^T lap(u0)."""
    m = 1.0 / vel ** 2
    du = (u1 - u0) / g.dt
    return np.sum(m * du * du) - np.sum(u1 * O.laplacian(g, u0))


@pytest.mark.parametrize("dims", [2, 3])
def test_discrete_energy_conserved_without_damping(dims):
    if dims == 2:
        shape, src, h, so = (40, 44), [[150.0, 0.0, 210.0]], 10.0, 8
    else:
        shape, src, h, so = (18, 20, 22), [[80.0, 95.0, 105.0]], 10.0, 4
    rng = np.random.default_rng(11)
    vel = 1.5 + rng.random(shape)
    nt_src = 20
    g = lambda nt: O.Grid(dims, shape, 0, h, so, 1.0, nt, 3.0)
    ser_full = O.ricker(120, 1.0, 0.04, 12.0)
    ser_full[nt_src:] = 0.0
    es = []
    for n in (40, 80, 119):
        _, u0 = O.forward(g(n), vel, src, ser_full[:n], [[0.0, 0.0, 0.0]], want_final=True)
        _, u1 = O.forward(g(n + 1), vel, src, ser_full[:n + 1], [[0.0, 0.0, 0.0]], want_final=True)
        es.append(_energy(g(n), vel, u1, u0))
    assert es[0] > 0
    assert abs(es[1] - es[0]) < 1e-12 * es[0]
    assert abs(es[2] - es[0]) < 1e-12 * es[0]


def test_damping_dissipates_energy():
    shape = (50, 50)
    vel = np.full(shape, 2.0)
    g = lambda nt: O.Grid(2, shape, 12, 10.0, 4, 1.0, nt, 2.0)
    ser = O.ricker(400, 1.0, 0.03, 40.0)
    ser[80:] = 0.0
    es = []
    for n in (100, 250, 399):
        _, u0 = O.forward(g(n), vel, [[130.0, 0, 130.0]], ser[:n], [[0.0, 0, 0.0]], want_final=True)
        _, u1 = O.forward(g(n + 1), vel, [[130.0, 0, 130.0]], ser[:n + 1], [[0.0, 0, 0.0]],
                          want_final=True)
        es.append(_energy(g(n), vel, u1, u0))
    assert es[1] < es[0] and es[2] < 0.05 * es[0]


def test_green_function_3d_homogeneous():
    """Receiver trace against u = h^3 s(t - r/c) / (4 pi r): the point source
    is injected with weight 1 at a grid point (no 1/h^3), so the grid sees a
    source density h^3 s(t) delta(x)."""
    n, h, c = 64, 10.0, 2.0
    nt = 226
    g = O.Grid(3, (n, n, n), 0, h, 8, 1.0, nt, c)
    vel = np.full(g.shape, c)
    f0 = 0.015
    t0 = 70.0
    s = O.ricker(nt, 1.0, f0, t0)
    src = [[320.0, 320.0, 320.0]]
    r = 200.0
    rec = [[320.0, 320.0, 320.0 + r]]
    d = O.forward(g, vel, src, s, rec)[:, 0]
    t = np.arange(nt + 1) * 1.0
    exact = h ** 3 * np.array(O.ricker(nt + 1, 1.0, f0, t0 + r / c)) / (4 * math.pi * r)
    win = t < 225
    err = np.linalg.norm(d[win] - exact[win]) / np.linalg.norm(exact[win])
    assert err < 0.03, err
    assert abs(np.argmax(d) - np.argmax(exact)) <= 1
