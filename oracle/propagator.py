"""FP64 forward modelling, adjoint and gradient of the acoustic wave equation.

Test infrastructure only.  Thin numpy front end of fwi_oracle.c; every
number is computed there (see that file's header for the discretisation,
which follows Sec. 6, Eq. "eqn:wave" and the misfit after it, with the
readings of what the paper leaves to its DSL).
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from ._lib import OraGrid, lib


@dataclass
class Grid:
    dims: int
    shape: tuple          # total grid (nz, ny, nx) in 3D, (nz, nx) in 2D
    nbl: int
    h: float              # [m]
    so: int               # space order
    dt: float             # [ms]
    nt: int               # number of time steps N
    vmax_damp: float      # [km/s]
    refl: float = 1e-3
    time_order: int = 2   # 2: OT2 kernel, 4: OT4 kernel (Sec. 6)

    @property
    def n3(self):
        if self.dims == 3:
            return tuple(self.shape)
        return (self.shape[0], 1, self.shape[1])

    def c(self):
        nz, ny, nx = self.n3
        return OraGrid(self.dims, nz, ny, nx, self.nbl, self.so, self.nt, self.h, self.dt,
                       self.vmax_damp, self.refl, self.time_order)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(st, what):
    if st < 0:
        raise ValueError("oracle %s failed with status %d" % (what, st))
    return st


def fd_weights(k):
    c = np.zeros(k + 1)
    _check(lib().ora_fd_weights(k, _p(c)), "fd_weights")
    return c


def laplacian(grid: Grid, u):
    u = _f64(u)
    out = np.empty_like(u)
    g = grid.c()
    _check(lib().ora_laplacian(ctypes.byref(g), _p(u), _p(out)), "laplacian")
    return out


def damping(grid: Grid):
    eta = np.empty(grid.shape)
    g = grid.c()
    _check(lib().ora_damping(ctypes.byref(g), _p(eta)), "damping")
    return eta


def ricker(nt, dt, f0, t0=None, amp=1.0):
    if t0 is None:
        t0 = 1.5 / f0
    s = np.empty(nt)
    _check(lib().ora_ricker(nt, dt, f0, t0, amp, _p(s)), "ricker")
    return s


def interp(grid: Grid, pos):
    pos = _f64(pos, (3,))
    idx = np.zeros(8, dtype=np.int64)
    wt = np.zeros(8)
    g = grid.c()
    n = _check(lib().ora_interp(ctypes.byref(g), _p(pos), _p(idx), _p(wt)), "interp")
    return idx[:n], wt[:n]


def _geom(src_pos, src_series, rec_pos, nt):
    src_pos = _f64(src_pos).reshape(-1, 3)
    nsrc = src_pos.shape[0]
    if src_series is None:
        ser = None
    else:
        ser = _f64(src_series).reshape(nsrc, nt)
    rec_pos = _f64(rec_pos).reshape(-1, 3)
    return src_pos, ser, rec_pos


def forward(grid: Grid, vel, src_pos, src_series, rec_pos, want_final=False):
    """d [nt+1][nrec] (d[0] = 0) and optionally u^N."""
    vel = _f64(vel)
    assert vel.size == int(np.prod(grid.shape))
    src_pos, ser, rec_pos = _geom(src_pos, src_series, rec_pos, grid.nt)
    d = np.zeros((grid.nt + 1, rec_pos.shape[0]))
    uf = np.zeros(grid.shape) if want_final else None
    g = grid.c()
    _check(lib().ora_forward(ctypes.byref(g), _p(vel), src_pos.shape[0], _p(src_pos), _p(ser),
                             rec_pos.shape[0], _p(rec_pos), _p(d), _p(uf)), "forward")
    return (d, uf) if want_final else d


def step(grid: Grid, vel, cur, prev):
    """u^{n+1} of the source-free recursion from u^n = cur, u^{n-1} = prev."""
    vel = _f64(vel)
    cur = _f64(cur, grid.shape)
    prev = _f64(prev, grid.shape)
    out = np.zeros(grid.shape)
    g = grid.c()
    _check(lib().ora_step(ctypes.byref(g), _p(vel), _p(cur), _p(prev), _p(out)), "step")
    return out


def adjoint(grid: Grid, vel, src_pos, src_series, rec_pos, r, want_grad=True,
            want_srcadj=False, want_lam0=False, seg=0):
    """Adjoint sweep driven by r [nt+1][nrec]; returns a dict with 'grad'
    (dphi/dm), 'srcadj' ([nsrc][nt], = F^T r) and/or 'lam0' as requested."""
    vel = _f64(vel)
    src_pos, ser, rec_pos = _geom(src_pos, src_series, rec_pos, grid.nt)
    r = _f64(r, (grid.nt + 1, rec_pos.shape[0]))
    out = {}
    grad = np.zeros(grid.shape) if want_grad else None
    sa = np.zeros((src_pos.shape[0], grid.nt)) if want_srcadj else None
    l0 = np.zeros(grid.shape) if want_lam0 else None
    g = grid.c()
    _check(lib().ora_adjoint(ctypes.byref(g), _p(vel), src_pos.shape[0], _p(src_pos), _p(ser),
                             rec_pos.shape[0], _p(rec_pos), _p(r), _p(grad), _p(sa), _p(l0),
                             int(seg)), "adjoint")
    if want_grad:
        out["grad"] = grad
    if want_srcadj:
        out["srcadj"] = sa
    if want_lam0:
        out["lam0"] = l0
    return out


def gradient(grid: Grid, vel, src_pos, src_series, rec_pos, dobs, seg=0):
    """(phi, dphi/dm, d_sim) for one shot."""
    vel = _f64(vel)
    src_pos, ser, rec_pos = _geom(src_pos, src_series, rec_pos, grid.nt)
    dobs = _f64(dobs, (grid.nt + 1, rec_pos.shape[0]))
    phi = ctypes.c_double(0.0)
    grad = np.zeros(grid.shape)
    dsim = np.zeros_like(dobs)
    g = grid.c()
    _check(lib().ora_gradient(ctypes.byref(g), _p(vel), src_pos.shape[0], _p(src_pos), _p(ser),
                              rec_pos.shape[0], _p(rec_pos), _p(dobs), ctypes.byref(phi),
                              _p(grad), _p(dsim), int(seg)), "gradient")
    return phi.value, grad, dsim


def misfit(grid: Grid, vel, src_pos, src_series, rec_pos, dobs):
    d = forward(grid, vel, src_pos, src_series, rec_pos)
    r = d[1:] - _f64(dobs, d.shape)[1:]
    return 0.5 * float(np.sum(r * r))
