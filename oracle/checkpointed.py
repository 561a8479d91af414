"""The gradient as a checkpointing executor computes it, with lossy storage.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3 reverses the N time steps with M checkpoint slots by the Revolve
actions; Sec. 4 stores every checkpoint compressed.  A state restored from a
slot is then the decoded copy, and every forward state recomputed from it
carries that copy's error into the imaging condition.  `gradient` executes
the oracle's own Revolve action list (oracle.revolve.schedule) with the FP64
forward and reverse steps of fwi_oracle.c:

  advance(s, k)   k forward steps from the current pair (u^s, u^{s-1})
  takeshot(s, b)  slot b <- (E(u^s), E(u^{s-1})); the current pair stays
  restore(s, b)   current pair <- the decoded slot b; slot 0 holds the
                  initial state u^0 = u^{-1} = 0, which every format below
                  stores exactly
  youturn(s)      reverse step j = s + 1: lam^s, and the gradient term of
                  n = s, which reads the current u^s

The first sweep (every action before the first youturn) starts from the
exact initial state and restores nothing, so the simulated data, the
residual and the misfit are the lossless ones.

Storage formats (encode then decode; "fp64" is the identity):
  fp32   round to float32 (to nearest, ties to even)
  fp16   float32 first, then IEEE binary16 (to nearest, ties to even)
  bf16   float32 first, then bfloat16: the upper 16 bits of the float32
         pattern, rounded to nearest, ties to even
  codec  float32 first, then the fixed-accuracy codec (oracle.codec) at the
         absolute bound `tol`
  rate   float32 first, then the codec's fixed-rate mode at `rate` bits per
         value
Every lossy format starts from the float32 value: a single-precision
propagator holds its states in that precision, and a rounding or
quantisation decision is taken in the precision of the value it rounds.
"""
import ctypes
import math

import numpy as np

from . import codec as _codec
from . import propagator as _prop
from . import revolve as _rev
from ._lib import lib

STORES = ("fp64", "fp32", "fp16", "bf16", "codec", "rate")


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def bf16_round(x):
    """float32 -> bfloat16 -> float32, to nearest with ties to even: add
    0x7FFF plus the lowest kept bit to the float32 pattern and clear the low
    16 bits.  Finite input only (a carry out of the largest finite values
    gives infinity, as rounding must)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("bf16_round: non-finite input")
    b = x.view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (r.astype(np.uint32) << 16).view(np.float32).reshape(x.shape)


def roundtrip(x, store, tol=None, rate=None):
    """The value a slot of format `store` gives back for the FP64 field x."""
    x = np.asarray(x, dtype=np.float64)
    if store == "fp64":
        return x.copy()
    x32 = x.astype(np.float32)
    if store == "fp32":
        y = x32
    elif store == "fp16":
        y = x32.astype(np.float16).astype(np.float32)
    elif store == "bf16":
        y = bf16_round(x32)
    elif store == "codec":
        if tol is None or not tol > 0:
            raise ValueError("codec storage needs tol > 0")
        stream, nonfinite = _codec.compress(x32, tol)
        if nonfinite:
            raise ValueError("non-finite value in a stored state")
        y = _codec.decompress(stream, x.shape)
    elif store == "rate":
        if rate is None:
            raise ValueError("rate storage needs rate")
        stream, nonfinite = _codec.compress_rate(x32, rate)
        if nonfinite:
            raise ValueError("non-finite value in a stored state")
        y = _codec.decompress(stream, x.shape)
    else:
        raise ValueError("unknown storage format %r" % (store,))
    if not np.all(np.isfinite(y)):
        raise ValueError("a stored state overflows the %s format" % store)
    return y.astype(np.float64)


class Stepper:
    """One forward / adjoint problem held in the C oracle between single
    steps (ora_problem_*)."""

    def __init__(self, grid, vel, src_pos, src_series, rec_pos):
        self._h = None
        vel = _prop._f64(vel)
        if vel.size != int(np.prod(grid.shape)):
            raise ValueError("velocity size does not match the grid")
        self.src_pos, ser, self.rec_pos = _prop._geom(src_pos, src_series, rec_pos, grid.nt)
        self.grid = grid
        self._g = grid.c()
        self._h = lib().ora_problem_create(ctypes.byref(self._g), _ptr(vel), self.src_pos.shape[0],
                                           _ptr(self.src_pos), _ptr(ser), self.rec_pos.shape[0],
                                           _ptr(self.rec_pos))
        if not self._h:
            raise ValueError("ora_problem_create rejected the problem")

    def close(self):
        if self._h:
            lib().ora_problem_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()

    def fwd(self, n, cur, prev):
        """u^{n+1} from cur = u^n, prev = u^{n-1} (source term q^n)."""
        out = np.empty(self.grid.shape)
        _prop._check(lib().ora_problem_fwd_step(self._h, int(n), _ptr(cur), _ptr(prev), _ptr(out)),
                     "fwd step")
        return out

    def adj(self, r, j, l1, l2, un=None, grad=None):
        """lam^{j-1} from l1 = lam^j, l2 = lam^{j+1} and r^j; with grad,
        accumulates the gradient term of n = j - 1 read from un = u^{j-1}."""
        out = np.empty(self.grid.shape)
        _prop._check(lib().ora_problem_adj_step(self._h, _ptr(r), int(j), _ptr(l1), _ptr(l2), _ptr(out),
                                                _ptr(un), _ptr(grad)), "adjoint step")
        return out


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gradient(grid, vel, src_pos, src_series, rec_pos, dobs, M, store="fp64", tol=None, rate=None):
    """(phi, dphi/dm, counts) of one shot with M Revolve slots whose
    checkpoints are stored in format `store` (module docstring).  counts is
    Revolve's {'p', 'W', 'R'}."""
    N = grid.nt
    if store not in STORES:
        raise ValueError("unknown storage format %r" % (store,))
    acts, counts = _rev.schedule(N, M)
    d = _prop.forward(grid, vel, src_pos, src_series, rec_pos)
    dobs = _prop._f64(dobs, d.shape)
    r = _c64(d - dobs)
    r[0] = 0.0
    phi = 0.5 * math.fsum(float(v) for v in (r[1:] * r[1:]).ravel())
    zero = np.zeros(grid.shape)
    grad = np.zeros(grid.shape)
    with Stepper(grid, vel, src_pos, src_series, rec_pos) as S:
        cur, prev = zero, zero
        slots = {0: (zero, zero)}
        l1, l2 = zero, zero          # lam^j, lam^{j+1}
        for op, a, b in acts:
            if op == _rev.ADVANCE:
                for n in range(a, a + b):
                    cur, prev = S.fwd(n, cur, prev), cur
            elif op == _rev.TAKESHOT:
                slots[b] = (roundtrip(cur, store, tol, rate), roundtrip(prev, store, tol, rate))
            elif op == _rev.RESTORE:
                cur, prev = slots[b]
            elif op == _rev.YOUTURN:
                l0 = S.adj(r, a + 1, l1, l2, un=_c64(cur), grad=grad)
                l1, l2 = l0, l1
            else:
                raise AssertionError(op)
    return phi, grad, counts
