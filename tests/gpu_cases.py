"""Matched inputs for the oracle and the CUDA library (test helper).

Both sides receive the same float32 velocity values, source / receiver
positions and grid parameters from paper_1810_05268_gb300.synth; each side
computes its own wavelet, stencil weights, damping and interpolation.
"""
from dataclasses import dataclass

import numpy as np

from oracle import propagator as O
from paper_1810_05268_gb300 import ckfwi as C
from paper_1810_05268_gb300 import synth


@dataclass
class Case:
    og: O.Grid
    pg: C.GridSpec
    vel: np.ndarray        # float32, total grid
    src: tuple
    rec: np.ndarray
    f0: float
    t0: float

    def shot(self):
        return C.ShotSpec(src=self.src, rec=self.rec, f0=self.f0, t0=self.t0)

    def oracle_series(self):
        return O.ricker(self.og.nt, self.og.dt, self.f0, self.t0)


def make_case(dims, so, shape, nbl, nt, h=10.0, dt=None, seed=0, vmin=1.5, vmax=3.0, f0=None, nrec=None,
              time_order=2):
    if dt is None:
        dt = 1.0 if so <= 4 else 0.8
    vel = synth.grf(shape, 3.0, seed, vmin, vmax).astype(np.float32)
    inner = [(n - 2 * nbl - 1) * h for n in shape]
    if dims == 3:
        src = (2.0 * h, 0.47 * inner[1], 0.53 * inner[2])
        ny = nrec or 5
        rec = synth.receiver_grid(2.5 * h, np.linspace(0, inner[1], ny), np.linspace(0.3 * h, inner[2], ny + 1))
    else:
        src = (2.0 * h, 0.0, 0.41 * inner[1])
        rec = synth.receiver_line(2.5 * h, np.linspace(0.5 * h, inner[1], nrec or 17))
    if f0 is None:
        f0 = vmin / (2.5 * 5 * h)          # >= 5 points per wavelength at 2.5 f0 [kHz]
    t0 = min(1.5 / f0, 0.45 * nt * dt)
    og = O.Grid(dims, tuple(shape), nbl, h, so, dt, nt, vmax, time_order=time_order)
    pg = C.GridSpec(dims, tuple(shape), nbl, h, so, dt, nt, vmax, time_order=time_order)
    return Case(og, pg, vel, src, np.asarray(rec, dtype=np.float64), f0, t0)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def misfit_tol(d_ref, phi_ref, rel=1e-5):
    """Misfit tolerance implied by a receiver tolerance: with
    |d - d_ref| <= rel |d_ref| and r = d_ref - d_obs,
    |phi - phi_ref| <= |d - d_ref| |r| + |d - d_ref|^2 / 2."""
    dd = rel * float(np.linalg.norm(np.asarray(d_ref, dtype=np.float64)))
    return dd * float(np.sqrt(2.0 * phi_ref)) + 0.5 * dd * dd
