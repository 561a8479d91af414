"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's Overthrust model (Sec. 6) is not available; these generators
stand in for it with the same kinds of structure (layers, faults, smooth
heterogeneity), spacing and absorbing-layer width.  They produce inputs
only -- velocity models, start models, source / receiver positions and
random perturbations -- and hold none of the method's arithmetic, so both
the oracle and the library can be fed from them.  All randomness comes from
numpy.random.Generator(PCG64(seed)) and all arrays are float64 until the
caller casts them.
"""
from dataclasses import dataclass

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def extend(interior, nbl):
    """Extend an interior model into the damping layer by edge replication."""
    return np.pad(interior, nbl, mode="edge")


def _gauss(x, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(x, sigma, mode="nearest")


def grf(shape, sigma, seed, vmin, vmax):
    """Gaussian random field: white noise, Gaussian filter (sigma in cells),
    min-max mapped to [vmin, vmax]."""
    w = rng(seed).standard_normal(shape)
    f = _gauss(w, sigma)
    f = (f - f.min()) / (f.max() - f.min())
    return vmin + (vmax - vmin) * f


def two_layer(shape, h, depth, v1, v2):
    """v1 above interior depth `depth` [m], v2 below (axis 0 is depth)."""
    z = np.arange(shape[0]) * h
    v = np.where(z < depth, v1, v2)
    return np.broadcast_to(v.reshape((-1,) + (1,) * (len(shape) - 1)), shape).astype(np.float64).copy()


def layered_faults(shape, h, seed, nlayers=12, vmin=1.5, vmax=6.0, max_dip_deg=10.0, nfaults=3,
                   throw=(50.0, 200.0), jitter=0.05):
    """Layers with velocity increasing with depth (+- jitter), planar dipping
    interfaces at a random azimuth, and planar faults with vertical throw."""
    r = rng(seed)
    nz = shape[0]
    depth = (nz - 1) * h
    coords = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    z = coords[0]
    lateral = coords[1:]
    az = r.uniform(0, 2 * np.pi)
    dip = np.tan(np.radians(r.uniform(0, max_dip_deg)))
    if len(lateral) == 2:
        ramp = dip * (np.cos(az) * lateral[0] + np.sin(az) * lateral[1])
    else:
        ramp = dip * np.cos(az) * lateral[0]
    zz = z - ramp
    for _ in range(nfaults):
        # fault plane through a random point, random strike; hanging wall shifted
        p = [r.uniform(0.2, 0.8) * (n - 1) * h for n in shape[1:]]
        strike = r.uniform(0, 2 * np.pi)
        if len(lateral) == 2:
            side = np.cos(strike) * (lateral[0] - p[0]) + np.sin(strike) * (lateral[1] - p[1])
        else:
            side = lateral[0] - p[0]
        side = side + 0.3 * (z - depth / 2)
        zz = zz + np.where(side > 0, r.uniform(*throw), 0.0)
    tops = np.sort(r.uniform(0.0, depth, nlayers - 1))
    vel_layers = np.linspace(vmin, vmax, nlayers) * (1 + jitter * r.uniform(-1, 1, nlayers))
    vel_layers = np.clip(vel_layers, vmin, vmax)
    idx = np.searchsorted(tops, zz)
    return vel_layers[idx]


def dipping_layers(shape, h, seed, nlayers=8, vmin=1.5, vmax=4.5, max_dip_deg=8.0):
    """2D model with `nlayers` layers of increasing velocity and dipping interfaces."""
    r = rng(seed)
    nz, nx = shape
    z = np.arange(nz)[:, None] * h
    x = np.arange(nx)[None, :] * h
    depth = (nz - 1) * h
    tops = np.sort(r.uniform(0.05 * depth, depth, nlayers - 1))
    dips = np.tan(np.radians(r.uniform(-max_dip_deg, max_dip_deg, nlayers - 1)))
    v = np.full(shape, vmin)
    vel_layers = np.linspace(vmin, vmax, nlayers)
    for k in range(nlayers - 1):
        v = np.where(z >= tops[k] + dips[k] * (x - x.mean()), vel_layers[k + 1], v)
    return v


def smooth_start(vel, sigma):
    """Start model: the true model blurred in m = 1/c^2 (sigma in cells)."""
    m = 1.0 / vel ** 2
    return 1.0 / np.sqrt(_gauss(m, sigma))


def smooth_perturbation(shape, sigma, seed):
    p = _gauss(rng(seed).standard_normal(shape), sigma)
    return p / np.abs(p).max()


def receiver_grid(z, ys, xs):
    """[ny*nx][3] receiver positions (z, y, x) on a regular surface grid."""
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([np.full(yy.size, float(z)), yy.ravel(), xx.ravel()], axis=1)


def receiver_line(z, xs):
    xs = np.asarray(xs, dtype=np.float64)
    return np.stack([np.full(xs.size, float(z)), np.zeros(xs.size), xs], axis=1)


@dataclass
class Workload:
    name: str
    dims: int
    shape: tuple         # total grid
    nbl: int
    h: float
    so: int
    dt: float
    nt: int
    vmax: float
    src: tuple
    f0: float
    rec: np.ndarray
    true: np.ndarray     # velocity [km/s], total grid
    start: np.ndarray


def workload(name, nt=None):
    """The hot path's workloads by size (see the sizes in each branch)."""
    if name == "2d-201x201-so4":
        # 2D, 201^2 interior + 40-cell layer at 10 m, order 4, 500 steps of
        # 1 ms, two layers 1.5 / 2.5 km/s, 10 Hz source, 101 receivers.
        nbl, h = 40, 10.0
        true = extend(two_layer((201, 201), h, 1000.0, 1.5, 2.5), nbl)
        return Workload(name, 2, true.shape, nbl, h, 4, 1.0, nt or 500, 2.5, (20.0, 0.0, 1000.0), 0.010,
                        receiver_line(20.0, np.arange(0.0, 2000.0 + 1e-9, 20.0)), true,
                        smooth_start(true, 8.0))
    if name == "3d-128cube-so8":
        # 3D, 128^3 interior + 40-cell layer (208^3) at 15 m, order 8, 1000
        # steps of 1 ms, Gaussian random field 1.5-4.5 km/s, 8 Hz source,
        # 64 x 64 receivers at 30 m depth.
        nbl, h = 40, 15.0
        inner = grf((128, 128, 128), 8.0, 1811, 1.5, 4.5)
        true = extend(inner, nbl)
        ext = 127 * h
        rec = receiver_grid(30.0, np.linspace(0.0, ext, 64), np.linspace(0.0, ext, 64))
        return Workload(name, 3, true.shape, nbl, h, 8, 1.0, nt or 1000, 4.5, (30.0, ext / 2, ext / 2), 0.008,
                        rec, true, smooth_start(true, 16.0))
    if name == "3d-300x600x600-so16":
        # 3D, 300 x 600 x 600 total (incl. 40-cell layer) at 25 m, order 16,
        # 3000 steps of 1.5 ms, layered model with dipping faults 1.5-6 km/s,
        # 5 Hz source, 64 x 64 receivers.
        nbl, h = 40, 25.0
        inner_shape = (300 - 2 * nbl, 600 - 2 * nbl, 600 - 2 * nbl)
        true = extend(layered_faults(inner_shape, h, 1812), nbl)
        ey, ex = (inner_shape[1] - 1) * h, (inner_shape[2] - 1) * h
        rec = receiver_grid(50.0, np.linspace(0.0, ey, 64), np.linspace(0.0, ex, 64))
        return Workload(name, 3, true.shape, nbl, h, 16, 1.5, nt or 3000, 6.0, (50.0, ey / 2, ex / 2), 0.005,
                        rec, true, smooth_start(true, 10.0))
    if name == "2d-1024x384-so8":
        # 2D, 1024 (x) x 384 (z) interior + 40-cell layer at 10 m, order 8,
        # 2000 steps of 1 ms, 8 dipping layers 1.5-4.5 km/s, 512 receivers.
        nbl, h = 40, 10.0
        true = extend(dipping_layers((384, 1024), h, 1814), nbl)
        return Workload(name, 2, true.shape, nbl, h, 8, 1.0, nt or 2000, 4.5, (20.0, 0.0, 5115.0), 0.010,
                        receiver_line(20.0, np.arange(0.0, 1024 * h - 1e-9, 2 * h)), true,
                        smooth_start(true, 15.0))
    raise KeyError(name)


@dataclass
class Window:
    shape: tuple         # total grid of the window (incl. its damping layer)
    offset: tuple        # (z, y, x) of its first point in the survey grid
    vel: np.ndarray      # velocity [km/s] of the window


def batched_apertures(nshots=32, seed=1813, survey=(256, 448, 448), small=(128, 128, 128),
                      large=(256, 320, 320)):
    """Shots with uneven 3D apertures cut from one survey model: a Gaussian
    random field (sigma 8 cells, 1.5-4.5 km/s) on the survey grid, and
    `nshots` windows whose sizes ramp from `small` to `large` (rounded to
    multiples of 8, order shuffled by the seed), each at a seeded offset that
    keeps it inside the survey.  Returns (survey velocity, windows)."""
    r = rng(seed)
    vel = grf(survey, 8.0, seed, 1.5, 4.5)
    sizes = []
    for i in range(nshots):
        t = i / max(1, nshots - 1)
        sizes.append(tuple(int(round((a + t * (b - a)) / 8.0)) * 8 for a, b in zip(small, large)))
    order = r.permutation(nshots)
    wins = []
    for i in order:
        s = sizes[i]
        off = tuple(int(r.integers(0, n - w + 1)) for n, w in zip(survey, s))
        sl = tuple(slice(o, o + w) for o, w in zip(off, s))
        wins.append(Window(s, off, np.ascontiguousarray(vel[sl])))
    return vel, wins
