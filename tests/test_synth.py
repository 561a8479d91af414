"""The seeded input generators: deterministic per seed, inside their stated
ranges, and shaped like the workloads they stand in for (total grids,
receivers inside the interior, a time step inside the leapfrog's stability
limit for the model's largest velocity)."""
import numpy as np
import pytest

from paper_1810_05268_gb300 import synth

pytest.importorskip("scipy")

# Courant limit sqrt(4 / (d |symbol|)) of the 2k-th order Laplacian at the
# Nyquist wavenumber, |symbol| = sum_j 4 c_j [j odd] (closed-form weights)
def _courant(so, dims):
    from math import factorial
    k = so // 2
    sym = sum(4 * 2 * factorial(k) ** 2 / (j * j * factorial(k - j) * factorial(k + j))
              for j in range(1, k + 1, 2))
    return (4.0 / (dims * sym)) ** 0.5


def test_courant_limits_match_the_closed_form_values():
    assert _courant(4, 2) == pytest.approx(0.612, abs=1e-3)
    assert _courant(8, 3) == pytest.approx(0.453, abs=1e-3)
    assert _courant(8, 2) == pytest.approx(0.555, abs=1e-3)
    assert _courant(16, 3) == pytest.approx(0.424, abs=1e-3)


def test_generators_are_seeded_and_in_range():
    a = synth.grf((20, 24, 28), 3.0, 5, 1.5, 4.5)
    b = synth.grf((20, 24, 28), 3.0, 5, 1.5, 4.5)
    c = synth.grf((20, 24, 28), 3.0, 6, 1.5, 4.5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() == pytest.approx(1.5) and a.max() == pytest.approx(4.5)
    lf = synth.layered_faults((40, 30, 30), 25.0, 3)
    assert np.array_equal(lf, synth.layered_faults((40, 30, 30), 25.0, 3))
    assert 1.5 <= lf.min() and lf.max() <= 6.0
    dl = synth.dipping_layers((60, 90), 10.0, 4)
    assert 1.5 <= dl.min() and dl.max() <= 4.5
    p = synth.smooth_perturbation((16, 18), 2.0, 1)
    assert np.abs(p).max() == pytest.approx(1.0)


def test_extension_replicates_the_edges():
    x = np.arange(12.0).reshape(3, 4)
    e = synth.extend(x, 2)
    assert e.shape == (7, 8)
    assert np.array_equal(e[2:5, 2:6], x)
    assert np.all(e[0, 2:6] == x[0]) and np.all(e[2:5, 0] == x[:, 0])


def test_start_model_is_the_blur_in_slowness_squared():
    v = synth.two_layer((60, 20), 10.0, 300.0, 1.5, 2.5)
    s = synth.smooth_start(v, 3.0)
    m, ms = 1.0 / v ** 2, 1.0 / s ** 2
    assert ms.min() >= m.min() - 1e-12 and ms.max() <= m.max() + 1e-12
    # rows 25 cells from the interface keep their slowness; the interface
    # row takes the mean of the two sides' m, not of their velocities
    assert np.allclose(ms[:5], m[:5]) and np.allclose(ms[-5:], m[-5:])
    mid = 0.5 * (m[29, 0] + m[30, 0])
    assert abs(0.5 * (ms[29, 0] + ms[30, 0]) - mid) < 1e-3 * mid


@pytest.mark.parametrize("name,shape,so,dims", [("2d-201x201-so4", (281, 281), 4, 2),
                                                ("3d-128cube-so8", (208, 208, 208), 8, 3),
                                                ("2d-1024x384-so8", (464, 1104), 8, 2)])
def test_workloads_have_the_stated_sizes(name, shape, so, dims):
    w = synth.workload(name, nt=10)
    assert tuple(w.shape) == shape and w.so == so and w.dims == dims and w.nt == 10
    assert w.true.shape == shape and w.start.shape == shape
    assert w.vmax >= w.true.max() - 1e-9
    assert w.vmax * w.dt / w.h < _courant(so, dims)
    inner = [(n - 2 * w.nbl - 1) * w.h for n in shape]
    rec = np.asarray(w.rec)
    lat = [0, 2] if dims == 2 else [0, 1, 2]
    ext = inner if dims == 3 else [inner[0], 0.0, inner[1]]
    for a in lat:
        assert rec[:, a].min() >= 0.0 and rec[:, a].max() <= ext[a] + 1e-6
        assert 0.0 <= w.src[a] <= ext[a]


def test_batched_apertures_shapes_and_placement():
    from paper_1810_05268_gb300 import synth
    vel, wins = synth.batched_apertures(nshots=6, survey=(64, 80, 80), small=(32, 32, 32), large=(48, 56, 64))
    assert len(wins) == 6
    sizes = sorted(w.shape for w in wins)
    assert sizes[0] == (32, 32, 32) and sizes[-1] == (48, 56, 64)
    for w in wins:
        assert all(s % 8 == 0 for s in w.shape)
        assert all(o >= 0 and o + s <= n for o, s, n in zip(w.offset, w.shape, vel.shape))
        sl = tuple(slice(o, o + s) for o, s in zip(w.offset, w.shape))
        assert np.array_equal(w.vel, vel[sl])
    assert 1.5 <= vel.min() and vel.max() <= 4.5
    vel2, wins2 = synth.batched_apertures(nshots=6, survey=(64, 80, 80), small=(32, 32, 32), large=(48, 56, 64))
    assert np.array_equal(vel, vel2) and [w.offset for w in wins] == [w.offset for w in wins2]
