"""torch.autograd wrapper: forward = library misfit, backward = checkpointed
adjoint (Sec. 6 gradient by the adjoint-state method; Sec. 3 checkpoints),
checked against the FP64 oracle and by finite differences."""
import numpy as np
import pytest

from gpu_cases import make_case, misfit_tol, rel_l2
from oracle import propagator as O

torch = pytest.importorskip("torch")
C = pytest.importorskip("paper_1810_05268_gb300.ckfwi")
A = pytest.importorskip("paper_1810_05268_gb300.autograd")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()


def _problem(nshots=3):
    case = make_case(2, 8, shape=(60, 120), nbl=10, nt=260, seed=31)
    inner_x = (120 - 2 * 10 - 1) * case.og.h
    srcs = [(20.0, 0.0, x) for x in np.linspace(0.15, 0.85, nshots) * inner_x]
    # a start model 4% slow everywhere: the residual is of the size of the
    # data (with |r| << |d| the FP32 residual's relative error ~1e-5 |d|/|r|
    # would bound the gradient's accuracy instead)
    true = case.vel.astype(np.float64) * 1.04
    true[30:, :] *= 1.06
    shots, dobs, ser = [], [], case.oracle_series()
    for s in srcs:
        shots.append(C.ShotSpec(src=s, rec=case.rec, f0=case.f0, t0=case.t0))
        dobs.append(O.forward(case.og, true, [s], ser, case.rec).astype(np.float32))
    return case, srcs, shots, dobs


def test_misfit_and_gradient_match_oracle_sum():
    case, srcs, shots, dobs = _problem()
    m = C.Model(case.pg)
    m0 = torch.from_numpy((1.0 / case.vel.astype(np.float64) ** 2).astype(np.float32)).cuda().requires_grad_(True)
    dd = [torch.from_numpy(d).cuda() for d in dobs]
    phi = A.misfit(m0, m, shots, dd, ckpt_slots=7)
    phi.backward()
    vel = (1.0 / np.sqrt(m0.detach().cpu().numpy().astype(np.float64)))
    phi_ref, g_ref, tol = 0.0, np.zeros(case.vel.shape), 0.0
    for s, d in zip(srcs, dobs):
        p, g, dsim = O.gradient(case.og, vel, [s], case.oracle_series(), case.rec, d.astype(np.float64))
        phi_ref += p
        g_ref += g
        tol += misfit_tol(dsim, p)
    phi = float(phi.detach())
    eg = rel_l2(m0.grad.cpu().numpy(), g_ref)
    print("misfit %.9e vs oracle %.9e (tol %.2e); gradient rel-L2 %.3e" % (phi, phi_ref, tol, eg))
    assert abs(phi - phi_ref) <= tol
    assert eg <= 1e-4


def test_gradient_directional_derivative_by_finite_differences():
    case, srcs, shots, dobs = _problem(2)
    m = C.Model(case.pg)
    dd = [torch.from_numpy(d).cuda() for d in dobs]
    m0 = torch.from_numpy((1.0 / case.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    x = m0.clone().requires_grad_(True)
    phi = A.misfit(x, m, shots, dd, ckpt_slots=260)
    (g,) = torch.autograd.grad(phi, x)
    from paper_1810_05268_gb300 import synth
    dm = torch.from_numpy((synth.smooth_perturbation(case.vel.shape, 4.0, 5) * 0.01).astype(np.float32)).cuda() * m0
    an = float((g.double() * dm.double()).sum())
    rel = {}
    for eps in (0.5, 0.2):
        with torch.no_grad():
            fp = float(A.misfit(m0 + eps * dm, m, shots, dd, ckpt_slots=260))
            fm = float(A.misfit(m0 - eps * dm, m, shots, dd, ckpt_slots=260))
        rel[eps] = abs((fp - fm) / (2 * eps) - an) / abs(an)
    print("central differences against the adjoint: relative difference %s" % rel)
    # measured on a GB300: 2.2e-4 and 2.9e-4
    assert rel[0.5] <= 1e-3 and rel[0.2] <= 1e-3, rel


def test_backward_scales_with_grad_output():
    case, srcs, shots, dobs = _problem(2)
    m = C.Model(case.pg)
    dd = [torch.from_numpy(d).cuda() for d in dobs]
    m0 = torch.from_numpy((1.0 / case.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    x = m0.clone().requires_grad_(True)
    (g1,) = torch.autograd.grad(A.misfit(x, m, shots, dd, ckpt_slots=9), x)
    (g3,) = torch.autograd.grad(3.0 * A.misfit(x, m, shots, dd, ckpt_slots=9), x)
    assert torch.allclose(g3, 3.0 * g1, rtol=1e-6, atol=0)
    (g0,) = torch.autograd.grad(0.0 * A.misfit(x, m, shots, dd, ckpt_slots=9), x)
    assert not bool(g0.any())


def test_steepest_descent_reduces_misfit():
    case, srcs, shots, dobs = _problem(3)
    m = C.Model(case.pg)
    dd = [torch.from_numpy(d).cuda() for d in dobs]
    m0 = torch.from_numpy((1.0 / case.vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    mf, hist = A.steepest_descent(m0, m, shots, dd, iterations=3, ckpt_slots=9, step=0.02,
                                  store_mode="codec", tol=1e-7, pool_bytes=64 << 20)
    print("misfit history", hist)
    assert hist[-1] < 0.9 * hist[0]
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert all(np.isfinite(hist))
