"""Two storage levels (multi-level checkpointing, a future-work item of
Sec. 8): Revolve slots placed in pinned host memory, read and written by the
step kernels over the host link.  Placement changes cost, never
values: the gradient with host slots is bitwise the all-device one."""
import numpy as np
import pytest

from gpu_cases import make_case

torch = pytest.importorskip("torch")
C = pytest.importorskip("paper_1810_05268_gb300.ckfwi")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("dims,so,shape,nbl,nt", [(3, 8, (35, 43, 70), 8, 90), (2, 8, (66, 131), 12, 200),
                                                  (3, 16, (41, 46, 53), 8, 80)])
@pytest.mark.parametrize("mode", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_host_slots_bitwise_equal_device_slots(dims, so, shape, nbl, nt, mode, use_graph):
    case = make_case(dims, so, shape, nbl, nt, seed=so + dims)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    d = m.forward_shot(case.shot()) * 1.02
    slots = 9
    phi0, g0, st0 = m.adjoint_gradient(case.shot(), d, slots, store_mode=mode, use_graph=use_graph)
    for hs in (1, 4, slots - 1, 50):
        phi, g, st = m.adjoint_gradient(case.shot(), d, slots, store_mode=mode, use_graph=use_graph,
                                        host_slots=hs)
        assert phi == phi0
        assert torch.equal(g, g0)
        assert st["p"] == st0["p"]
    # back to device slots after host ones (the pools keep zero halos)
    phi1, g1, _ = m.adjoint_gradient(case.shot(), d, slots, store_mode=mode, use_graph=use_graph)
    assert phi1 == phi0 and torch.equal(g1, g0)


def test_more_slots_in_host_memory_cut_recomputation():
    case = make_case(3, 8, (35, 43, 70), 8, 120, seed=5)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    d = m.forward_shot(case.shot()) * 1.02
    _, g_a, st_a = m.adjoint_gradient(case.shot(), d, 6)
    _, g_b, st_b = m.adjoint_gradient(case.shot(), d, 30, host_slots=24)
    assert st_b["fwd_steps"] < st_a["fwd_steps"]
    assert torch.equal(g_a, g_b)
