"""CKFWI_DEBUG=1: the executor checks, on the host and before every step
launch, that each field a step reads or writes lies inside the allocation
its role names and that no step writes a field it reads.  Every schedule
and storage placement passes those checks, and the checked gradients are
bitwise the unchecked ones."""
import os

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


def _run(m, case, d, kw):
    if kw.pop("batch", False):
        s = case.shot()
        _, g, _ = m.batch_gradient([s, s], [d, d], **kw)
        return g.clone()
    _, g, _ = m.adjoint_gradient(case.shot(), d, **kw)
    return g.clone()


@pytest.mark.parametrize("time_order", [2, 4])
def test_debug_checks_pass_and_change_nothing(time_order):
    case = make_case(3, 8, (35, 43, 70), 8, 60, seed=3, time_order=time_order)
    m = C.Model(case.pg)
    m.set_model(torch.from_numpy(case.vel).cuda())
    d = m.forward_shot(case.shot()) * 1.02
    configs = [dict(ckpt_slots=60), dict(ckpt_slots=7), dict(ckpt_slots=7, store_mode="fp16"),
               dict(ckpt_slots=7, store_mode="bf16", host_slots=3),
               dict(ckpt_slots=7, store_mode="codec", tol=1e-4),
               dict(ckpt_slots=12, host_slots=8), dict(ckpt_slots=12, host_slots=11, use_graph=True),
               dict(ckpt_slots=7, store_mode="fp16", batch=True)]
    for kw in configs:
        g0 = _run(m, case, d, dict(kw))
        os.environ["CKFWI_DEBUG"] = "1"
        try:
            g1 = _run(m, case, d, dict(kw))
        finally:
            del os.environ["CKFWI_DEBUG"]
        assert torch.equal(g0, g1), kw
    m.close()
