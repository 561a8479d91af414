"""Host logic of the autograd wrapper that needs no GPU: a zero upstream
gradient returns a zero gradient without running the adjoint (the library
reads a gradient scale of 0 as 1)."""
import types

import pytest

torch = pytest.importorskip("torch")


def test_zero_upstream_gradient_skips_the_adjoint():
    from paper_1810_05268_gb300 import autograd as A

    class NoModel:
        def __getattr__(self, name):
            raise AssertionError("the model must not be used for a zero upstream gradient")

    m = torch.full((5, 7), 0.25)
    ctx = types.SimpleNamespace(saved_tensors=(m,), model=NoModel(), shots=[], d_obs=[],
                                opts={"ckpt_slots": 3})
    g, *rest = A.CheckpointedMisfit.backward(ctx, torch.tensor(0.0, dtype=torch.float64))
    assert g.shape == m.shape and not bool(g.any())
    assert rest == [None, None, None, None]
