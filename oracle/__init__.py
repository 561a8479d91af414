"""FP64 CPU oracle of the checkpointed, compressed adjoint gradient.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import anything under oracle/.
The product path (paper_1810_05268_gb300) never imports it and shares no
code with it: the oracle computes its own stencil weights, damping, Ricker
wavelet, interpolation weights, Revolve schedule and codec from the paper
(Sec. 3 Eq. "eqn:recompute", Sec. 4, Sec. 6 Eq. "eqn:wave") and from the
readings listed in the headers of fwi_oracle.c and codec_oracle.c.

Modules
  oracle.propagator  forward modelling, adjoint, misfit and gradient (C, FP64)
  oracle.revolve     binomial checkpointing schedule and its counts (Python)
  oracle.codec       fixed-accuracy 4^d block-transform codec (C, integer)
  oracle.checkpointed  the gradient a Revolve executor computes when its
                     checkpoints are stored rounded or compressed (Python
                     over the C steps)
"""
