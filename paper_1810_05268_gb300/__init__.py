"""ckfwi: checkpointed, compressed adjoint-state gradients of acoustic
seismic inversion on GB300 (arXiv 1810.05268).

  paper_1810_05268_gb300.ckfwi     binding of the C-ABI in include/ckfwi.h
  paper_1810_05268_gb300.autograd  torch.autograd.Function around the gradient
  paper_1810_05268_gb300.synth     seeded synthetic models and geometries
  paper_1810_05268_gb300.build     in-tree build of libckfwi.so

Importing the package loads nothing; the CUDA library is loaded on first
use and raises if it is missing.
"""
