"""X-Gaussian Differentiable Radiative Rasterization on GB300 (sm_103a).

The compute path is the C-ABI library ``libxg.so`` built from ``csrc/``; ``binding``
marshals arguments into it, ``render`` wraps it as a ``torch.autograd.Function`` and
``batch`` captures whole multi-view steps in CUDA graphs.  ``synth`` generates the
seeded synthetic inputs.
"""
__all__ = ["synth"]
