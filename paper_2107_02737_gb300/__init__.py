"""GB300-native DNN-SP2 density-matrix solver (arXiv 2107.02737, electronic-structure hot path).

``sp2`` binds the C ABI of ``libsp2.so`` (include/sp2.h): ``density``, ``response``,
``adjoint``, ``density_batched``, ``apply_layers`` and the ``DensityMatrix``
autograd function.  ``inputs`` builds seeded synthetic Hamiltonians.  ``build``
compiles the CUDA library for sm_103a.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "sp2", "build"]
