"""CPU FP64 oracle for the SP2 density-matrix path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it, and shares no code with it.

Contents
--------
``density``  The definition the method converges to: D = theta(mu I - H) from a
             dense symmetric eigendecomposition (Eq. DM-outer-product and
             Eq. theta of the section "The density matrix"), the chemical
             potential, the band energy Tr[DH], and the first-order response
             D1 and adjoint dTr[DG]/dH from eigenbasis perturbation theory.
``sp2``      The DNN-SP2 chain itself in FP64 (Eq. Deep_NN and the layer rule of
             the section "Deep-neural network electronic structure solver"):
             Gershgorin bounds, the input layer, the trace-correcting layer
             choice, the stop rule, the same chain applied to scalar eigenvalues,
             and the chain's own response, adjoint and divided-difference
             derivative.

Every function works in float64 with plain NumPy/LAPACK calls so that it can be
checked against the paper by eye.  The pins that tie it to something other than
itself live in ``tests/test_oracle_*.py``.
"""
from . import density, sp2  # noqa: F401
