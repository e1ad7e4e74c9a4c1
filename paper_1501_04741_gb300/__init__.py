"""GB300-native adjoint Lattice Boltzmann (Laniewski-Wollk & Rokicki).

The compute path is the C-ABI library ``libalbm.so`` (hand-written sm_103a
CUDA kernels, built by :mod:`paper_1501_04741_gb300.build`); the Python
binding in :mod:`paper_1501_04741_gb300.albm` marshals arguments only.
Importing this package does not load the library; ``albm`` does, and fails
loudly when it is missing.
"""
__all__ = ["inputs"]
