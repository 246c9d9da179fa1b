"""GB300 (sm_103a) implementation of the BTDF immersed-boundary lattice
Boltzmann time step (Jiang & Liu, arXiv 1806.09403) behind a C ABI.

``btdf`` is the ctypes binding of ``include/btdf.h``; the compute path is the
CUDA library built in-tree by ``_build.build()``.
"""
from . import btdf  # noqa: F401
