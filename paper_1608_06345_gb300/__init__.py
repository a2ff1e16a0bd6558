"""GB300-native double-distribution thermal lattice Boltzmann library.

Implements the fused pull-stream + BGK-collide step of Hu, Zhang & Geng's
thermal lattice Boltzmann scheme with flexible specific-heat ratio
(arXiv 1608.06345) on the D2Q37 and D3Q107 velocity sets, as hand-written
CUDA for sm_103a behind the C ABI of ``include/lbm.h``.  ``lbm`` is the thin
Python binding (argument marshalling only).
"""
from . import lbm  # noqa: F401
