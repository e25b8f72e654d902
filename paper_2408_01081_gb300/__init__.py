"""GB300-native vectorial lattice Boltzmann (D2Q4^5) for 2D linear elastodynamics.

Hand-written CUDA kernels for sm_103a behind the C ABI of ``include/lbm.h``;
:mod:`paper_2408_01081_gb300.lbm` is the ctypes binding with the same names.
"""
from . import build  # noqa: F401

__all__ = ["build", "lbm"]
