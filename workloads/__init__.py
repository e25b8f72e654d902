"""Seeded synthetic input generators shared by the oracle tests, the GPU tests and the benchmark.

This package holds no arithmetic of the lattice Boltzmann scheme: it only
builds the problem data (manufactured solutions, Gaussian random fields,
material constants, batch layouts) that the paper's experiments feed into it.
"""
from . import grf, material, mms  # noqa: F401
from .configs import (LatticeSpec, Workload, batch_spec, dirichlet_mms, energy_box, plane_wave_periodic,  # noqa: F401
                      grf_periodic, periodic_mms)
