"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only manufactures input data: a crystal cell, a Gamma-centred
k mesh, plane-wave Bloch coefficients C_G(k) and band energies E(k) from an
empirical pseudopotential, frequency lists and optional cRPA weights T.
It holds no step of the polarization / screened-interaction method itself.
"""
from .epm import (HARTREE_EV, Cell, Bands, fcc_cell, sc_cell, kmesh_frac,
                  psi_sphere, make_bands)
from .configs import CONFIGS, Workload, make_workload
from .metal import metal_bands, metal_view

__all__ = ["HARTREE_EV", "Cell", "Bands", "fcc_cell", "sc_cell", "kmesh_frac",
           "psi_sphere", "make_bands", "CONFIGS", "Workload", "make_workload",
           "metal_bands", "metal_view"]
