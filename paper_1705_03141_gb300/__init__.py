"""GB300-native D3Q27 colour-fluid lattice Boltzmann update.

Implements, as hand-written CUDA for sm_103a behind the C ABI of
include/lbm.h, the per-node, per-step update of the colour-fluid model of
Saito, Abe & Koyama, "Lattice Boltzmann modeling and simulation of liquid jet
breakup" (arXiv 1705.03141): D3Q27 MRT collision with the enhanced
equilibrium (Sec. II), MRT body forcing, the generalised perturbation
operator, recolouring, streaming and the jet boundaries of Sec. IV.A.

``Lattice`` is the Python binding (argument marshalling only); ``build``
compiles the library.
"""
from .lbm import (Batch, Lattice, LbmError, STORAGE, SYMBOLS, library, moment_matrix, selfcheck, diag_fields_static,  # noqa: F401,E501
                  measure_fp32_peak, selftest_tma,
                  BC_PERIODIC, BC_NOSLIP, BC_FREESLIP, BC_INFLOW_WALL, BC_OUTFLOW, BC_HALO)
from . import slabs  # noqa: F401
from .build import build as build_library  # noqa: F401
from .mlp import Mlp  # noqa: F401
