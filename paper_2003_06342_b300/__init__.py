"""B300-native lattice Boltzmann phase-field solver for two-phase flow with
phase change (Verdier, Kestener & Cartalade, arXiv:2003.06342).

The per-step hot path -- conservative Allen-Cahn phase field with the
interfacial production source, incompressible Navier-Stokes with surface
tension and buoyancy, heat equation with the latent-heat source, and the
gradient / Laplacian / chemical-potential stencils -- runs as one fused
sm_103a CUDA kernel per time step behind the C ABI of include/lbm_pf.h.
This package is the thin Python binding of that ABI (argument marshalling,
device memory and streams from PyTorch).
"""
from .solver import Solver, make_params, make_grid, workspace_bytes  # noqa: F401
from . import units  # noqa: F401
