"""Seeded synthetic workloads (meshes, bathymetry, initial fields).

This package produces *inputs* only: triangle meshes, bathymetry, layer counts,
boundary tags and initial nodal fields.  It holds none of the discretisation's
arithmetic (no quadrature, no fluxes, no mass matrices), so that both the CPU
oracle and the CUDA library can consume the same inputs without sharing any
computation.  Every generator is deterministic for a given seed.
"""
from .meshes import (Mesh, square_mesh, basin_mesh, graded_mesh, hilbert_order, permute_triangles,
                     c1_mesh, c2_mesh, c4_mesh, c5_mesh, cached_mesh)
from .fields import (node_positions_sigma, c1_velocity, c1_tracer, c2_initial_state, basin_velocity,
                     c4_initial_state, c5_initial_state, WORKLOADS)

__all__ = ["Mesh", "square_mesh", "basin_mesh", "hilbert_order", "permute_triangles",
           "graded_mesh", "c1_mesh", "c2_mesh", "c4_mesh", "c5_mesh", "cached_mesh",
           "node_positions_sigma", "c1_velocity", "c1_tracer", "c2_initial_state", "basin_velocity",
           "c4_initial_state", "c5_initial_state", "WORKLOADS"]
