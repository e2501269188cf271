"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds input generation only: octree leaf lists (top-down
refinement by a predicate, then 2:1 balancing) and nodal fields evaluated at
node coordinates that the caller supplies.  It contains none of the CHNS
method's arithmetic (no basis functions, quadrature, residual terms or
solvers), so both sides can import it without sharing numerical code.
"""
from .octree import (uniform_leaves, refine_leaves, balance_leaves, sphere_band_leaves,
                     plane_band_leaves, morton_encode, leaves_to_array, graded_band_leaves, layer_distance)
from .fields import (drop_phi, fourier_velocity, layer_phi, random_vectors, config_params, two_drops)

__all__ = [
    "uniform_leaves", "refine_leaves", "balance_leaves", "sphere_band_leaves", "graded_band_leaves",
    "layer_distance",
    "plane_band_leaves", "morton_encode", "leaves_to_array", "drop_phi", "fourier_velocity",
    "layer_phi", "random_vectors", "config_params", "two_drops",
]
