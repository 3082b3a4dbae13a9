"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package holds geometry and right-hand-side generators only: triangle
meshes (icosphere, two spheres, unit cube, cube-sphere), their collocation
points and panel areas, and seeded right-hand sides.  It holds none of the
H-matrix method's arithmetic (no kernel entries, no cluster tree, no ACA, no
matrix-vector product, no solver), so both sides can consume identical inputs
without sharing any of the code under test.
"""
from .mesh import (Mesh, icosphere, two_spheres, unit_cube, cube_sphere,
                   uneven_batch_specs, mesh_from_spec)
from .rhs import (splitmix64_uniform, splitmix64_normal, rhs_constant,
                  rhs_one_plus_half_z, rhs_two_spheres, rhs_normal_columns)

__all__ = ["Mesh", "icosphere", "two_spheres", "unit_cube", "cube_sphere",
           "uneven_batch_specs", "mesh_from_spec",
           "splitmix64_uniform", "splitmix64_normal", "rhs_constant",
           "rhs_one_plus_half_z", "rhs_two_spheres", "rhs_normal_columns"]
