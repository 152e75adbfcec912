"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds no arithmetic of the method itself (no quadrature points,
no Green's function, no expansions): only surface meshes, random densities and
incident directions, each a pure function of its arguments and seed.
"""
from .meshes import (  # noqa: F401
    icosphere,
    bisect_longest_edges,
    sphere_mesh,
    refined_cap_sphere,
    ellipsoid_mesh,
    star_mesh,
    geodesic_sphere,
    triangle_soup,
    corner_lattice_soup,
    serving_shape,
    serving_requests,
    workload_mesh,
    WORKLOADS,
)
from .fields import random_density, fibonacci_directions  # noqa: F401
