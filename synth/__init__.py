"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package only *generates inputs*: triangulated closed surfaces (the
unit sphere and its perturbed / ellipsoidal relatives that the paper's
experiments use, Sect. 2 and Sect. 8), right-hand sides and exterior field
points.  It contains none of the method's arithmetic (no kernel function,
no quadrature, no clustering, no cross approximation), so both sides can
import it without sharing any part of the computation they are compared on.
"""

from .meshes import (  # noqa: F401
    icosahedron,
    icosphere,
    subdivided_icosahedron,
    perturb_sphere,
    scale_axes,
    mesh_for_config,
    edge_midpoints_for_config,
    batch_meshes,
)
from .rhs import uniform_rhs, normal_rhs, exterior_points  # noqa: F401
