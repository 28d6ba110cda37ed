"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds no arithmetic of the hybridisation method: it only makes
meshes (vertex coordinates and simplices), smooth source terms, their element
means f̄_K (the data the method consumes through R_K, Section 3.1), and the
velocity field about which a Navier-Stokes step is linearised.  Both sides of
every parity test receive the same arrays from here.

Stand-ins: the paper's 2D runs use the triangular "Mesh1" family of a public
benchmark, which is not available; structured, optionally perturbed squares
split into two triangles take its place.  The 3D runs of the paper use cubes
split into 6 tetrahedra (Section 4.1), which ``mesh3d_kuhn`` reproduces.
"""

from .mesh import mesh2d_square, mesh3d_kuhn, batch_sizes
from .fields import (
    fourier_modes,
    fourier_force,
    element_means,
    manufactured_stokes,
    stream_velocity,
    config_problem,
    batch_problems,
)

__all__ = [
    "mesh2d_square",
    "mesh3d_kuhn",
    "batch_sizes",
    "fourier_modes",
    "fourier_force",
    "element_means",
    "manufactured_stokes",
    "stream_velocity",
    "config_problem",
    "batch_problems",
]
