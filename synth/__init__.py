"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds geometry and noise generators only: icospheres, spherical-
harmonic radial deformations, axis-aligned boxes, tissue packing and detector
noise. None of the renderer's arithmetic (mesh Fourier transform, transfer
function, inverse transform, loss, adjoint) lives here, so both the CPU oracle
and the CUDA path can consume these inputs without sharing method code.
"""

from .meshes import (
    icosphere,
    sphere_mesh,
    sh_deformed_sphere,
    sh_radius,
    box_mesh,
    box_foam,
    scale_about,
    random_triangles,
    pack_cells,
)
from .images import add_gaussian_noise, add_poisson_gaussian_noise, random_half_spectrum
from .configs import Grid, Psf, config_c1, config_c2, config_c3, config_c4_cells, config_c5_job

__all__ = [
    "icosphere",
    "sphere_mesh",
    "sh_deformed_sphere",
    "sh_radius",
    "box_mesh",
    "box_foam",
    "scale_about",
    "random_triangles",
    "pack_cells",
    "add_gaussian_noise",
    "add_poisson_gaussian_noise",
    "random_half_spectrum",
    "Grid",
    "Psf",
    "config_c1",
    "config_c2",
    "config_c3",
    "config_c4_cells",
    "config_c5_job",
]
