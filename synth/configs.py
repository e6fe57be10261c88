"""Workload recipes: the meshes, grids and PSF parameters of the five benchmark cases.

Everything here is a seeded recipe of inputs. Target images are produced by a
renderer (the oracle in tests, the CUDA path in the benchmark) from the meshes
returned here; this module never renders.

Readings of the workload text (all lengths in micrometres unless noted):
* case 1 works in voxel units (h = 1);
* cases 2-5 use voxels (0.5, 0.5, 1.0); "radius 30 voxels" means 30 * h_x = 15;
* case 3 uses radius 30, true sigma (0.25, 0.25, 0.7) and initial sigma (0.3, 0.3, 0.9);
* case 4 draws icosphere levels uniformly from {3, 4, 5} (log-uniform over the
  attainable triangle counts 1280..20480) and crops 64/96/128-voxel cubes by radius;
* case 5 draws levels from {2..6} and grid sides log-uniformly from {64, 96, 128, 192, 256}.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .meshes import pack_cells, sh_deformed_sphere, sphere_mesh


@dataclass
class Grid:
    n: tuple  # voxels per axis (Nx, Ny, Nz); arrays are C-ordered [x][y][z]
    h: tuple  # voxel size per axis
    origin: tuple = (0.0, 0.0, 0.0)  # position of voxel (0, 0, 0)

    @property
    def L(self) -> np.ndarray:
        return np.asarray(self.n, dtype=np.float64) * np.asarray(self.h, dtype=np.float64)

    @property
    def center(self) -> np.ndarray:
        return np.asarray(self.origin) + 0.5 * self.L


@dataclass
class Psf:
    sigma: tuple  # spatial standard deviations of the Gaussian PSF per axis
    band_tau: float = 0.0  # keep frequencies with OTF > tau * max OTF; 0 keeps all
    cov: tuple = field(default=None)  # optional full covariance (xx, yy, zz, xy, xz, yz)


@dataclass
class Case:
    name: str
    grid: Grid
    psf: Psf
    V_true: np.ndarray
    F: np.ndarray
    V_init: np.ndarray
    loss: str = "mse"
    psf_init: Psf | None = None
    noise: dict = field(default_factory=dict)


def config_c1() -> Case:
    """Icosphere level 2, R = 10 voxels, centred in 32^3 (h = 1), sigma (1, 1, 2.5), full spectrum."""
    g = Grid(n=(32, 32, 32), h=(1.0, 1.0, 1.0))
    V, F = sphere_mesh(2, 10.0, g.center)
    from .meshes import scale_about

    V_t = scale_about(V, (1.1, 0.9, 1.0), g.center)
    return Case(
        "c1_icosphere2_32cube",
        g,
        Psf(sigma=(1.0, 1.0, 2.5), band_tau=0.0),
        V_true=V_t,
        F=F,
        V_init=V,
        noise={"kind": "gaussian", "rel_sigma": 0.05, "seed": 0},
    )


def config_c2(seed: int = 2) -> Case:
    """Icosphere level 4 (5120 triangles), R = 15, SH l <= 6, 128^3, h (0.5, 0.5, 1), sigma (0.2, 0.2, 0.6), tau 1e-3."""
    g = Grid(n=(128, 128, 128), h=(0.5, 0.5, 1.0))
    R = 30 * g.h[0]
    V_t, F = sh_deformed_sphere(4, R, g.center, lmax=6, coef_sigma=0.03 * R, seed=seed)
    V0, _ = sphere_mesh(4, R, g.center)
    return Case("c2_cell_sh6_128cube", g, Psf(sigma=(0.2, 0.2, 0.6), band_tau=1e-3), V_t, F, V0)


def config_c3(seed: int = 3) -> Case:
    """Icosphere level 5 (20480 triangles), R = 30, SH l <= 10, 256x256x128, h (0.5, 0.5, 1)."""
    g = Grid(n=(256, 256, 128), h=(0.5, 0.5, 1.0))
    R = 30.0
    V_t, F = sh_deformed_sphere(5, R, g.center, lmax=10, coef_sigma=0.03 * R, seed=seed)
    V0, _ = sphere_mesh(5, R, g.center)
    return Case(
        "c3_cell_sh10_256x256x128",
        g,
        Psf(sigma=(0.25, 0.25, 0.7), band_tau=0.0),
        V_t,
        F,
        V0,
        psf_init=Psf(sigma=(0.3, 0.3, 0.9), band_tau=0.0),
    )


def config_c4_cells(seed: int = 4, n_cells: int = 32):
    """32 SH-deformed cells packed in a 256^3 (h 0.5, 0.5, 1) tissue; one cropped fit job per cell.

    Returns a list of dicts with the crop ``Grid`` (origin at the crop corner,
    in tissue coordinates), the true and initial meshes and the PSF.
    """
    h = (0.5, 0.5, 1.0)
    tissue = Grid(n=(256, 256, 256), h=h)
    sigma = (0.25, 0.25, 0.7)
    rng = np.random.default_rng(seed)
    levels = rng.integers(3, 6, size=n_cells)
    cells = pack_cells(n_cells, tissue.L, (8.0, 20.0), 2 * sigma[2], seed + 1000)
    jobs = []
    for k, ((c, r), lev) in enumerate(zip(cells, levels)):
        side = next((s for s in (64, 96, 128) if s * h[0] >= 2 * r + 6.0), 128)
        n = (side, side, side)
        L = np.asarray(n) * np.asarray(h)
        origin = tuple(np.asarray(c) - 0.5 * L)
        grid = Grid(n=n, h=h, origin=origin)
        V_t, F = sh_deformed_sphere(int(lev), r, c, lmax=6, coef_sigma=0.03 * r, seed=seed * 100 + k)
        V0, _ = sphere_mesh(int(lev), r, c)
        jobs.append(dict(grid=grid, psf=Psf(sigma=sigma, band_tau=1e-3), V_true=V_t, F=F, V_init=V0, level=int(lev)))
    return tissue, jobs


def config_c5_job(rng: np.random.Generator, job_id: int):
    """One serving request: level in {2..6}, side in {64, 96, 128, 192, 256}, random anisotropic PSF."""
    lev = int(rng.integers(2, 7))
    side = int(rng.choice([64, 96, 128, 192, 256]))
    h = (0.5, 0.5, 1.0)
    n = (side, side, side)
    grid = Grid(n=n, h=h)
    sxy = float(rng.uniform(0.15, 0.3))
    sz = float(rng.uniform(0.4, 0.9))
    R = 0.3 * float(min(grid.L))  # x/y extent bounds the cell
    V_t, F = sh_deformed_sphere(lev, R, grid.center, lmax=6, coef_sigma=0.03 * R, seed=10_000 + job_id)
    V0, _ = sphere_mesh(lev, R, grid.center)
    return dict(grid=grid, psf=Psf(sigma=(sxy, sxy, sz), band_tau=1e-3), V_true=V_t, F=F, V_init=V0, level=lev)
