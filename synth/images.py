"""Seeded detector noise and random spectra (no renderer arithmetic)."""

from __future__ import annotations

import numpy as np


def add_gaussian_noise(img: np.ndarray, rel_sigma: float, seed: int) -> np.ndarray:
    """i.i.d. N(0, (rel_sigma * max(img))^2) added to every voxel."""
    rng = np.random.default_rng(seed)
    peak = float(np.max(img))
    return img + rng.normal(0.0, rel_sigma * peak, size=img.shape)


def add_poisson_gaussian_noise(img: np.ndarray, peak_counts: float, read_sigma: float, seed: int):
    """Scale to ``peak_counts`` at the maximum, draw Poisson photon counts, add N(0, read_sigma^2).

    Returns ``(noisy, scale)`` with ``noisy ~ Poisson(scale * img) + N(0, read_sigma^2)``.
    """
    rng = np.random.default_rng(seed)
    scale = peak_counts / float(np.max(img))
    lam = np.clip(scale * img, 0.0, None)
    noisy = rng.poisson(lam).astype(np.float64) + rng.normal(0.0, read_sigma, size=img.shape)
    return noisy, scale


def random_half_spectrum(n, seed: int) -> np.ndarray:
    """Complex array of shape (Nx, Ny, Nz//2 + 1) with i.i.d. standard normal parts."""
    nx, ny, nz = (int(v) for v in n)
    rng = np.random.default_rng(seed)
    shape = (nx, ny, nz // 2 + 1)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
