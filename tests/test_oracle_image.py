"""Pins of the oracle's spectral image model (Eq. 1 in Fourier space, Eq. 2 OTF, Section 5.1 band)
and of its loss/gradient chain (Section 5.1-5.2, Eq. 6).

References: a direct double sum (no FFT), unit total intensity (Eq. 3), the
dot-product identity of the image adjoint, finite differences of the full loss,
and the Gaussian convolution limit for an isolated sphere.
"""

import numpy as np
import pytest

import oracle
import synth


def _small_case(n=(12, 10, 9), h=(1.0, 1.2, 1.5), sigma=(0.9, 1.1, 1.6), tau=0.0, level=2, seed=0):
    grid = synth.Grid(n=n, h=h, origin=(0.3, -0.4, 0.2))
    V, F = synth.sh_deformed_sphere(level, 0.27 * min(grid.L), grid.center, lmax=3, coef_sigma=0.3, seed=seed)
    return grid, synth.Psf(sigma=sigma, band_tau=tau), V, F


@pytest.mark.parametrize("n", [(8, 8, 8), (12, 10, 9), (9, 7, 6), (16, 8, 12)])
def test_fft_image_matches_direct_sum(n):
    grid, psf, V, F = _small_case(n=n)
    r = oracle.render(V, F, grid, psf)
    direct = oracle.spectrum_to_image(r["X"], r["nvec"], r["c"], grid, method="dft")
    assert np.max(np.abs(r["image"] - direct)) <= 1e-12 * np.max(np.abs(direct))


@pytest.mark.parametrize("mode", ["surface", "volume"])
def test_unit_total_intensity(mode):
    grid, psf, V, F = _small_case()
    img = oracle.render(V, F, grid, psf, mode)["image"]
    assert abs(img.sum() * np.prod(grid.h) - 1.0) < 1e-12


def test_narrow_band_keeps_only_strong_otf():
    grid, psf, V, F = _small_case(n=(16, 16, 16), h=(1, 1, 1), sigma=(1.5, 1.5, 2.0), tau=1e-2)
    r = oracle.render(V, F, grid, psf)
    nvec, _ = oracle.half_spectrum(grid.n)
    h_all = oracle.otf(oracle.wavevectors(nvec, grid), psf)
    assert r["band"].sum() == np.sum(h_all > 1e-2) and 0 < r["band"].sum() < len(h_all)
    full = oracle.render(V, F, grid, synth.Psf(sigma=psf.sigma, band_tau=0.0))["image"]
    # the dropped components carry h_hat <= tau: the truncated image stays close
    assert np.linalg.norm(r["image"] - full) < 2e-2 * np.linalg.norm(full)


def test_image_adjoint_dot_product():
    grid, psf, V, F = _small_case(n=(10, 12, 8))
    nvec, c = oracle.half_spectrum(grid.n)
    rng = np.random.default_rng(4)
    X = rng.normal(size=len(c)) + 1j * rng.normal(size=len(c))
    R = rng.normal(size=grid.n)
    I = oracle.spectrum_to_image(X, nvec, c, grid)
    G = oracle.image_adjoint(R, nvec, c, grid)
    assert abs(np.sum(I * R) - np.sum(np.real(np.conj(G) * X))) < 1e-10 * np.sum(np.abs(I * R))


def test_sphere_image_approaches_gaussian_blurred_shell():
    """Far from the box walls, the image is the shell density convolved with the Gaussian (Eq. 1).

    The icosphere error shrinks ~4x per subdivision level.
    """
    grid = synth.Grid(n=(32, 32, 32), h=(1.0, 1.0, 1.0))
    R, sig = 6.0, 1.2
    j = np.arange(32) + 0.0
    r = np.abs(j - grid.center[0])
    sel = r > 0.4
    # radial profile of a uniform unit-mass shell blurred by an isotropic Gaussian
    ref = (np.exp(-((r[sel] - R) ** 2) / (2 * sig**2)) - np.exp(-((r[sel] + R) ** 2) / (2 * sig**2))) / (
        4 * np.pi * R * r[sel] * np.sqrt(2 * np.pi) * sig
    )
    errs = []
    for lev in (3, 4):
        V, F = synth.sphere_mesh(lev, R, grid.center)
        prof = oracle.render(V, F, grid, synth.Psf(sigma=(sig, sig, sig)))["image"][:, 16, 16]
        errs.append(np.max(np.abs(prof[sel] - ref)) / np.max(ref))
    assert errs[1] < 5e-3 and errs[0] / errs[1] > 3.0, errs


@pytest.mark.parametrize("kind", ["l2", "mse", "weighted"])
@pytest.mark.parametrize("mode", ["surface", "volume"])
def test_loss_gradient_matches_finite_differences(kind, mode):
    grid, psf, V, F = _small_case(n=(10, 9, 8), level=1)
    T = oracle.render(V * 1.03 + 0.05, F, grid, psf, mode)["image"]
    T = synth.add_gaussian_noise(T, 0.05, seed=3)
    L, dV, dpsf, _ = oracle.loss_and_grad(V, F, grid, psf, T, kind, mode)
    rng = np.random.default_rng(8)
    h = 1e-6

    def Lof(W, p):
        return oracle.loss_value(oracle.render(W, F, grid, p, mode)["image"], T, kind)[0]

    for _ in range(4):
        d = rng.normal(size=V.shape)
        fd = (Lof(V + h * d, psf) - Lof(V - h * d, psf)) / (2 * h)
        assert abs(np.sum(dV * d) - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(dV).sum())
    for a in range(3):
        sp = list(psf.sigma)
        sm = list(psf.sigma)
        sp[a] += h
        sm[a] -= h
        fd = (Lof(V, synth.Psf(sigma=tuple(sp))) - Lof(V, synth.Psf(sigma=tuple(sm)))) / (2 * h)
        assert abs(dpsf[a] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(dpsf).sum())


def test_full_covariance_gradient_matches_finite_differences():
    grid, _, V, F = _small_case(n=(10, 9, 8), level=1)
    cov = (0.9, 1.1, 1.7, 0.2, -0.1, 0.15)
    psf = synth.Psf(sigma=(1, 1, 1), cov=cov)
    T = oracle.render(V * 0.97, F, grid, psf)["image"]
    L, dV, dcov, _ = oracle.loss_and_grad(V, F, grid, psf, T, "l2")
    h = 1e-6
    for k in range(6):
        cp, cm = list(cov), list(cov)
        cp[k] += h
        cm[k] -= h
        Lp = oracle.loss_value(oracle.render(V, F, grid, synth.Psf(sigma=(1, 1, 1), cov=tuple(cp)))["image"], T, "l2")[0]
        Lm = oracle.loss_value(oracle.render(V, F, grid, synth.Psf(sigma=(1, 1, 1), cov=tuple(cm)))["image"], T, "l2")[0]
        assert abs(dcov[k] - (Lp - Lm) / (2 * h)) <= 1e-6 * np.abs(dcov).sum()


def _interface_case(seed=11):
    """A cell whose triangles on one side carry two membranes (Section 3.3: a cell-cell interface
    has twice the fluorophore density of a free membrane)."""
    grid, psf, V, F = _small_case(n=(10, 9, 8), level=1, seed=seed)
    cen = V[F].mean(axis=1)
    shared = cen[:, 0] > grid.center[0] + 0.3
    w = np.where(shared, 2.0, 1.0)
    return grid, psf, V, F, shared, w


def test_density_two_equals_a_doubled_sheet():
    """rho_T = 2 is the same surface density as two coincident copies of the triangle."""
    grid, psf, V, F, shared, w = _interface_case()
    F2 = np.concatenate([F, F[shared]])
    a = oracle.render(V, F, grid, psf, weights=w)
    b = oracle.render(V, F2, grid, psf)
    assert abs(a["norm"] - b["norm"]) < 1e-13 * b["norm"]
    assert np.max(np.abs(a["image"] - b["image"])) < 1e-12 * np.max(np.abs(b["image"]))
    T = synth.add_gaussian_noise(oracle.render(V * 1.02, F2, grid, psf)["image"], 0.05, seed=1)
    La, dVa, dpa, _ = oracle.loss_and_grad(V, F, grid, psf, T, "l2", weights=w)
    Lb, dVb, dpb, _ = oracle.loss_and_grad(V, F2, grid, psf, T, "l2")
    assert abs(La - Lb) < 1e-12 * Lb
    assert np.linalg.norm(dVa - dVb) < 1e-11 * np.linalg.norm(dVb)
    assert np.linalg.norm(dpa - dpb) < 1e-11 * np.linalg.norm(dpb)
    # and the interface is visible: the weighted image differs from the unweighted one
    c = oracle.render(V, F, grid, psf)
    assert np.linalg.norm(a["image"] - c["image"]) > 1e-2 * np.linalg.norm(c["image"])


def test_uniform_density_leaves_the_image_unchanged():
    """The image is normalised by sum_T rho_T A_T (Eq. 3 unit mass), so a constant rho cancels."""
    grid, psf, V, F, _, _ = _interface_case()
    a = oracle.render(V, F, grid, psf, weights=np.full(len(F), 3.0))["image"]
    b = oracle.render(V, F, grid, psf)["image"]
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))
    assert abs(a.sum() * np.prod(grid.h) - 1.0) < 1e-12


def test_weighted_loss_gradient_matches_finite_differences():
    grid, psf, V, F, _, _ = _interface_case()
    w = np.random.default_rng(5).uniform(0.5, 2.5, len(F))
    T = synth.add_gaussian_noise(oracle.render(V * 1.03 + 0.05, F, grid, psf)["image"], 0.05, seed=3)
    L, dV, dpsf, _ = oracle.loss_and_grad(V, F, grid, psf, T, "mse", weights=w)
    rng = np.random.default_rng(9)
    h = 1e-6

    def Lof(W, p):
        return oracle.loss_value(oracle.render(W, F, grid, p, weights=w)["image"], T, "mse")[0]

    for _ in range(4):
        d = rng.normal(size=V.shape)
        fd = (Lof(V + h * d, psf) - Lof(V - h * d, psf)) / (2 * h)
        assert abs(np.sum(dV * d) - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(dV).sum())
    sp = list(psf.sigma)
    sm = list(psf.sigma)
    sp[2] += h
    sm[2] -= h
    fd = (Lof(V, synth.Psf(sigma=tuple(sp))) - Lof(V, synth.Psf(sigma=tuple(sm)))) / (2 * h)
    assert abs(dpsf[2] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(dpsf).sum())
