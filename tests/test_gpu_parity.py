"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (the benchmark spec): relative L2 image error <= 1e-10 on the FP64 path and
<= 1e-4 on the FP32 path; gradients <= 1e-3 relative L2 on the FP32 path. The
FP64 path's gradients are held to 1e-9. Spectra are compared relative to their
L2 norm and maximum (single small entries of a cancelling sum carry no relative
accuracy in FP32).
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def r64():
    from paper_2303_10440_b300 import Renderer

    r = Renderer("fp64")
    yield r
    r.close()


@pytest.fixture(scope="module")
def r32():
    from paper_2303_10440_b300 import Renderer

    r = Renderer("fp32")
    yield r
    r.close()


def _cuda(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _meshes():
    out = {}
    out["sh_sphere"] = synth.sh_deformed_sphere(2, 6.0, (8.0, 7.5, 9.0), lmax=4, coef_sigma=0.6, seed=1)
    out["box"] = synth.box_mesh((3.0, 4.0, 2.0), (11.0, 9.0, 14.0))  # edges on the axes: e.xi = 0 on grid
    Vt, Ft = synth.random_triangles(40, seed=2, extent=6.0, center=(8, 8, 8))
    out["soup"] = (Vt, Ft)
    # slivers and tiny triangles
    rng = np.random.default_rng(3)
    V = []
    for k in range(30):
        a = rng.uniform(4, 12, 3)
        d = rng.normal(size=3)
        V += [a, a + d * 2.0, a + d * 2.0 + rng.normal(size=3) * (1e-4 if k % 2 else 1e-2)]
    out["slivers"] = (np.array(V), np.arange(90, dtype=np.int32).reshape(30, 3))
    return out


GRID = synth.Grid(n=(16, 16, 16), h=(1.0, 1.0, 1.25), origin=(0.25, -0.5, 0.0))


def _freqs(seed=0, M=300):
    nvec, _ = oracle.half_spectrum(GRID.n)
    rng = np.random.default_rng(seed)
    sel = np.concatenate([[0], rng.choice(len(nvec), size=M - 1, replace=False)])
    return nvec[sel].astype(np.int32)


@pytest.mark.parametrize("name", ["sh_sphere", "box", "soup", "slivers"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_meshft_matches_oracle(name, prec, r64, r32):
    V, F = _meshes()[name]
    fn = _freqs()
    xi = oracle.wavevectors(fn, GRID)
    ref = oracle.mesh_ft(V - np.asarray(GRID.origin), F, xi)
    r = r64 if prec == "fp64" else r32
    S = r.meshft(_cuda(V), _cuda(F), GRID, _cuda(fn)).cpu().numpy()
    tol = 1e-11 if prec == "fp64" else 2e-6
    assert rel(S, ref) < tol
    assert np.max(np.abs(S - ref)) < tol * 10 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_meshft_volume_matches_oracle(prec, r64, r32):
    V, F = synth.sh_deformed_sphere(2, 5.0, (8.0, 8.0, 9.0), lmax=3, coef_sigma=0.4, seed=5)
    fn = _freqs(1)
    xi = oracle.wavevectors(fn, GRID)
    ref = oracle.mesh_ft(V - np.asarray(GRID.origin), F, xi, "volume", c0=0.5 * GRID.L)
    r = r64 if prec == "fp64" else r32
    S = r.meshft(_cuda(V), _cuda(F), GRID, _cuda(fn), label="volume").cpu().numpy()
    assert rel(S, ref) < (1e-11 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("label", ["surface", "volume"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_meshft_adjoint_matches_oracle(label, prec, r64, r32):
    if label == "surface":
        V, F = _meshes()["sh_sphere"]
    else:
        V, F = synth.sh_deformed_sphere(2, 5.0, (8.0, 8.0, 9.0), lmax=3, coef_sigma=0.4, seed=5)
    fn = _freqs(2, M=200)
    xi = oracle.wavevectors(fn, GRID)
    rng = np.random.default_rng(9)
    G = (rng.normal(size=len(fn)) + 1j * rng.normal(size=len(fn))) / np.sqrt(len(fn))
    ref = oracle.mesh_ft_adjoint(V - np.asarray(GRID.origin), F, xi, G, label, c0=0.5 * GRID.L)
    r = r64 if prec == "fp64" else r32
    dV = r.meshft_adjoint(_cuda(V), _cuda(F), GRID, _cuda(fn), _cuda(G), label=label).cpu().numpy()
    assert rel(dV, ref) < (1e-10 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("n", [(16, 16, 16), (12, 10, 9), (8, 6, 15), (32, 24, 20), (1, 4, 8), (96, 8, 6),
                               (14, 11, 26), (7, 13, 22), (2048, 2, 4), (64, 128, 256), (512, 16, 32),
                               (8, 1024, 6), (6, 4, 1024), (1, 1, 64), (1, 512, 3), (33, 256, 128)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_matches_direct_definition(n, prec, r64, r32):
    r = r64 if prec == "fp64" else r32
    grid = synth.Grid(n=n, h=(1, 1, 1))
    X = synth.random_half_spectrum(n, seed=4)
    nvec, c = oracle.half_spectrum(n)
    # oracle image definition times the box volume: unnormalised inverse on H with weights c
    ref = oracle.spectrum_to_image(X.ravel(), nvec, c, grid) * np.prod(grid.L)
    Xd = torch.as_tensor(X).to(r.cplx).cuda()
    X0 = Xd.clone()
    img = r.c2r(grid, Xd).cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert rel(img, ref) < tol
    assert torch.equal(Xd, X0)  # the input spectrum is only read
    R = np.random.default_rng(5).normal(size=n)
    refG = np.fft.fftn(R)[nvec[:, 0] % n[0], nvec[:, 1] % n[1], nvec[:, 2] % n[2]]
    spec = r.r2c(grid, torch.as_tensor(R).cuda()).cpu().numpy().ravel()
    assert rel(spec, refG) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_c2r_into_the_buffer_that_holds_the_spectrum(prec, r64, r32):
    """dm_c2r with the image written over its own input spectrum (one buffer): the spectrum is then
    copied into the workspace before the passes instead of being read in place."""
    import ctypes

    from paper_2303_10440_b300.api import _grid

    r = r64 if prec == "fp64" else r32
    n = (32, 16, 64)
    grid = synth.Grid(n=n, h=(1, 1, 1))
    X = synth.random_half_spectrum(n, seed=8)
    nvec, c = oracle.half_spectrum(n)
    ref = oracle.spectrum_to_image(X.ravel(), nvec, c, grid) * np.prod(grid.L)
    Xd = torch.as_tensor(X).to(r.cplx).cuda().contiguous()
    g = _grid(grid)
    st = r.lib.dm_c2r(r.ctx, ctypes.byref(g), Xd.data_ptr(), Xd.data_ptr(), None)
    assert st == 0
    torch.cuda.synchronize()
    img = Xd.view(r.real).ravel()[: int(np.prod(n))].reshape(n).cpu().numpy()
    assert rel(img, ref) < (1e-12 if prec == "fp64" else 2e-6)


def test_fft_longest_axes_and_refused_lengths(r64, r32):
    """An FP32 axis of 4096 (the longest; the FP64 lines of that length do not fit in shared memory and are
    refused), and a length with the prime factor 17 (refused by both paths)."""
    from paper_2303_10440_b300 import DeltaMicError

    n = (2, 4096, 3)
    grid = synth.Grid(n=n, h=(1, 1, 1))
    X = synth.random_half_spectrum(n, seed=6)
    nvec, c = oracle.half_spectrum(n)
    ref = oracle.spectrum_to_image(X.ravel(), nvec, c, grid) * np.prod(grid.L)
    assert rel(r32.c2r(grid, torch.as_tensor(X).cuda()).cpu().numpy(), ref) < 2e-6
    with pytest.raises(DeltaMicError, match="UNSUPPORTED"):
        r64.c2r(grid, torch.as_tensor(X).cuda())
    bad = synth.Grid(n=(17, 4, 4), h=(1, 1, 1))
    for r in (r64, r32):
        with pytest.raises(DeltaMicError, match="UNSUPPORTED"):
            r.r2c(bad, torch.zeros(bad.n, dtype=r.real).cuda())


@pytest.mark.parametrize("tau", [1e-3, 1e-2, 0.3])
def test_band_is_bit_exact(tau, r64):
    grid = synth.Grid(n=(24, 20, 16), h=(0.5, 0.5, 1.0))
    psf = synth.Psf(sigma=(0.9, 1.2, 2.0), band_tau=tau)
    nvec, _ = oracle.half_spectrum(grid.n)
    mask = oracle.band_mask(oracle.otf(oracle.wavevectors(nvec, grid), psf), tau)
    idx = r64.band(grid, psf).numpy()
    assert np.array_equal(idx, np.nonzero(mask)[0].astype(np.int32))


@pytest.mark.parametrize("tau", [1e-3, 0.2])
def test_band_is_bit_exact_for_an_oblique_covariance(tau, r64):
    """A full, strongly anisotropic covariance (condition number ~100, cross terms that cancel): the
    band decided in FP32 away from the threshold and in FP64 near it is the oracle's, bit for bit."""
    from paper_2303_10440_b300 import PSF

    grid = synth.Grid(n=(64, 48, 40), h=(0.5, 0.5, 1.0))
    A = np.array([[1.0, 0.9, 0.3], [0.0, 0.3, 0.5], [0.0, 0.0, 0.4]])
    S = A @ A.T * 0.8
    cov = (S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2])
    psf = PSF(cov=cov, band_tau=tau)
    nvec, _ = oracle.half_spectrum(grid.n)
    mask = oracle.band_mask(oracle.otf(oracle.wavevectors(nvec, grid), psf), tau)
    idx = r64.band(grid, psf).numpy()
    assert 0 < mask.sum() < len(mask)
    assert np.array_equal(idx, np.nonzero(mask)[0].astype(np.int32))


def _case_small(mode="surface", tau=0.0, n=(16, 12, 10)):
    grid = synth.Grid(n=n, h=(1.0, 1.0, 1.5), origin=(0.5, -0.25, 1.0))
    psf = synth.Psf(sigma=(0.8, 1.0, 1.4), band_tau=tau)
    V, F = synth.sh_deformed_sphere(2, 4.0, grid.center, lmax=4, coef_sigma=0.4, seed=7)
    Vt = synth.scale_about(V, (1.1, 0.9, 1.0), grid.center)
    T = oracle.render(Vt, F, grid, psf, mode)["image"]
    T = synth.add_gaussian_noise(T, 0.05, seed=0)
    return grid, psf, V, F, T


@pytest.mark.parametrize("mode", ["surface", "volume"])
@pytest.mark.parametrize("tau", [0.0, 1e-2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_render_matches_oracle(mode, tau, prec, r64, r32):
    grid, psf, V, F, _ = _case_small(mode, tau)
    ref = oracle.render(V, F, grid, psf, mode)["image"]
    r = r64 if prec == "fp64" else r32
    img = r.render(_cuda(V), _cuda(F), grid, psf, label=mode).cpu().numpy()
    assert rel(img, ref) < (1e-10 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("mode", ["surface", "volume"])
@pytest.mark.parametrize("nz", [24, 32, 33])
def test_band_that_holds_all_of_the_half_spectrum(mode, nz, r32):
    """A band that holds every frequency of H (tau far below every h_hat of the grid) gives bitwise the image of
    tau = 0 (the same frequencies in the same order through the band list), which matches the oracle; and the
    forward on the explicit list of H (dm_meshft) matches the oracle's spectrum. Even and odd Nz."""
    grid = synth.Grid(n=(18, 20, nz), h=(1.0, 1.1, 1.2), origin=(0.3, -0.2, 0.1))
    V, F = synth.sh_deformed_sphere(2, 0.27 * float(min(grid.L)), grid.center, lmax=4, coef_sigma=0.5, seed=21)
    if mode == "volume":
        V, F = synth.sh_deformed_sphere(2, 0.27 * float(min(grid.L)), grid.center, lmax=3, coef_sigma=0.3, seed=22)
    psf0 = synth.Psf(sigma=(0.7, 0.8, 1.1), band_tau=0.0)
    psf1 = synth.Psf(sigma=(0.7, 0.8, 1.1), band_tau=1e-9)  # every h_hat of this grid is far above 1e-9
    a = r32.render(_cuda(V), _cuda(F), grid, psf0, label=mode)
    b = r32.render(_cuda(V), _cuda(F), grid, psf1, label=mode)
    assert torch.equal(a, b)
    ref = oracle.render(V, F, grid, psf0, mode)["image"]
    assert rel(a.cpu().numpy(), ref) < 1e-5
    nvec, _ = oracle.half_spectrum(grid.n)
    S_list = r32.meshft(_cuda(V), _cuda(F), grid, _cuda(nvec.astype(np.int32)), label=mode).cpu().numpy()
    S_ref = oracle.mesh_ft(V - np.asarray(grid.origin), F, oracle.wavevectors(nvec, grid), mode,
                           c0=0.5 * np.asarray(grid.L) if mode == "volume" else None)
    assert rel(S_list, S_ref) < 1e-5


@pytest.mark.parametrize("kind", ["mse", "l2", "weighted"])
@pytest.mark.parametrize("mode", ["surface", "volume"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_loss_and_grad_matches_oracle(kind, mode, prec, r64, r32):
    grid, psf, V, F, T = _case_small(mode)
    L0, dV0, dpsf0, _ = oracle.loss_and_grad(V, F, grid, psf, T, kind, mode)
    r = r64 if prec == "fp64" else r32
    L, dV, dpsf, img = r.loss_and_grad(_cuda(V), _cuda(F), grid, psf, _cuda(T), loss=kind, label=mode, want_image=True)
    tl, tg = (1e-10, 1e-9) if prec == "fp64" else (2e-4, 1e-3)
    assert abs(L - L0) <= tl * abs(L0)
    assert rel(dV.cpu().numpy(), dV0) < tg
    assert rel(dpsf.numpy(), dpsf0) < tg


@pytest.mark.parametrize("mesh", ["ico0_20", "ico1_80", "soup_130"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_meshes_over_many_chunks(mesh, prec, r64, r32):
    """Meshes of 20, 80 and 130 triangles on a 64^3 grid: one partial record tile, a part-padding
    warp, and a triangle block that is almost all padding; the adjoint runs ~500 frequency chunks
    per triangle block and sums them in the chunk reduction."""
    grid = synth.Grid(n=(64, 64, 64), h=(0.5, 0.5, 1.0))
    if mesh == "soup_130":
        V, F = synth.random_triangles(130, seed=5, extent=6.0, center=grid.center)
    else:
        V, F = synth.sphere_mesh(int(mesh[3]), 6.0, grid.center)
    psf = synth.Psf(sigma=(0.3, 0.3, 0.8), band_tau=1e-3)
    T = oracle.render(synth.scale_about(V, (1.05, 0.97, 1.0), grid.center), F, grid, psf)["image"]
    L0, dV0, dpsf0, r0 = oracle.loss_and_grad(V, F, grid, psf, T, "mse")
    r = r64 if prec == "fp64" else r32
    L, dV, dpsf, img = r.loss_and_grad(_cuda(V), _cuda(F), grid, psf, _cuda(T), "mse", want_image=True)
    ti, tl, tg = (1e-10, 1e-10, 1e-9) if prec == "fp64" else (1e-4, 2e-4, 1e-3)
    assert rel(img.cpu().numpy(), r0["image"]) < ti
    assert abs(L - L0) <= tl * abs(L0)
    assert rel(dV.cpu().numpy(), dV0) < tg
    assert rel(dpsf.numpy(), dpsf0) < tg


def test_case1_fp64_matches_oracle(r64):
    case = synth.config_c1()
    T = oracle.render(case.V_true, case.F, case.grid, case.psf)["image"]
    T = synth.add_gaussian_noise(T, 0.05, seed=0)
    L0, dV0, dpsf0, r0 = oracle.loss_and_grad(case.V_init, case.F, case.grid, case.psf, T, "mse")
    L, dV, dpsf, img = r64.loss_and_grad(_cuda(case.V_init), _cuda(case.F), case.grid, case.psf, _cuda(T), "mse",
                                         want_image=True)
    assert rel(img.cpu().numpy(), r0["image"]) < 1e-10
    assert abs(L - L0) < 1e-10 * L0
    assert rel(dV.cpu().numpy(), dV0) < 1e-9
    assert rel(dpsf.numpy(), dpsf0) < 1e-9


def test_render_adjoint_is_the_loss_gradient(r64):
    grid, psf, V, F, T = _case_small()
    L, dV, dpsf, img = r64.loss_and_grad(_cuda(V), _cuda(F), grid, psf, _cuda(T), "l2", want_image=True)
    dLdI = 2.0 * (img - _cuda(T))
    dV2, dpsf2 = r64.render_adjoint(_cuda(V), _cuda(F), grid, psf, dLdI)
    assert rel(dV2.cpu().numpy(), dV.cpu().numpy()) < 1e-12
    assert rel(dpsf2.numpy(), dpsf.numpy()) < 1e-12


def test_host_buffers_match_device_buffers(r32):
    grid, psf, V, F, T = _case_small()
    a = r32.loss_and_grad(_cuda(V), _cuda(F), grid, psf, _cuda(T), "mse")
    b = r32.loss_and_grad(torch.as_tensor(V), torch.as_tensor(F), grid, psf, torch.as_tensor(T), "mse")
    assert a[0] == b[0]
    assert torch.equal(a[1].cpu(), b[1])


def test_repeat_runs_are_bitwise_identical(r32):
    case = synth.config_c2()
    grid, psf = case.grid, case.psf
    T = torch.zeros(tuple(grid.n), dtype=torch.float32, device="cuda")
    Vd, Fd = _cuda(case.V_true), _cuda(case.F)
    a = r32.loss_and_grad(Vd, Fd, grid, psf, T, "mse")
    b = r32.loss_and_grad(Vd, Fd, grid, psf, T, "mse")
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_argument_errors_are_reported(r32):
    from paper_2303_10440_b300 import DeltaMicError

    grid, psf, V, F, T = _case_small()
    bad = F.copy()
    bad[3, 1] = V.shape[0] + 5
    with pytest.raises(DeltaMicError, match="DM_ERR_ARG"):
        r32.render(torch.as_tensor(V), torch.as_tensor(bad), grid, psf)
    with pytest.raises(DeltaMicError, match="DM_ERR_ARG"):
        r32.render(_cuda(V), _cuda(F), grid, synth.Psf(sigma=(1.0, -1.0, 1.0)))
    with pytest.raises(DeltaMicError, match="DM_ERR_UNSUPPORTED"):
        r32.render(_cuda(V), _cuda(F), synth.Grid(n=(17, 17, 17), h=(1, 1, 1)), psf)
    # an out-of-range index in device memory is caught by the kernels' bounds checks
    with pytest.raises(DeltaMicError, match="DM_ERR_ARG"):
        r32.loss_and_grad(_cuda(V), _cuda(bad), grid, psf, torch.as_tensor(T), "mse")
    # the context stays usable afterwards
    img = r32.render(_cuda(V), _cuda(F), grid, psf)
    assert torch.isfinite(img).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_degenerate_and_open_meshes_are_reported(prec, r64, r32):
    """Zero total area and non-positive enclosed volume are reported by the render calls themselves
    (DM_ERR_DEGENERATE, from the device normaliser); dm_check_mesh also finds volume-label meshes that
    are not closed and consistently oriented (DM_ERR_OPEN_MESH)."""
    from paper_2303_10440_b300 import DeltaMicError

    r = r64 if prec == "fp64" else r32
    grid, psf, V, F, T = _case_small()
    Td = _cuda(T)
    flat = np.repeat(V[:1], len(V), axis=0)  # every vertex at one point: zero area, zero volume
    with pytest.raises(DeltaMicError, match="DM_ERR_DEGENERATE"):
        r.loss_and_grad(_cuda(flat), _cuda(F), grid, psf, Td, "mse")
    with pytest.raises(DeltaMicError, match="DM_ERR_DEGENERATE"):  # inward: negative volume
        r.loss_and_grad(_cuda(V), _cuda(F[:, ::-1].copy()), grid, psf, Td, "mse", label="volume")
    with pytest.raises(DeltaMicError, match="DM_ERR_DEGENERATE"):
        r.loss_and_grad(_cuda(V), _cuda(F), grid, psf, Td, "mse",
                        weights=torch.zeros(len(F), dtype=torch.float32).cuda())
    # an asynchronous call reports it at the next synchronisation
    r.render(_cuda(flat), _cuda(F), grid, psf)
    with pytest.raises(DeltaMicError, match="DM_ERR_DEGENERATE"):
        r.sync()
    img = r.render(_cuda(V), _cuda(F), grid, psf)  # the context stays usable
    r.sync()
    assert torch.isfinite(img).all()
    # the debug check, on host and on device arrays
    for dev in (False, True):
        cv = (lambda x: _cuda(x)) if dev else (lambda x: x)
        r.check_mesh(cv(V), cv(F), label="volume")
        r.check_mesh(cv(V), cv(F[:-1].copy()), label="surface")  # an open surface is fine
        with pytest.raises(DeltaMicError, match="DM_ERR_OPEN_MESH"):
            r.check_mesh(cv(V), cv(F[:-1].copy()), label="volume")  # one face missing
        flipped = F.copy()
        flipped[0] = flipped[0, ::-1]
        with pytest.raises(DeltaMicError, match="DM_ERR_OPEN_MESH"):
            r.check_mesh(cv(V), cv(flipped), label="volume")  # one face turned inward
        with pytest.raises(DeltaMicError, match="DM_ERR_DEGENERATE"):
            r.check_mesh(cv(V), cv(F[:, ::-1].copy()), label="volume")
        bad = F.copy()
        bad[0, 0] = -1
        with pytest.raises(DeltaMicError, match="DM_ERR_ARG"):
            r.check_mesh(cv(V), cv(bad))


@pytest.mark.parametrize("wkind", ["interface", "random"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weighted_density_matches_oracle(wkind, prec, r64, r32):
    """Per-triangle fluorophore density (Section 3.3): image, loss and gradients vs the oracle."""
    grid, psf, V, F, T = _case_small()
    if wkind == "interface":
        cen = V[F].mean(axis=1)
        w = np.where(cen[:, 0] > grid.center[0], 2.0, 1.0).astype(np.float32)
    else:
        w = np.random.default_rng(21).uniform(0.25, 3.0, len(F)).astype(np.float32)
    w64 = w.astype(np.float64)
    r = r64 if prec == "fp64" else r32
    ref = oracle.render(V, F, grid, psf, weights=w64)["image"]
    img = r.render(_cuda(V), _cuda(F), grid, psf, weights=_cuda(w)).cpu().numpy()
    assert rel(img, ref) < (1e-10 if prec == "fp64" else 1e-4)
    L0, dV0, dpsf0, _ = oracle.loss_and_grad(V, F, grid, psf, T, "mse", weights=w64)
    L, dV, dpsf, _ = r.loss_and_grad(_cuda(V), _cuda(F), grid, psf, _cuda(T), "mse", weights=_cuda(w))
    tl, tg = (1e-10, 1e-9) if prec == "fp64" else (2e-4, 1e-3)
    assert abs(L - L0) <= tl * abs(L0)
    assert rel(dV.cpu().numpy(), dV0) < tg
    assert rel(dpsf.numpy(), dpsf0) < tg


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weighted_meshft_and_adjoint_match_oracle(prec, r64, r32):
    V, F = _meshes()["sh_sphere"]
    w = np.random.default_rng(22).uniform(0.5, 2.0, len(F)).astype(np.float32)
    w64 = w.astype(np.float64)
    fn = _freqs(5)
    xi = oracle.wavevectors(fn, GRID)
    Vo = V - np.asarray(GRID.origin)
    r = r64 if prec == "fp64" else r32
    S0 = oracle.mesh_ft(Vo, F, xi, weights=w64)
    S = r.meshft(_cuda(V), _cuda(F), GRID, _cuda(fn), weights=_cuda(w)).cpu().numpy()
    assert rel(S, S0) < (1e-11 if prec == "fp64" else 2e-6)
    rng = np.random.default_rng(6)
    G = (rng.normal(size=len(fn)) + 1j * rng.normal(size=len(fn))) / np.sqrt(len(fn))
    dV0 = oracle.mesh_ft_adjoint(Vo, F, xi, G, weights=w64)
    dV = r.meshft_adjoint(_cuda(V), _cuda(F), GRID, _cuda(fn), _cuda(G), weights=_cuda(w)).cpu().numpy()
    assert rel(dV, dV0) < (1e-10 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tissue_foam_matches_oracle(prec, r64, r32):
    """A multi-cell tissue in one non-manifold mesh (2 x 2 x 1 jittered box cells, walls at density 2)."""
    grid = synth.Grid(n=(24, 24, 16), h=(0.75, 0.75, 1.0), origin=(-0.5, 0.25, 0.0))
    V, F, rho = synth.box_foam((2, 2, 1), (7.0, 6.5, 8.0), subdiv=4, origin=(2.0, 2.0, 3.5), jitter=0.15, seed=3)
    w = rho.astype(np.float32)
    psf = synth.Psf(sigma=(0.7, 0.7, 1.2), band_tau=1e-3)
    Vt = V + 0.2 * np.sin(V[:, [1, 2, 0]] / 3.0)
    T = synth.add_gaussian_noise(oracle.render(Vt, F, grid, psf, weights=rho)["image"], 0.03, seed=8)
    r = r64 if prec == "fp64" else r32
    ref = oracle.render(V, F, grid, psf, weights=rho)["image"]
    img = r.render(_cuda(V), _cuda(F), grid, psf, weights=_cuda(w)).cpu().numpy()
    assert rel(img, ref) < (1e-10 if prec == "fp64" else 1e-4)
    L0, dV0, dpsf0, _ = oracle.loss_and_grad(V, F, grid, psf, T, "weighted", weights=rho)
    L, dV, dpsf, _ = r.loss_and_grad(_cuda(V), _cuda(F), grid, psf, _cuda(T), "weighted", weights=_cuda(w))
    tl, tg = (1e-10, 1e-9) if prec == "fp64" else (2e-4, 1e-3)
    assert abs(L - L0) <= tl * abs(L0)
    assert rel(dV.cpu().numpy(), dV0) < tg
    assert rel(dpsf.numpy(), dpsf0) < tg


@pytest.mark.parametrize("scale", [0.02, 0.15, 0.6])
@pytest.mark.parametrize("label", ["surface", "volume"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_in_and_around_the_series_region(scale, label, prec, r64, r32):
    """Small triangles: at scale 0.02 every term has its three phases within 0.5 (series only), at 0.15
    and 0.6 the terms straddle the switch between the series and the closed form with Taylor gaps."""
    V, F = synth.sh_deformed_sphere(1, 1.0, (0.0, 0.0, 0.0), lmax=2, coef_sigma=0.1, seed=4)
    V = V * (scale * 8.0) + np.array([8.0, 7.5, 9.0])
    fn = _freqs(3, M=256)
    xi = oracle.wavevectors(fn, GRID)
    rng = np.random.default_rng(10)
    G = (rng.normal(size=len(fn)) + 1j * rng.normal(size=len(fn))) / np.sqrt(len(fn))
    Vo = V - np.asarray(GRID.origin)
    S0 = oracle.mesh_ft(Vo, F, xi, label, c0=0.5 * GRID.L)
    dV0 = oracle.mesh_ft_adjoint(Vo, F, xi, G, label, c0=0.5 * GRID.L)
    r = r64 if prec == "fp64" else r32
    S = r.meshft(_cuda(V), _cuda(F), GRID, _cuda(fn), label=label).cpu().numpy()
    dV = r.meshft_adjoint(_cuda(V), _cuda(F), GRID, _cuda(fn), _cuda(G), label=label).cpu().numpy()
    assert rel(S, S0) < (1e-11 if prec == "fp64" else 2e-6)
    assert rel(dV, dV0) < (1e-10 if prec == "fp64" else 1e-4)
