"""Staggered fit on the GPU (Section 5.1-5.2) vs the oracle: the smoothing solve of the
large-steps update, the uniform-Adam step, and whole staggered fits.

Tolerances: the FP64 path's conjugate gradients stop at a relative residual of 1e-12, so
solutions agree to ~kappa * 1e-12 (kappa <= 1 + lambda * 2 * max degree ~ 600 for the meshes
here); the FP32 path stops at 1e-6, hence 1e-3.
"""

import numpy as np
import pytest
import torch

import oracle
import oracle.optim as opt
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


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


def _meshes():
    out = {}
    out["sh_l3"] = synth.sh_deformed_sphere(3, 8.0, (0, 0, 0), lmax=4, coef_sigma=0.5, seed=1)
    out["sh_l5"] = synth.sh_deformed_sphere(5, 30.0, (0, 0, 0), lmax=6, coef_sigma=1.0, seed=2)
    Vt, Ft = synth.random_triangles(60, seed=3, extent=6.0, center=(0, 0, 0))
    out["soup"] = (Vt, Ft)
    # two cells sharing a wall: non-manifold edges along the wall's rim
    Va, Fa = synth.box_mesh((0, 0, 0), (2, 2, 2))
    Vb, Fb = synth.box_mesh((2, 0, 0), (4, 2, 2))
    V = np.concatenate([Va, Vb])
    F = np.concatenate([Fa, Fb + len(Va)])
    key = {tuple(np.round(v, 9)): i for i, v in enumerate(V)}  # merge the coincident corners
    remap = np.array([key[tuple(np.round(v, 9))] for v in V])
    out["two_boxes"] = (V, remap[F].astype(np.int32))
    return out


@pytest.mark.parametrize("name", ["sh_l3", "sh_l5", "soup", "two_boxes"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smooth_solve_matches_oracle(name, prec, r64, r32):
    V, F = _meshes()[name]
    n_v = len(V)
    B = np.random.default_rng(7).normal(size=(n_v, 3))
    ref = opt.smooth_solve(F, n_v, 50.0, B)
    r = r64 if prec == "fp64" else r32
    X, (total, most, unconv) = r.smooth_solve(torch.as_tensor(F).cuda(), n_v, torch.as_tensor(B).cuda(), 50.0)
    assert unconv == 0 and most > 0 and total >= most
    assert rel(X.cpu().numpy(), ref) < (1e-9 if prec == "fp64" else 1e-3)
    # started at the solution, the solve stops at once (FP64) or after a few corrections of the
    # rounding of the start to FP32
    X2, (total2, _, _) = r.smooth_solve(torch.as_tensor(F).cuda(), n_v, torch.as_tensor(B).cuda(), 50.0,
                                        X0=torch.as_tensor(ref).cuda(), tol=1e-6)
    assert total2 <= 3 if prec == "fp64" else total2 < total


def test_smooth_solve_of_zero_and_of_lambda_zero(r64):
    V, F = _meshes()["sh_l3"]
    n_v = len(V)
    X, it = r64.smooth_solve(torch.as_tensor(F).cuda(), n_v, torch.zeros(n_v, 3, dtype=torch.float64).cuda(),
                             X0=torch.ones(n_v, 3, dtype=torch.float64).cuda())
    assert torch.count_nonzero(X) == 0 and it[0] == 0
    B = torch.as_tensor(np.random.default_rng(1).normal(size=(n_v, 3))).cuda()
    X, _ = r64.smooth_solve(torch.as_tensor(F).cuda(), n_v, B, lam=0.0)
    assert torch.allclose(X, B, rtol=1e-12, atol=0)


def test_adam_uniform_matches_oracle(r64):
    rng = np.random.default_rng(3)
    n = 3 * 700
    m0, v0 = np.zeros(n), np.zeros(n)
    m, v = torch.zeros(n, dtype=torch.float64).cuda(), torch.zeros(n, dtype=torch.float64).cuda()
    for t in range(1, 5):
        g = rng.normal(size=n) * 1e-9
        d0, m0, v0 = opt.adam_uniform(g, m0, v0, t, 0.3, 0.9, 0.999, 1e-20)
        d = r64.adam_uniform(torch.as_tensor(g).cuda(), m, v, t, 0.3, 0.9, 0.999, 1e-20)
        assert rel(d.cpu().numpy(), d0) < 1e-14
        assert rel(m.cpu().numpy(), m0) < 1e-15 and rel(v.cpu().numpy(), v0) < 1e-15


def test_adam_matches_oracle(r64, r32):
    """dm_adam (the fit loop's vertex and PSF optimiser) against the oracle's Adam, step by step."""
    rng = np.random.default_rng(8)
    n = 3 * 900
    for r, tol in ((r64, 1e-14), (r32, 1e-14)):
        p0, m0, v0 = rng.normal(size=n), np.zeros(n), np.zeros(n)
        p = torch.as_tensor(p0.copy()).cuda()
        m, v = torch.zeros(n, dtype=torch.float64).cuda(), torch.zeros(n, dtype=torch.float64).cuda()
        for t in range(1, 6):
            g = rng.normal(size=n) * 1e-9
            d0, m0, v0 = opt.adam(g, m0, v0, t, 0.3, 0.9, 0.999, 1e-20)
            p0 = p0 - d0
            r.adam(p, torch.as_tensor(g).cuda(), m, v, t, 0.3, 0.9, 0.999, 1e-20)
            assert rel(p.cpu().numpy(), p0) < tol
            assert rel(m.cpu().numpy(), m0) < 1e-15 and rel(v.cpu().numpy(), v0) < 1e-15


def _tiny_case():
    grid = synth.Grid(n=(12, 12, 10), h=(1.0, 1.0, 1.5), origin=(0.2, -0.1, 0.3))
    V0, F = synth.sphere_mesh(1, 3.2, grid.center)
    Vt = synth.scale_about(V0, (1.08, 0.95, 1.0), grid.center)
    true_cov = (1.0, 1.1, 2.0, 0.25, 0.1, -0.15)
    T = oracle.render(Vt, F, grid, opt._psf_full(true_cov, 0.0))["image"]
    T = synth.add_gaussian_noise(T, 0.02, seed=4)
    return grid, V0, F, T


@pytest.mark.parametrize("optimizer,lr_vertex", [("large_steps", 0.5), ("adam", 0.03)])
def test_fit_staggered_matches_oracle(optimizer, lr_vertex, r64):
    """FP64 path: the whole staggered fit against the oracle's. The per-step gradients agree to ~1e-13; the
    smoothing filter (1 + lambda L)^-2 can amplify a relative gradient error by up to its condition bound
    kappa = 1 + 2 lambda (max degree) in the displacement, and Adam divides each coordinate by its own
    moment, so a coordinate whose gradient is near zero carries a larger relative error: 1e-8 on the
    displacement and 1e-9 on the covariance and losses leave room for both over 10 steps."""
    grid, V0, F, T = _tiny_case()
    psf0 = synth.Psf(sigma=(1.1, 1.1, 1.3), band_tau=1e-3)
    kw = dict(rounds=2, shape_steps=3, psf_steps=2, lr_vertex=lr_vertex, lr_psf=0.02, optimizer=optimizer)
    V1, cov1, hs1, hp1 = opt.fit_staggered(V0, F, grid, psf0, T, **kw)
    V, psf, hs, hp, cg = r64.fit_staggered(torch.as_tensor(V0).cuda(), torch.as_tensor(F).cuda(), grid, psf0,
                                           torch.as_tensor(T).cuda(), **kw)
    assert rel(V.cpu().numpy() - V0, V1 - V0) < 1e-8
    assert rel(psf.cov, cov1) < 1e-9
    assert rel(hs.numpy(), hs1) < 1e-9 and rel(hp.numpy(), hp1) < 1e-9
    if optimizer == "large_steps":
        assert cg["iterations"] > 0 and cg["unconverged"] == 0
    else:
        assert cg["iterations"] == 0


@pytest.mark.parametrize("optimizer,lr_vertex", [("large_steps", 0.5), ("adam", 0.03)])
def test_fit_staggered_fp32_steps_match_oracle(optimizer, lr_vertex, r32):
    """FP32 path: the parity unit is the step at identical inputs. FP32 and FP64 trajectories separate (Adam
    divides each coordinate by its own moment, so gradient errors far inside the tolerance flip the steps of
    coordinates whose gradient is near zero, and the fit amplifies the difference), so each state the oracle's
    fit passes through is fed to the FP32 path, whose loss and gradient (dL/dV on the narrow band for shape
    steps, dL/dcov on the whole half spectrum for PSF steps) must match the oracle's there within the path's
    tolerances: 1e-4 on the loss (the image tolerance), 1e-3 on the gradients. The whole FP32 fit is run too,
    and must match the oracle's first loss within 1e-4 and lower its PSF loss."""
    from paper_2303_10440_b300 import PSF

    grid, V0, F, T = _tiny_case()
    psf0 = synth.Psf(sigma=(1.1, 1.1, 1.3), band_tau=1e-3)
    kw = dict(rounds=2, shape_steps=3, psf_steps=2, lr_vertex=lr_vertex, lr_psf=0.02, optimizer=optimizer)
    trace = []
    opt.fit_staggered(V0, F, grid, psf0, T, trace=trace, **kw)
    assert len(trace) == 10
    Fd, Td = torch.as_tensor(F).cuda(), torch.as_tensor(T).cuda().float()
    errs = []
    for st in trace:
        shape = st["kind"] == "shape"
        psf = PSF(cov=tuple(st["cov"]), band_tau=psf0.band_tau if shape else 0.0)
        L, dV, dcov, _ = r32.loss_and_grad(torch.as_tensor(st["V"]).cuda(), Fd, grid, psf, Td,
                                           "weighted" if shape else "l2")
        g = dV.cpu().numpy() if shape else dcov.numpy()
        eL, eg = abs(L - st["L"]) / st["L"], rel(g, st["grad"])
        errs.append((st["kind"], eL, eg))
        assert eL < 1e-4 and eg < 1e-3, (st["kind"], eL, eg)
    print(f"\n[FP32 staggered steps vs oracle, {optimizer}] worst loss {max(e[1] for e in errs):.2e}, "
          f"worst gradient {max(e[2] for e in errs):.2e}")
    V, psf, hs, hp, cg = r32.fit_staggered(torch.as_tensor(V0).cuda(), Fd, grid, psf0, Td, **kw)
    assert abs(float(hs[0]) - trace[0]["L"]) < 1e-4 * trace[0]["L"]
    assert float(hp[-1]) < float(hp[0])


@pytest.mark.parametrize("variant", ["volume", "tissue_foam"])
def test_fit_staggered_variants_match_oracle(variant, r64):
    """FP64 staggered fits of a volume-labelled cell and of a weighted multi-cell foam."""
    if variant == "volume":
        grid, V0, F, T = _tiny_case()
        kw = dict(mode="volume")
        gkw = dict(label="volume")
        T = oracle.render(synth.scale_about(V0, (1.06, 0.96, 1.0), grid.center), F, grid,
                          opt._psf_full((1.0, 1.1, 2.0, 0.25, 0.1, -0.15), 0.0), "volume")["image"]
    else:
        grid = synth.Grid(n=(16, 16, 12), h=(1.0, 1.0, 1.25))
        V0, F, rho = synth.box_foam((2, 1, 1), (5.0, 6.0, 6.0), subdiv=2, origin=(3.0, 5.0, 4.5), jitter=0.1, seed=2)
        Vt = V0 + 0.25 * np.cos(V0[:, [2, 0, 1]] / 2.5)
        T = oracle.render(Vt, F, grid, opt._psf_full((1.0, 1.1, 1.8, 0.2, 0.0, 0.1), 0.0), weights=rho)["image"]
        kw = dict(weights=rho)  # densities 1 and 2: exact in the FP32 weights the library takes
        gkw = dict(weights=torch.as_tensor(rho.astype(np.float32)).cuda())
    psf0 = synth.Psf(sigma=(1.1, 1.1, 1.3), band_tau=1e-3)
    common = dict(rounds=2, shape_steps=2, psf_steps=2, lr_vertex=0.3, lr_psf=0.02)
    V1, cov1, hs1, hp1 = opt.fit_staggered(V0, F, grid, psf0, T, **common, **kw)
    V, psf, hs, hp, cg = r64.fit_staggered(torch.as_tensor(V0).cuda(), torch.as_tensor(F).cuda(), grid, psf0,
                                           torch.as_tensor(T).cuda(), **common, **gkw)
    # the smoothing filter (1 + lambda L)^-2 keeps the low modes of dL/dv and drops the rest, so a
    # relative gradient error e (1e-9 on the FP64 path) can grow up to kappa e in the displacement,
    # kappa = 1 + 2 lambda (max degree) the smoothing matrix's condition bound
    kappa = 1.0 + 2 * 50.0 * opt.laplacian(F, len(V0)).diagonal().max()
    assert rel(V.cpu().numpy() - V0, V1 - V0) < 1e-9 * kappa
    assert rel(psf.cov, cov1) < 1e-9
    assert rel(hs.numpy(), hs1) < 1e-9 and rel(hp.numpy(), hp1) < 1e-9
    assert cg["unconverged"] == 0


def test_fit_staggered_recovers_shape_and_covariance(r32):
    """FP32 path, 64^3: an anisotropic cell under an oblique PSF, started from a sphere and a round PSF."""
    grid = synth.Grid(n=(64, 64, 64), h=(0.5, 0.5, 1.0))
    V0, F = synth.sphere_mesh(3, 8.0, grid.center)
    Vt = synth.scale_about(V0, (1.06, 0.96, 1.0), grid.center)
    true_cov = (0.16, 0.2, 0.5, 0.04, 0.02, -0.03)
    Fd = torch.as_tensor(F).cuda()
    from paper_2303_10440_b300 import PSF

    T = r32.render(torch.as_tensor(Vt).cuda(), Fd, grid, PSF(cov=true_cov))
    psf0 = PSF(sigma=(0.45, 0.45, 0.8), band_tau=1e-3)
    V, psf, hs, hp, cg = r32.fit_staggered(torch.as_tensor(V0).cuda(), Fd, grid, psf0, T, rounds=8, shape_steps=10,
                                           psf_steps=5, lr_vertex=2.0, lr_psf=0.01)
    err0 = np.abs(np.array([0.45**2, 0.45**2, 0.64, 0, 0, 0]) - true_cov).sum()
    err1 = np.abs(np.array(psf.cov) - true_cov).sum()
    d0 = np.abs(np.linalg.norm(V0 - grid.center, axis=1) - np.linalg.norm(Vt - grid.center, axis=1)).mean()
    d1 = np.abs(np.linalg.norm(V.cpu().numpy() - grid.center, axis=1) - np.linalg.norm(Vt - grid.center, axis=1)).mean()
    print(f"\n[staggered 8x(10+5)] shape loss {hs[0]:.3e} -> {hs[-1]:.3e}; psf loss {hp[0]:.3e} -> {hp[-1]:.3e}; "
          f"cov err {err0:.3f} -> {err1:.3f}; radial err {d0:.3f} -> {d1:.3f}; cg {cg}")
    assert hp[-1] < 0.5 * hp[0]
    assert err1 < 0.5 * err0
    assert d1 < 0.7 * d0
