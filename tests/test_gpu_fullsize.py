"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

* 128^3 single cell (5120 triangles, band = 1,064,960 frequencies): the FP32 path against the
  FP64 GPU path (itself held to 1e-10 of the oracle at small sizes) over the whole image, loss
  and gradients; and both paths against the oracle on sampled frequencies, which the oracle can
  evaluate one by one (spectrum and mesh adjoint at the full mesh size).
* 256x256x128 cell (20480 triangles, the whole half spectrum of 4,259,840 frequencies): the FP32
  path against one FP64 autograd pass over the whole image, loss and gradients; sampled spectrum
  and mesh adjoint against the oracle; the autograd gradient against central differences (step
  1e-6, FP64) on 64 directions; properties that hold at any size (unit total intensity, repeat
  determinism).
* The largest serving request (81,920 triangles on 256^3): sampled spectrum and mesh adjoint
  against the oracle, unit total intensity and repeat determinism of a fit step.

Errors are printed (run with -s to see them).
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def renderers():
    from paper_2303_10440_b300 import Renderer

    r32, r64 = Renderer("fp32"), Renderer("fp64")
    yield r32, r64
    r32.close()
    r64.close()


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def test_c2_fp32_matches_fp64_over_the_whole_image(renderers):
    r32, r64 = renderers
    case = synth.config_c2()
    Fd = _dev(case.F)
    T64 = r64.render(_dev(case.V_true), Fd, case.grid, case.psf)
    L64, dV64, dp64, I64 = r64.loss_and_grad(_dev(case.V_init), Fd, case.grid, case.psf, T64, "mse", want_image=True)
    L32, dV32, dp32, I32 = r32.loss_and_grad(_dev(case.V_init), Fd, case.grid, case.psf, T64.float(), "mse",
                                             want_image=True)
    e_img = rel(I32.double().cpu(), I64.cpu())
    e_L = abs(L32 - L64) / L64
    e_dV = rel(dV32.cpu(), dV64.cpu())
    e_dp = rel(dp32, dp64)
    print(f"\n[c2 128^3] FP32 vs FP64: image {e_img:.2e}  loss {e_L:.2e}  dV {e_dV:.2e}  dsigma {e_dp:.2e}")
    assert e_img < 1e-4 and e_L < 2e-4 and e_dV < 1e-3 and e_dp < 1e-3
    # unit total intensity (Eq. 3): the band is the whole half spectrum here
    assert abs(float(I32.double().sum()) * np.prod(case.grid.h) - 1.0) < 1e-5
    assert abs(float(I64.sum()) * np.prod(case.grid.h) - 1.0) < 1e-12


def _sample_band(case, n, seed):
    nvec, _ = oracle.half_spectrum(case.grid.n)
    band = oracle.band_mask(oracle.otf(oracle.wavevectors(nvec, case.grid), case.psf), case.psf.band_tau)
    idx = np.nonzero(band)[0]
    rng = np.random.default_rng(seed)
    sel = np.concatenate([[idx[0]], rng.choice(idx, size=n - 1, replace=False)])
    return nvec[sel].astype(np.int32)


@pytest.mark.parametrize("which", ["c2", "c3"])
def test_full_mesh_spectrum_on_sampled_frequencies(which, renderers):
    r32, r64 = renderers
    case = synth.config_c2() if which == "c2" else synth.config_c3()
    fn = _sample_band(case, 512, seed=5)
    ref = oracle.mesh_ft(case.V_true - np.asarray(case.grid.origin), case.F, oracle.wavevectors(fn, case.grid))
    S32 = r32.meshft(_dev(case.V_true), _dev(case.F), case.grid, _dev(fn)).cpu().numpy()
    S64 = r64.meshft(_dev(case.V_true), _dev(case.F), case.grid, _dev(fn)).cpu().numpy()
    e32, e64 = rel(S32, ref), rel(S64, ref)
    print(f"\n[{which} sampled spectrum] FP32 {e32:.2e}  FP64 {e64:.2e}  (n_t = {case.F.shape[0]})")
    assert e64 < 1e-11 and e32 < 1e-5


@pytest.mark.parametrize("which", ["c2", "c3"])
def test_mesh_adjoint_on_sampled_frequencies(which, renderers):
    r32, r64 = renderers
    case = synth.config_c2() if which == "c2" else synth.config_c3()
    fn = _sample_band(case, 256, seed=6)
    rng = np.random.default_rng(7)
    G = (rng.normal(size=len(fn)) + 1j * rng.normal(size=len(fn))) / len(fn)
    ref = oracle.mesh_ft_adjoint(case.V_init - np.asarray(case.grid.origin), case.F,
                                 oracle.wavevectors(fn, case.grid), G)
    d32 = r32.meshft_adjoint(_dev(case.V_init), _dev(case.F), case.grid, _dev(fn), _dev(G)).cpu().numpy()
    d64 = r64.meshft_adjoint(_dev(case.V_init), _dev(case.F), case.grid, _dev(fn), _dev(G)).cpu().numpy()
    e32, e64 = rel(d32, ref), rel(d64, ref)
    print(f"\n[{which} sampled adjoint] FP32 {e32:.2e}  FP64 {e64:.2e}  (n_t = {case.F.shape[0]})")
    assert e64 < 1e-10 and e32 < 1e-4


@pytest.fixture(scope="module")
def c3_fp64(renderers):
    """One FP64 autograd pass (forward render, backward through the recomputing adjoint) of the MSE loss at
    the 256x256x128 cell's start: V = the undeformed level-5 sphere, sigma = (0.3, 0.3, 0.9) um, target = the
    deformed cell rendered with sigma = (0.25, 0.25, 0.7) um."""
    from paper_2303_10440_b300.autograd import render

    r32, r64 = renderers
    case = synth.config_c3()
    Fd = _dev(case.F)
    T = r32.render(_dev(case.V_true), Fd, case.grid, case.psf).double()
    V = _dev(case.V_init).requires_grad_(True)
    sig = torch.tensor(case.psf_init.sigma, dtype=torch.float64, requires_grad=True)
    img = render(V, sig, Fd, r64, case.grid)
    loss = ((img - T) ** 2).mean()
    loss.backward()
    return dict(case=case, Fd=Fd, T=T, img=img.detach(), L=float(loss.detach()), gV=V.grad.detach().clone(),
                gs=sig.grad.detach().clone())


def test_c3_fp32_matches_fp64_over_the_whole_image(renderers, c3_fp64):
    r32, _ = renderers
    c = c3_fp64
    case = c["case"]
    L32, dV32, dp32, I32 = r32.loss_and_grad(_dev(case.V_init), c["Fd"], case.grid, case.psf_init, c["T"].float(),
                                             "mse", want_image=True)
    e_img = rel(I32.double().cpu(), c["img"].cpu())
    e_L = abs(L32 - c["L"]) / c["L"]
    e_dV = rel(dV32.cpu(), c["gV"].cpu())
    e_dp = rel(dp32, c["gs"].cpu())
    print(f"\n[c3 256x256x128] FP32 vs FP64: image {e_img:.2e}  loss {e_L:.2e}  dV {e_dV:.2e}  dsigma {e_dp:.2e}")
    assert e_img < 1e-4 and e_L < 2e-4 and e_dV < 1e-3 and e_dp < 1e-3
    assert abs(float(c["img"].sum()) * np.prod(case.grid.h) - 1.0) < 1e-12


def _half_spectrum_n(n):
    """Integer frequencies of the half spectrum in its storage order [Nx][Ny][Nz/2+1] (fftfreq on x, y)."""
    ax = [np.fft.fftfreq(n[0], 1.0 / n[0]), np.fft.fftfreq(n[1], 1.0 / n[1]), np.arange(n[2] // 2 + 1)]
    g = np.meshgrid(*ax, indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1).astype(np.int32)


def _area(V, F):
    e1, e2 = V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum()


@pytest.mark.slow
def test_c3_autograd_matches_central_differences(renderers, c3_fp64):
    """Central differences (step 1e-6, FP64) of the MSE loss along 64 directions at full size.

    The mesh transform is a sum over triangles (Eq. 5), so moving one vertex changes only the terms of the
    triangles around it: S(V') = S(V) - S_star(V) + S_star(V') exactly (up to rounding), the area likewise.
    Directions 2..63 move one random vertex (and, in part, sigma) and are evaluated through that split:
    the FP64 spectrum of the whole mesh once, then the FP64 transforms of the vertex's few triangles,
    the transfer function, the FP64 inverse DFT and the loss. When only a vertex moves, L(+) - L(-) is
    ~1/n_v of a dense direction's, so I(+) - I(-) is formed from the star's own differences (subtracting
    two FP64 images of the whole mesh would leave ~1e-4 of it as rounding). Directions 0 and 1 move every
    vertex (the second also sigma) and run through whole FP64 renders. The split is first checked against
    the autograd forward's image."""
    from paper_2303_10440_b300 import PSF

    _, r64 = renderers
    c = c3_fp64
    case, Fd, T = c["case"], c["Fd"], c["T"]
    grid, F, V0 = case.grid, case.F, case.V_init
    sig0 = np.asarray(case.psf_init.sigma, dtype=np.float64)
    n = grid.n
    L = np.asarray(grid.L)
    fn = _dev(_half_spectrum_n(n))
    xi2 = ((2 * np.pi * fn.double() / _dev(L)) ** 2)  # [M, 3]
    S_full = r64.meshft(_dev(V0), Fd, grid, fn)
    A_full = float(_area(V0, F))

    def image(S, A, sig):
        h_hat = torch.exp(-0.5 * (xi2 * _dev(sig ** 2)).sum(1))
        X = (S / A * h_hat / float(np.prod(L))).reshape(n[0], n[1], n[2] // 2 + 1)
        return r64.c2r(grid, X)

    def dL(Ip, Im):  # (L(+) - L(-)) without subtracting two large sums
        return float(((Ip - Im) * (Ip + Im - 2 * T)).mean())

    I0 = image(S_full, A_full, sig0)
    e_base = rel(I0.cpu(), c["img"].cpu())
    assert e_base < 1e-12, e_base

    gV, gs = c["gV"].cpu().numpy(), c["gs"].cpu().numpy()
    rng = np.random.default_rng(33)
    h = 1e-6
    errs = []
    for k in range(64):
        ds = rng.normal(size=3) * 0.1 if k % 3 != 2 else np.zeros(3)
        if k < 2:
            d = rng.normal(size=V0.shape)
            if k == 0:
                ds = np.zeros(3)
            I = []
            for sgn in (1.0, -1.0):
                psf = PSF(sigma=tuple(sig0 + sgn * h * ds))
                I.append(r64.render(_dev(V0 + sgn * h * d), Fd, grid, psf))
            an = float((gV * d).sum() + (gs * ds).sum())
            scale = np.linalg.norm(gV) * np.linalg.norm(d) / np.sqrt(d.size) + np.linalg.norm(gs) * np.linalg.norm(ds)
        else:
            v = int(rng.integers(len(V0)))
            dv = rng.normal(size=3) if k not in (3, 4) else np.zeros(3)  # directions 3 and 4: sigma only
            star = F[(F == v).any(axis=1)]
            Fs = _dev(star)
            S_rest = S_full - r64.meshft(_dev(V0), Fs, grid, fn)
            A_rest = A_full - float(_area(V0, star))
            Vs = [V0.copy(), V0.copy()]
            Vs[0][v] += h * dv
            Vs[1][v] -= h * dv
            Ss = [r64.meshft(_dev(x), Fs, grid, fn) for x in Vs]  # the star's spectra at V(+), V(-)
            As = [float(_area(x, star)) for x in Vs]
            I = [image(S_rest + Ss[0], A_rest + As[0], sig0 + h * ds), image(S_rest + Ss[1], A_rest + As[1], sig0 - h * ds)]
            if not ds.any():
                # one vertex moves: I(+) - I(-) from the star's own differences, without subtracting two images
                # of the whole mesh: (S_rest + S+)/A+ - (S_rest + S-)/A- = [(S+ - S-) A- + (S_rest + S-)(A_s- - A_s+)]
                # / (A+ A-), A+- = A_rest + A_s+-, then the same transfer function and inverse DFT (linear)
                Ap, Am = A_rest + As[0], A_rest + As[1]
                dX = ((Ss[0] - Ss[1]) * Am + (S_rest + Ss[1]) * (As[1] - As[0])) / (Ap * Am)
                dI = image(dX, 1.0, sig0)
                I = [I[0] + I[1] + dI, I[0] + I[1] - dI]  # (dL below uses only I(+) - I(-) and I(+) + I(-))
                I = [0.5 * x for x in I]
            an = float(gV[v] @ dv + gs @ ds)
            scale = np.linalg.norm(gV[v]) * np.linalg.norm(dv) + np.linalg.norm(gs) * np.linalg.norm(ds)
        fd = dL(I[0], I[1]) / (2 * h)
        errs.append(abs(fd - an) / max(abs(an), 0.1 * scale))
    print(f"\n[c3 autograd FP64 vs central differences, 64 directions] max rel err {max(errs):.2e}, "
          f"median {np.median(errs):.2e}")
    assert max(errs) < 1e-5


def test_c3_properties_and_determinism(renderers):
    r32, _ = renderers
    case = synth.config_c3()
    Vd, Fd = _dev(case.V_true), _dev(case.F)
    img = r32.render(Vd, Fd, case.grid, case.psf)
    total = float(img.double().sum()) * np.prod(case.grid.h)
    print(f"\n[c3 256x256x128] total intensity - 1 = {total - 1:.2e}")
    assert abs(total - 1.0) < 1e-5
    T = torch.zeros_like(img)
    a = r32.loss_and_grad(Vd, Fd, case.grid, case.psf, T, "mse")
    b = r32.loss_and_grad(Vd, Fd, case.grid, case.psf, T, "mse")
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def _largest_request():
    grid = synth.Grid(n=(256, 256, 256), h=(0.5, 0.5, 1.0))
    R = 0.3 * float(min(grid.L))
    V, F = synth.sh_deformed_sphere(6, R, grid.center, lmax=6, coef_sigma=0.03 * R, seed=10_006)
    psf = synth.Psf(sigma=(0.2, 0.2, 0.6), band_tau=1e-3)
    return grid, psf, V, F


class _Case:
    def __init__(self, grid, psf):
        self.grid, self.psf = grid, psf


def test_largest_request_against_the_oracle_on_sampled_frequencies(renderers):
    r32, r64 = renderers
    grid, psf, V, F = _largest_request()
    fn = _sample_band(_Case(grid, psf), 128, seed=8)
    xi = oracle.wavevectors(fn, grid)
    Vo = V - np.asarray(grid.origin)
    ref = oracle.mesh_ft(Vo, F, xi)
    rng = np.random.default_rng(9)
    G = (rng.normal(size=len(fn)) + 1j * rng.normal(size=len(fn))) / len(fn)
    dref = oracle.mesh_ft_adjoint(Vo, F, xi, G)
    S32 = r32.meshft(_dev(V), _dev(F), grid, _dev(fn)).cpu().numpy()
    d32 = r32.meshft_adjoint(_dev(V), _dev(F), grid, _dev(fn), _dev(G)).cpu().numpy()
    e_s, e_d = rel(S32, ref), rel(d32, dref)
    print(f"\n[81920 triangles, 256^3] FP32 sampled spectrum {e_s:.2e}  adjoint {e_d:.2e}")
    assert e_s < 1e-5 and e_d < 1e-4


def test_largest_request_properties_and_determinism(renderers):
    r32, _ = renderers
    grid, psf, V, F = _largest_request()
    Vd, Fd = _dev(V), _dev(F)
    img = r32.render(Vd, Fd, grid, psf)
    total = float(img.double().sum()) * np.prod(grid.h)
    print(f"\n[81920 triangles, 256^3] total intensity - 1 = {total - 1:.2e}")
    assert abs(total - 1.0) < 1e-5
    T = torch.zeros_like(img)
    a = r32.loss_and_grad(Vd, Fd, grid, psf, T, "mse")
    b = r32.loss_and_grad(Vd, Fd, grid, psf, T, "mse")
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
