"""The hand-written adjoint behind torch.autograd: central finite differences and the oracle.

Workload: the SH l <= 10 cell of the 256x256x128 case, at icosphere level 4, on a 64x64x32
grid spanning the same 128 um box (voxels (2, 2, 4) um), sigma (0.25, 0.25, 0.7) um, MSE
against a render of the deformed cell with sigma (0.3, 0.3, 0.9).
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _case():
    grid = synth.Grid(n=(64, 64, 32), h=(2.0, 2.0, 4.0))
    V_t, F = synth.sh_deformed_sphere(4, 30.0, grid.center, lmax=10, coef_sigma=0.9, seed=3)
    V0, _ = synth.sphere_mesh(4, 30.0, grid.center)
    return grid, V_t, V0, F


@pytest.fixture(scope="module")
def rr():
    from paper_2303_10440_b300 import Renderer

    r32, r64 = Renderer("fp32"), Renderer("fp64")
    yield r32, r64
    r32.close()
    r64.close()


def _loss_fn(renderer, grid, F, T):
    from paper_2303_10440_b300.autograd import render

    def L(V, sigma):
        img = render(V, sigma, F, renderer, grid)
        return ((img.double() - T) ** 2).mean()

    return L


def test_autograd_matches_central_differences_fp64(rr):
    _, r64 = rr
    grid, V_t, V0, F = _case()
    dev = torch.device("cuda")
    Fd = torch.as_tensor(F).to(dev)
    T = r64.render(torch.as_tensor(V_t).to(dev), Fd, grid, synth.Psf(sigma=(0.25, 0.25, 0.7)))
    L = _loss_fn(r64, grid, Fd, T)
    V = torch.as_tensor(V0).to(dev).requires_grad_(True)
    sig = torch.tensor([0.3, 0.3, 0.9], dtype=torch.float64, requires_grad=True)
    loss = L(V, sig)
    loss.backward()
    gV, gs = V.grad.double(), sig.grad.double()
    rng = np.random.default_rng(0)
    h = 1e-6
    errs = []
    with torch.no_grad():
        for k in range(64):
            dV = torch.as_tensor(rng.normal(size=V0.shape)).to(dev)
            ds = torch.as_tensor(rng.normal(size=3) * 0.1)
            if k < 8:  # a few pure-PSF and pure-vertex directions
                dV = dV * 0 if k % 2 == 0 else dV
                ds = ds if k % 2 == 0 else ds * 0
            fd = (L(V + h * dV, sig + h * ds) - L(V - h * dV, sig - h * ds)) / (2 * h)
            an = (gV * dV).sum() + (gs * ds).sum()
            errs.append(abs(float(fd - an)) / max(abs(float(an)), 1e-30))
    print(f"\n[autograd FP64 vs central differences, 64 directions] max rel err {max(errs):.2e}, "
          f"median {np.median(errs):.2e}")
    assert max(errs) < 1e-5


def test_autograd_fp32_gradient_matches_fp64(rr):
    r32, r64 = rr
    grid, V_t, V0, F = _case()
    dev = torch.device("cuda")
    Fd = torch.as_tensor(F).to(dev)
    T = r64.render(torch.as_tensor(V_t).to(dev), Fd, grid, synth.Psf(sigma=(0.25, 0.25, 0.7)))
    grads = []
    for r in (r32, r64):
        V = torch.as_tensor(V0).to(dev).requires_grad_(True)
        sig = torch.tensor([0.3, 0.3, 0.9], dtype=torch.float64, requires_grad=True)
        _loss_fn(r, grid, Fd, T)(V, sig).backward()
        grads.append((V.grad.cpu().numpy(), sig.grad.numpy()))
    eV = np.linalg.norm(grads[0][0] - grads[1][0]) / np.linalg.norm(grads[1][0])
    es = np.linalg.norm(grads[0][1] - grads[1][1]) / np.linalg.norm(grads[1][1])
    print(f"\n[autograd FP32 vs FP64] dV {eV:.2e} dsigma {es:.2e}")
    assert eV < 1e-3 and es < 1e-3


def test_autograd_matches_oracle_gradient(rr):
    _, r64 = rr
    grid = synth.Grid(n=(16, 12, 10), h=(1.0, 1.0, 1.5), origin=(0.5, -0.25, 1.0))
    V, F = synth.sh_deformed_sphere(2, 4.0, grid.center, lmax=4, coef_sigma=0.4, seed=7)
    psf = synth.Psf(sigma=(0.8, 1.0, 1.4))
    T = oracle.render(V * 1.02, F, grid, psf)["image"]
    _, dV0, dp0, _ = oracle.loss_and_grad(V, F, grid, psf, T, "l2")
    dev = torch.device("cuda")
    from paper_2303_10440_b300.autograd import render

    Vt = torch.as_tensor(V).to(dev).requires_grad_(True)
    sig = torch.tensor(psf.sigma, dtype=torch.float64, requires_grad=True)
    img = render(Vt, sig, torch.as_tensor(F).to(dev), r64, grid)
    # only the inputs are kept for backward: the spectrum is recomputed in the adjoint call
    saved = img.grad_fn.saved_tensors
    assert sum(t.numel() for t in saved) == Vt.numel() + 3
    ((img - torch.as_tensor(T).to(dev)) ** 2).sum().backward()
    assert np.linalg.norm(Vt.grad.cpu().numpy() - dV0) < 1e-9 * np.linalg.norm(dV0)
    assert np.linalg.norm(sig.grad.numpy() - dp0) < 1e-9 * np.linalg.norm(dp0)
