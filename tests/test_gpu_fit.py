"""The on-device Adam fit (dm_fit) equals the per-step C-ABI loop and reduces the loss."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def r32():
    from paper_2303_10440_b300 import Renderer

    r = Renderer("fp32")
    yield r
    r.close()


def test_fit_equals_manual_loop(r32):
    case = synth.config_c2()
    grid, psf = case.grid, case.psf
    Fd = _dev(case.F)
    T = r32.render(_dev(case.V_true), Fd, grid, psf)
    lr, steps = 1e-2 * min(grid.h), 4
    Vf, sig, hist = r32.fit(_dev(case.V_init), Fd, grid, psf, T, steps=steps, lr_vertex=lr)
    V = _dev(case.V_init).clone()
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    losses = []
    for k in range(steps):
        L, dV, dp, _ = r32.loss_and_grad(V, Fd, grid, psf, T, "mse")
        losses.append(L)
        r32.adam(V, dV, m, v, k + 1, lr)
    torch.cuda.synchronize()
    assert np.array_equal(hist.numpy(), np.array(losses))
    assert torch.equal(Vf, V)


def test_fit_reduces_the_loss_and_adapts_sigma(r32):
    """A well-posed fit: a 3% dilated cell under a blur wider than the displacement."""
    grid = synth.Grid(n=(64, 64, 64), h=(0.5, 0.5, 1.0))
    V0, F = synth.sphere_mesh(3, 8.0, grid.center)
    Vt = synth.scale_about(V0, (1.03, 1.03, 1.03), grid.center)
    true_psf = synth.Psf(sigma=(0.4, 0.4, 0.8))
    Fd = _dev(F)
    T = r32.render(_dev(Vt), Fd, grid, true_psf)
    psf0 = synth.Psf(sigma=(0.45, 0.45, 0.9))
    Vf, sig, hist = r32.fit(_dev(V0), Fd, grid, psf0, T, steps=40, lr_vertex=0.02, lr_psf=0.003)
    h = hist.numpy()
    r_err0 = np.abs(np.linalg.norm(V0 - grid.center, axis=1) - 8.24).mean()
    r_err1 = np.abs(np.linalg.norm(Vf.cpu().numpy() - grid.center, axis=1) - 8.24).mean()
    print(f"\n[fit 40 steps] loss {h[0]:.3e} -> {h[-1]:.3e}; mean radius error {r_err0:.3f} -> {r_err1:.3f} um; "
          f"sigma {tuple(round(s, 4) for s in sig)}")
    assert h[-1] < 0.3 * h[0]
    assert r_err1 < 0.5 * r_err0
    assert sig[0] < 0.45  # the PSF moved toward the truth (0.4)


def test_resumed_fit_equals_the_uninterrupted_fit(r32):
    """Checkpoint / resume: 3 + 5 steps through dm_fit_resume equal 8 steps of dm_fit, bit for bit."""
    grid = synth.Grid(n=(48, 48, 48), h=(0.5, 0.5, 1.0))
    V0, F = synth.sphere_mesh(3, 6.0, grid.center)
    Fd = _dev(F)
    T = r32.render(_dev(synth.scale_about(V0, (1.04, 0.97, 1.0), grid.center)), Fd, grid, synth.Psf(sigma=(0.4, 0.4, 0.8)))
    psf0 = synth.Psf(sigma=(0.45, 0.45, 0.9))
    kw = dict(lr_vertex=0.02, lr_psf=0.003)
    V8, sig8, h8 = r32.fit(_dev(V0), Fd, grid, psf0, T, steps=8, **kw)
    Va, siga, ha, st = r32.fit_resume(_dev(V0), Fd, grid, psf0, T, 3, state=None, **kw)
    assert st["step"] == 3
    Vb, sigb, hb, st2 = r32.fit_resume(Va, Fd, grid, psf0, T, 5, state=st, **kw)
    assert st2["step"] == 8
    assert torch.equal(Vb, V8)
    assert sigb == sig8
    assert np.array_equal(np.concatenate([ha.numpy(), hb.numpy()]), h8.numpy())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_graph_replayed_fit_equals_the_directly_enqueued_fit(prec):
    """dm_fit replays one captured CUDA graph per step; with graphs off every step's kernels are
    enqueued one by one. Same kernels, same order, same arguments: bitwise the same fit."""
    import time

    from paper_2303_10440_b300 import Renderer

    grid = synth.Grid(n=(32, 32, 32), h=(0.5, 0.5, 1.0))
    V0, F = synth.sphere_mesh(1, 4.0, grid.center)
    Fd = _dev(F)
    rg, rd = Renderer(prec), Renderer(prec, graphs=False)
    T = rg.render(_dev(synth.scale_about(V0, (1.05, 0.96, 1.0), grid.center)), Fd, grid,
                  synth.Psf(sigma=(0.4, 0.4, 0.8), band_tau=1e-3))
    psf0 = synth.Psf(sigma=(0.45, 0.45, 0.9), band_tau=1e-3)
    out, ms = {}, {}
    for name, r in (("graph", rg), ("direct", rd)):
        r.fit(_dev(V0), Fd, grid, psf0, T, steps=3, lr_vertex=0.02, lr_psf=0.003)  # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        out[name] = r.fit(_dev(V0), Fd, grid, psf0, T, steps=50, lr_vertex=0.02, lr_psf=0.003)
        torch.cuda.synchronize()
        ms[name] = (time.perf_counter() - t) * 1e3 / 50
    print(f"\n[{prec} fit, 80 triangles, 32^3, band] ms per step: graph {ms['graph']:.3f}, direct {ms['direct']:.3f}")
    (Vg, sg, hg), (Vd, sd, hd) = out["graph"], out["direct"]
    assert torch.equal(Vg, Vd)
    assert sg == sd
    assert np.array_equal(hg.numpy(), hd.numpy())
    rg.close()
    rd.close()
