"""Pins of the oracle's optimisation layer (Section 5.1 staggered scheme and large-steps update,
Section 5.2 PSF step).

References: the spectrum of the icosahedron graph, a brute-force dense Laplacian, the closed
forms of uniform and plain Adam under a constant gradient
and without memory, plain Adam's moments written as explicit weighted sums, the dense matrix power (1 + lambda L)^-2,
finite differences through Sigma = C C^T, and the invariants of the two sub-problems.
"""

import numpy as np
import pytest

import oracle
import oracle.optim as opt
import synth


def _dense_laplacian(F, n_v):
    """Brute force: degree minus adjacency from a Python set of edges."""
    E = set()
    for t in F:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            if a != b:
                E.add((min(a, b), max(a, b)))
    L = np.zeros((n_v, n_v))
    for a, b in E:
        L[a, b] -= 1
        L[b, a] -= 1
        L[a, a] += 1
        L[b, b] += 1
    return L


def test_icosahedron_laplacian_spectrum():
    """The icosahedron graph is 5-regular with adjacency eigenvalues 5, sqrt5 (x3), -1 (x5), -sqrt5 (x3)."""
    V, F = synth.sphere_mesh(0, 1.0, (0.0, 0.0, 0.0))
    ev = np.linalg.eigvalsh(opt.laplacian(F, 12).toarray())
    s5 = np.sqrt(5.0)
    ref = np.sort([0.0] + [5 - s5] * 3 + [6.0] * 5 + [5 + s5] * 3)
    assert np.max(np.abs(ev - ref)) < 1e-12


def test_laplacian_and_solve_match_brute_force():
    V, F = synth.sh_deformed_sphere(2, 5.0, (0, 0, 0), lmax=3, coef_sigma=0.3, seed=2)
    n_v = len(V)
    Ld = _dense_laplacian(F, n_v)
    assert np.array_equal(opt.laplacian(F, n_v).toarray(), Ld)
    B = np.random.default_rng(0).normal(size=(n_v, 3))
    X = opt.smooth_solve(F, n_v, 50.0, B)
    Xd = np.linalg.solve(np.eye(n_v) + 50.0 * Ld, B)
    assert np.max(np.abs(X - Xd)) < 1e-10 * np.max(np.abs(Xd))
    # constants are in the null space of L: (1 + lam L) 1 = 1
    assert np.allclose(opt.smooth_solve(F, n_v, 50.0, np.ones((n_v, 3))), 1.0, atol=1e-12)


def test_uniform_adam_closed_forms():
    g = np.random.default_rng(1).normal(size=(40, 3))
    m, v = np.zeros_like(g), np.zeros_like(g)
    # a constant gradient: the bias-corrected moments are exactly g and g^2 at every step
    for t in range(1, 6):
        d, m, v = opt.adam_uniform(g, m, v, t, 0.1, 0.9, 0.999, 0.0)
        assert np.max(np.abs(d - 0.1 * g / np.abs(g).max())) < 1e-14
    # no memory: the step is the gradient scaled by its largest magnitude
    g2 = np.random.default_rng(2).normal(size=(40, 3))
    d, _, _ = opt.adam_uniform(g2, m, v, 7, 0.3, 0.0, 0.0, 0.0)
    assert np.max(np.abs(d - 0.3 * g2 / np.abs(g2).max())) < 1e-14


def test_adam_closed_forms():
    """Plain Adam (Kingma and Ba 2014; the PSF step of Section 5.2 and the plain vertex optimiser)."""
    g = np.random.default_rng(5).normal(size=(40, 3))
    m, v = np.zeros_like(g), np.zeros_like(g)
    # a constant gradient: the bias-corrected moments are exactly g and g^2, so every step is
    # lr g / (|g| + eps) (a missing or wrong bias correction scales steps 1..5 differently)
    for t in range(1, 6):
        d, m, v = opt.adam(g, m, v, t, 0.1, 0.9, 0.999, 1e-3)
        assert np.max(np.abs(d - 0.1 * g / (np.abs(g) + 1e-3))) < 1e-14
    # no memory (beta1 = beta2 = 0): the step is lr g / (|g| + eps) whatever the history
    g2 = np.random.default_rng(6).normal(size=(40, 3))
    d, _, _ = opt.adam(g2, m, v, 7, 0.3, 0.0, 0.0, 1e-2)
    assert np.max(np.abs(d - 0.3 * g2 / (np.abs(g2) + 1e-2))) < 1e-14
    # the first step is lr sign(g) when eps = 0, for any beta
    d, _, _ = opt.adam(g2, np.zeros_like(g2), np.zeros_like(g2), 1, 0.2, 0.7, 0.95, 0.0)
    assert np.max(np.abs(d - 0.2 * np.sign(g2))) < 1e-14


def test_adam_matches_the_moments_written_as_weighted_sums():
    """The recursion against the moments' explicit form: m_hat_t = sum_i b1^(t-i) (1 - b1) g_i / (1 - b1^t)
    (the bias correction makes the weights sum to one), likewise v_hat with g_i^2; also the scale invariance
    of the step (eps = 0) and Kingma and Ba's bound |step| <= lr (1 - b1) / sqrt(1 - b2) for (1 - b1) >
    sqrt(1 - b2)."""
    rng = np.random.default_rng(7)
    b1, b2, lr, eps = 0.9, 0.999, 0.05, 1e-8
    gs = [rng.normal(size=(30, 3)) * rng.uniform(0.1, 3.0) for _ in range(9)]
    m, v = np.zeros((30, 3)), np.zeros((30, 3))
    for t in range(1, len(gs) + 1):
        d, m, v = opt.adam(gs[t - 1], m, v, t, lr, b1, b2, eps)
        w1 = np.array([b1 ** (t - i) * (1 - b1) for i in range(1, t + 1)])
        w2 = np.array([b2 ** (t - i) * (1 - b2) for i in range(1, t + 1)])
        assert abs(w1.sum() - (1 - b1**t)) < 1e-15 and abs(w2.sum() - (1 - b2**t)) < 1e-15
        mh = sum(w * g for w, g in zip(w1, gs[:t])) / w1.sum()
        vh = sum(w * g * g for w, g in zip(w2, gs[:t])) / w2.sum()
        ref = lr * mh / (np.sqrt(vh) + eps)
        assert np.max(np.abs(d - ref)) < 1e-13 * lr
    # scale invariance with eps = 0: gradients times c > 0 give the same steps
    m1, v1, m2, v2 = (np.zeros((30, 3)) for _ in range(4))
    for t, g in enumerate(gs, start=1):
        d1, m1, v1 = opt.adam(g, m1, v1, t, lr, b1, b2, 0.0)
        d2, m2, v2 = opt.adam(1e-9 * g, m2, v2, t, lr, b1, b2, 0.0)
        assert np.max(np.abs(d1 - d2)) < 1e-13 * lr
    # the step bound, on the worst case for it: one large gradient after many zeros
    b1, b2 = 0.5, 0.99  # (1 - b1) = 0.5 > sqrt(1 - b2) = 0.1
    m, v = np.zeros(1), np.zeros(1)
    steps = []
    for t in range(1, 60):
        # with eps = 0 the zero-gradient steps are 0/0; only the moments carry over from them
        with np.errstate(invalid="ignore"):
            d, m, v = opt.adam(np.array([1.0 if t == 59 else 0.0]), m, v, t, 1.0, b1, b2, 0.0)
        steps.append(abs(d[0]) if t == 59 else 0.0)
    bound = (1 - b1) / np.sqrt(1 - b2)
    assert steps[-1] <= bound * (1 + 1e-12) and steps[-1] > 0.6 * bound


def test_large_steps_without_moments_is_the_printed_update():
    """With beta1 = beta2 = 0 the update is v - eta (1 + lam L)^-2 dL/dv (one uniform scale)."""
    V, F = synth.sh_deformed_sphere(1, 5.0, (0, 0, 0), lmax=2, coef_sigma=0.3, seed=3)
    n_v, lam = len(V), 50.0
    g = np.random.default_rng(4).normal(size=(n_v, 3))
    gu = opt.smooth_solve(F, n_v, lam, g)
    d, _, _ = opt.adam_uniform(gu, np.zeros_like(g), np.zeros_like(g), 1, 0.05, 0.0, 0.0, 0.0)
    step = opt.smooth_solve(F, n_v, lam, d)
    Ainv = np.linalg.inv(np.eye(n_v) + lam * _dense_laplacian(F, n_v))
    ref = 0.05 / np.abs(Ainv @ g).max() * (np.linalg.matrix_power(Ainv, 2) @ g)
    assert np.max(np.abs(step - ref)) < 1e-10 * np.max(np.abs(ref))


def test_cholesky_round_trip_and_psd():
    c = np.array([0.9, 1.1, 1.6, 0.2, -0.3, 0.25])
    cov = opt.chol_to_cov(c)
    assert np.allclose(opt.cov_to_chol(cov), c, atol=1e-14)
    S = oracle.covariance(synth.Psf(sigma=(1, 1, 1), cov=cov))
    assert np.all(np.linalg.eigvalsh(S) > 0)


def test_cholesky_gradient_matches_finite_differences():
    grid = synth.Grid(n=(10, 9, 8), h=(1.0, 1.2, 1.5), origin=(0.3, -0.4, 0.2))
    V, F = synth.sh_deformed_sphere(1, 0.27 * min(grid.L), grid.center, lmax=3, coef_sigma=0.3, seed=0)
    c = np.array([0.9, 1.0, 1.4, 0.15, -0.1, 0.2])
    T = oracle.render(V * 0.97 + 0.1, F, grid, opt._psf_full(opt.chol_to_cov(c * 1.1), 0.0))["image"]

    def L(cc):
        return oracle.loss_value(oracle.render(V, F, grid, opt._psf_full(opt.chol_to_cov(cc), 0.0))["image"], T,
                                 "l2")[0]

    _, _, dcov, _ = oracle.loss_and_grad(V, F, grid, opt._psf_full(opt.chol_to_cov(c), 0.0), T, "l2")
    gc = opt.chol_grad(c, dcov)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd = (L(c + e) - L(c - e)) / (2 * h)
        assert abs(gc[k] - fd) <= 1e-6 * np.abs(gc).sum()


def _tiny_fit_case():
    grid = synth.Grid(n=(12, 12, 10), h=(1.0, 1.0, 1.5))
    V0, F = synth.sphere_mesh(1, 3.2, grid.center)
    Vt = synth.scale_about(V0, (1.08, 0.95, 1.0), grid.center)
    true_cov = (1.0, 1.1, 2.0, 0.25, 0.1, -0.15)
    T = oracle.render(Vt, F, grid, opt._psf_full(true_cov, 0.0))["image"]
    return grid, V0, F, T, true_cov


def test_the_two_sub_problems_hold_their_other_unknown():
    grid, V0, F, T, _ = _tiny_fit_case()
    psf0 = synth.Psf(sigma=(1.1, 1.1, 1.3), band_tau=1e-2)
    V1, cov1, hs, hp = opt.fit_staggered(V0, F, grid, psf0, T, rounds=1, shape_steps=0, psf_steps=2,
                                         lr_vertex=0.05, lr_psf=0.01)
    assert np.array_equal(V1, V0) and len(hs) == 0 and len(hp) == 2
    assert cov1 != opt.initial_cov(psf0)
    # the PSF loss is taken on the whole half spectrum, not on the band of tau
    full = oracle.loss_value(oracle.render(V0, F, grid, synth.Psf(sigma=psf0.sigma))["image"], T, "l2")[0]
    assert abs(hp[0] - full) < 1e-12 * full
    V2, cov2, hs, hp = opt.fit_staggered(V0, F, grid, psf0, T, rounds=1, shape_steps=2, psf_steps=0,
                                         lr_vertex=0.05, lr_psf=0.01)
    assert np.allclose(cov2, opt.initial_cov(psf0), rtol=1e-14) and not np.array_equal(V2, V0)
    band = oracle.loss_value(oracle.render(V0, F, grid, psf0)["image"], T, "weighted")[0]
    assert abs(hs[0] - band) < 1e-12 * band


@pytest.mark.parametrize("optimizer,lr_vertex", [("large_steps", 0.5), ("adam", 0.03)])
def test_staggered_fit_recovers_shape_and_covariance(optimizer, lr_vertex):
    grid, V0, F, T, true_cov = _tiny_fit_case()
    psf0 = synth.Psf(sigma=(1.1, 1.1, 1.3), band_tau=1e-3)
    V1, cov1, hs, hp = opt.fit_staggered(V0, F, grid, psf0, T, rounds=6, shape_steps=5, psf_steps=5,
                                         lr_vertex=lr_vertex, lr_psf=0.02, optimizer=optimizer)
    assert hp[-1] < 0.3 * hp[0] and hs[-1] < 0.5 * hs[0]
    err0 = np.abs(np.array(opt.initial_cov(psf0)) - true_cov).sum()
    err1 = np.abs(np.array(cov1) - true_cov).sum()
    assert err1 < 0.6 * err0, (cov1, true_cov)
