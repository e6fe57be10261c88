"""Pins of the oracle's triangle transform and its gradient (Section 4.1.2-4.1.3, Eq. 7-12).

Each check is independent of the oracle's own algorithm (sorted divided-difference
recursion + series): 50-digit evaluation of the generic Eq. 8 expansion,
Gauss-Legendre quadrature of the defining integral, exact symmetry laws of the
Fourier integral, and finite differences.
"""

import mpmath as mp
import numpy as np
import pytest

import oracle


def _duffy_quadrature(v1, v2, v3, xi, n=60):
    """int_T exp(-i x.xi) dS by n x n Gauss-Legendre on the unit square (Duffy map)."""
    g, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (g + 1.0)
    ws = 0.5 * w
    S, T = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws)
    x = v1[None, None, :] + S[..., None] * (v2 - v1)[None, None, :] + (S * T)[..., None] * (v3 - v2)[None, None, :]
    A2 = np.linalg.norm(np.cross(v2 - v1, v3 - v1))
    return A2 * np.sum(W * S * np.exp(-1j * (x @ xi)))


def _generic_g_mp(phis):
    """Eq. 8 in 50-digit arithmetic: sum_p exp(-i phi_p) / ((e_{p-}.xi)(e_{p+}.xi)).

    With e_p = v_{p-1} - v_{p+1}: e_{p-}.xi = phi_{p+1} - phi_p and e_{p+}.xi = phi_p - phi_{p-1}.
    """
    mp.mp.dps = 50
    z = [mp.mpf(float(p)) for p in phis]
    tot = mp.mpc(0)
    for p in range(3):
        em = z[(p + 1) % 3] - z[p]
        ep = z[p] - z[(p - 1) % 3]
        tot += mp.exp(-1j * z[p]) / (em * ep)
    return complex(tot)


def test_dd_matches_high_precision_generic_formula():
    rng = np.random.default_rng(1)
    cases = [rng.normal(size=3) * s for s in (0.01, 0.3, 1.0, 5.0, 40.0)]
    cases += [np.array([0.0, 1e-7, 2.0]), np.array([1.0, 1.0 + 1e-9, 1.0 + 3e-9]), np.array([0.0, 0.0, 50.0])]
    cases += [np.array([300.0, 300.2, 299.9]), np.array([-700.0, -650.0, -712.5])]
    for z in cases:
        if min(abs(z[0] - z[1]), abs(z[1] - z[2]), abs(z[0] - z[2])) == 0:
            continue
        ref = _generic_g_mp(z)
        got = oracle.dd(z, 2)
        # absolute rounding of exp(-i phi) at |phi| ~ 700 is ~1e-13; |f| >= ~1e-4 here
        assert abs(got - ref) <= 1e-13 * max(1.0, np.max(np.abs(z))) * max(abs(ref), 1e-3), (z, got, ref)


def test_dd_special_cases_eq12():
    """Eq. 12a/12b (with vertex phases and exp(-i.), the reading the special cases themselves use)."""
    for u in (0.0, 0.7, -3.2, 250.0):
        assert abs(oracle.dd([u, u, u], 2) - np.exp(-1j * u) / 2) < 1e-14
    for t, u in ((0.3, 1.9), (-2.0, 5.0), (10.0, 10.6), (0.0, 1e-3)):
        ref = 1j * np.exp(-1j * t) / (t - u) + np.exp(-1j * t) / (t - u) ** 2 - np.exp(-1j * u) / (t - u) ** 2
        if abs(t - u) > 0.1:
            for nodes in ([t, t, u], [u, t, t], [t, u, t]):
                assert abs(oracle.dd(nodes, 2) - ref) < 1e-13
        # confluent limit is continuous: a split of 1e-9 changes f by O(1e-9)
        assert abs(oracle.dd([t, t + 1e-9, u], 2) - oracle.dd([t, t, u], 2)) < 1e-8


@pytest.mark.parametrize("seed", range(6))
def test_triangle_ft_matches_quadrature(seed):
    rng = np.random.default_rng(100 + seed)
    v = rng.normal(size=(3, 3))
    diam = max(np.linalg.norm(v[i] - v[j]) for i in range(3) for j in range(3))
    for scale in (0.0, 0.05, 1.0, 8.0, 20.0):
        xi = rng.normal(size=3)
        xi *= scale / (np.linalg.norm(xi) * diam)
        ref = _duffy_quadrature(v[0], v[1], v[2], xi)
        got = oracle.tri_ft(v[0], v[1], v[2], xi)
        assert abs(got - ref) <= 1e-12 * max(abs(ref), 1e-2), (scale, got, ref)


def test_triangle_ft_degenerate_wavevectors_match_quadrature():
    """xi orthogonal to an edge (e.xi = 0 exactly) or to the whole triangle."""
    v = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.5, 1.5, 0.0]])
    for xi in ([0.0, 3.0, 0.0], [0.0, 0.0, 7.0], [1e-9, 2.0, 0.0], [0.0, 0.0, 0.0], [4.0, 0.0, 0.0]):
        xi = np.array(xi)
        ref = _duffy_quadrature(v[0], v[1], v[2], xi)
        assert abs(oracle.tri_ft(v[0], v[1], v[2], xi) - ref) <= 1e-12 * max(abs(ref), 1e-2)


def test_triangle_symmetries():
    rng = np.random.default_rng(7)
    v = rng.normal(size=(3, 3))
    A = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    assert abs(oracle.tri_ft(v[0], v[1], v[2], np.zeros(3)) - A) < 1e-15
    for _ in range(5):
        xi = rng.normal(size=3) * 3
        u = oracle.tri_ft(v[0], v[1], v[2], xi)
        # Hermitian symmetry of the transform of a real density
        assert abs(oracle.tri_ft(v[0], v[1], v[2], -xi) - np.conj(u)) < 1e-14
        # translation by t multiplies by exp(-i xi.t)
        t = rng.normal(size=3) * 10
        ut = oracle.tri_ft(v[0] + t, v[1] + t, v[2] + t, xi)
        assert abs(ut - np.exp(-1j * xi @ t) * u) < 1e-12
        # scaling x -> s x: u_{sT}(xi) = s^2 u_T(s xi)
        s = 1.7
        assert abs(oracle.tri_ft(s * v[0], s * v[1], s * v[2], xi) - s * s * oracle.tri_ft(v[0], v[1], v[2], s * xi)) < 1e-13
        # vertex order (cyclic and reflected) does not change the surface integral
        assert abs(oracle.tri_ft(v[1], v[2], v[0], xi) - u) < 1e-14
        assert abs(oracle.tri_ft(v[0], v[2], v[1], xi) - u) < 1e-14
        # 1 -> 4 midpoint subdivision leaves the integral unchanged
        m01, m12, m20 = 0.5 * (v[0] + v[1]), 0.5 * (v[1] + v[2]), 0.5 * (v[2] + v[0])
        parts = [(v[0], m01, m20), (v[1], m12, m01), (v[2], m20, m12), (m01, m12, m20)]
        assert abs(sum(oracle.tri_ft(*p, xi) for p in parts) - u) < 1e-13


def _paper_eq10_bracket(v, xi, p):
    """The printed Eq. 10 bracket for vertex p (0-based), with e_p = v_{p-1} - v_{p+1}."""
    phi = v @ xi
    e = [v[2] - v[1], v[0] - v[2], v[1] - v[0]]
    em, ep, e0 = e[(p - 1) % 3] @ xi, e[(p + 1) % 3] @ xi, e[p] @ xi
    return (
        np.exp(-1j * phi[(p + 1) % 3]) / (em**2 * e0)
        - np.exp(-1j * phi[(p - 1) % 3]) / (e0 * ep**2)
        - 1j * np.exp(-1j * phi[p]) / (em * ep)
        + np.exp(-1j * phi[p]) / (em**2 * ep)
        - np.exp(-1j * phi[p]) / (em * ep**2)
    )


def test_triangle_gradient_eq9_eq10_and_fd():
    rng = np.random.default_rng(11)
    for trial in range(6):
        v = rng.normal(size=(3, 3))
        xi = rng.normal(size=3) * (0.05 if trial == 0 else 2.0)
        G = oracle.tri_grad(v[0], v[1], v[2], xi)
        h = 1e-6
        for p in range(3):
            for a in range(3):
                vp, vm = v.copy(), v.copy()
                vp[p, a] += h
                vm[p, a] -= h
                fd = (oracle.tri_ft(*vp, xi) - oracle.tri_ft(*vm, xi)) / (2 * h)
                assert abs(G[p, a] - fd) < 1e-7 * max(1.0, abs(fd)), (trial, p, a, G[p, a], fd)
        # sum over vertices of the gradient = gradient of a translation = -i xi u
        u = oracle.tri_ft(v[0], v[1], v[2], xi)
        assert np.allclose(G.sum(axis=0), -1j * xi * u, atol=1e-12)
        if trial > 0:
            # Eq. 9 with the printed Eq. 10 bracket (generic, well-separated phases)
            e = [v[2] - v[1], v[0] - v[2], v[1] - v[0]]
            n = np.cross(e[2], e[0])
            A = 0.5 * np.linalg.norm(n)
            N = n / (2 * A)
            f = u / (2 * A)
            for p in range(3):
                w = np.cross(e[p], N)
                ref = -f * w + 2 * A * xi * _paper_eq10_bracket(v, xi, p)
                assert np.allclose(G[p], ref, rtol=1e-8, atol=1e-10)


def test_gradient_at_zero_frequency_is_area_gradient():
    rng = np.random.default_rng(5)
    v = rng.normal(size=(3, 3))
    G = oracle.tri_grad(v[0], v[1], v[2], np.zeros(3))
    h = 1e-6
    for p in range(3):
        for a in range(3):
            vp, vm = v.copy(), v.copy()
            vp[p, a] += h
            vm[p, a] -= h
            area = lambda w: 0.5 * np.linalg.norm(np.cross(w[1] - w[0], w[2] - w[0]))
            assert abs(G[p, a] - (area(vp) - area(vm)) / (2 * h)) < 1e-8
