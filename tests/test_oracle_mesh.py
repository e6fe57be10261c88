"""Pins of the oracle's mesh transform (Eq. 5), the volume-labelled mode and the mesh adjoint.

Independent references: the closed-form transform of an axis-aligned box (surface
and volume, a product of sincs), the analytic sphere shell / ball transforms that
fine icospheres converge to, k = 0 (area, volume), the divergence-theorem form of
the volume transform, and finite differences for the adjoint.
"""

import numpy as np
import pytest

import oracle
import synth


def _seg(xi, lo, hi):
    """int_lo^hi exp(-i xi t) dt."""
    ell = hi - lo
    return ell * np.exp(-1j * xi * 0.5 * (lo + hi)) * np.sinc(xi * ell / (2 * np.pi))


def _box_surface(xi, lo, hi):
    Ia = [_seg(xi[a], lo[a], hi[a]) for a in range(3)]
    tot = 0j
    for a in range(3):
        b, c = [k for k in range(3) if k != a]
        tot += (np.exp(-1j * xi[a] * lo[a]) + np.exp(-1j * xi[a] * hi[a])) * Ia[b] * Ia[c]
    return tot


def _box_volume(xi, lo, hi):
    return np.prod([_seg(xi[a], lo[a], hi[a]) for a in range(3)])


def test_box_closed_form_on_grid_frequencies():
    """Grid frequencies of a box with edges on the axes hit e.xi = 0 exactly (Section 4.1.3)."""
    lo, hi = np.array([3.0, 5.0, 2.0]), np.array([11.0, 9.0, 14.0])
    V, F = synth.box_mesh(lo, hi)
    grid = synth.Grid(n=(16, 16, 16), h=(1.0, 1.0, 1.25))
    nvec, _ = oracle.half_spectrum(grid.n)
    xi = oracle.wavevectors(nvec, grid)
    S = oracle.mesh_ft(V, F, xi, "surface")
    Sv = oracle.mesh_ft(V, F, xi, "volume", c0=0.5 * grid.L)
    ref = np.array([_box_surface(x, lo, hi) for x in xi])
    refv = np.array([_box_volume(x, lo, hi) for x in xi])
    assert np.max(np.abs(S - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(Sv - refv)) <= 1e-13 * np.max(np.abs(refv))
    area = 2 * ((hi - lo)[0] * (hi - lo)[1] + (hi - lo)[1] * (hi - lo)[2] + (hi - lo)[0] * (hi - lo)[2])
    assert abs(S[0] - area) < 1e-11 and abs(Sv[0] - np.prod(hi - lo)) < 1e-11


def test_sphere_convergence_rate():
    """Icospheres approach 4 pi R^2 sin(kR)/(kR) and 4 pi (sin kR - kR cos kR)/k^3 at ~4x per level."""
    R, k = 1.3, 3.1
    dirs = np.array([[1, 0, 0], [0, 0.6, 0.8], [0.48, 0.6, 0.64]])
    xi = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * k
    shell = 4 * np.pi * R * R * np.sin(k * R) / (k * R)
    ball = 4 * np.pi * (np.sin(k * R) - k * R * np.cos(k * R)) / k**3
    es, ev = [], []
    for lev in (2, 3, 4, 5):
        V, F = synth.sphere_mesh(lev, R, (0.3, -0.2, 0.1))
        ph = np.exp(-1j * xi @ np.array([0.3, -0.2, 0.1]))
        es.append(np.max(np.abs(oracle.mesh_ft(V, F, xi) - shell * ph)) / abs(shell))
        ev.append(np.max(np.abs(oracle.mesh_ft(V, F, xi, "volume") - ball * ph)) / abs(ball))
    for e in (es, ev):
        ratios = np.array(e[:-1]) / np.array(e[1:])
        assert np.all(ratios > 3.5) and np.all(ratios < 4.5), e
    assert es[-1] < 1e-3 and ev[-1] < 5e-3


def test_zero_frequency_area_and_volume():
    V, F = synth.sh_deformed_sphere(3, 5.0, (1.0, 2.0, 3.0), lmax=4, coef_sigma=0.3, seed=9)
    S0 = oracle.mesh_ft(V, F, np.zeros((1, 3)))[0]
    Sv0 = oracle.mesh_ft(V, F, np.zeros((1, 3)), "volume", c0=np.array([1.0, 2.0, 3.0]))[0]
    assert abs(S0 - oracle.surface_area(V, F)) < 1e-11
    assert abs(Sv0 - oracle.enclosed_volume(V, F)) < 1e-10


def test_volume_tetrahedra_match_divergence_theorem():
    """int_V exp(-i x.xi) dV = (i/|xi|^2) sum_T (xi . n_T) int_T exp(-i x.xi) dS / (2 A_T) (closed mesh)."""
    V, F = synth.sh_deformed_sphere(2, 4.0, (0.5, 0.0, -1.0), lmax=3, coef_sigma=0.4, seed=4)
    rng = np.random.default_rng(3)
    xi = rng.normal(size=(20, 3)) * 1.5
    Sv = oracle.mesh_ft(V, F, xi, "volume", c0=np.array([7.0, -3.0, 2.0]))
    for m in range(xi.shape[0]):
        tot = 0j
        for a, b, c in F:
            n = np.cross(V[b] - V[a], V[c] - V[a])
            A2 = np.linalg.norm(n)
            tot += (xi[m] @ n) * oracle.tri_ft(V[a], V[b], V[c], xi[m]) / A2
        ref = 1j * tot / (xi[m] @ xi[m])
        assert abs(Sv[m] - ref) < 1e-11 * max(1.0, abs(ref))


def test_translation_and_hermitian_on_mesh():
    V, F = synth.sphere_mesh(2, 3.0, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(12)
    xi = rng.normal(size=(8, 3))
    t = np.array([4.0, -1.5, 2.25])
    S = oracle.mesh_ft(V, F, xi)
    assert np.allclose(oracle.mesh_ft(V + t, F, xi), S * np.exp(-1j * xi @ t), atol=1e-12)
    assert np.allclose(oracle.mesh_ft(V, F, -xi), np.conj(S), atol=1e-12)


@pytest.mark.parametrize("mode", ["surface", "volume"])
def test_mesh_adjoint_matches_finite_differences(mode):
    V, F = synth.sh_deformed_sphere(1, 2.0, (0.2, 0.1, -0.3), lmax=3, coef_sigma=0.2, seed=21)
    rng = np.random.default_rng(22)
    xi = rng.normal(size=(12, 3)) * 1.2
    xi[0] = 0.0
    Gs = rng.normal(size=12) + 1j * rng.normal(size=12)
    c0 = np.array([0.5, -0.5, 0.25])
    dV = oracle.mesh_ft_adjoint(V, F, xi, Gs, mode, c0)

    def J(W):
        return float(np.sum(np.real(np.conj(Gs) * oracle.mesh_ft(W, F, xi, mode, c0))))

    h = 1e-6
    for _ in range(8):
        d = rng.normal(size=V.shape)
        fd = (J(V + h * d) - J(V - h * d)) / (2 * h)
        assert abs(np.sum(dV * d) - fd) < 1e-7 * max(1.0, abs(fd))
    # a pure translation: sum_v dS/dv = -i xi S
    S = oracle.mesh_ft(V, F, xi, mode, c0)
    ref = np.real(np.conj(Gs)[:, None] * (-1j * xi * S[:, None])).sum(axis=0)
    assert np.allclose(dV.sum(axis=0), ref, atol=1e-10)


def test_box_foam_with_doubled_walls_is_the_sum_of_its_cells():
    """A tissue of 2 x 2 x 1 box cells in one non-manifold mesh, shared walls at density 2
    (Section 3.3), equals the sum of the four cells' closed surfaces (closed-form sinc products)."""
    size, org = np.array([6.0, 5.0, 7.0]), np.array([2.0, 1.5, 3.0])
    V, F, rho = synth.box_foam((2, 2, 1), size, subdiv=3, origin=org)
    grid = synth.Grid(n=(16, 16, 12), h=(1.0, 1.0, 1.25))
    nvec, _ = oracle.half_spectrum(grid.n)
    xi = oracle.wavevectors(nvec, grid)[::7]
    S = oracle.mesh_ft(V, F, xi, "surface", weights=rho)
    ref = np.zeros(len(xi), dtype=complex)
    for i in range(2):
        for j in range(2):
            lo = org + size * np.array([i, j, 0])
            ref += np.array([_box_surface(x, lo, lo + size) for x in xi])
    assert np.max(np.abs(S - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(oracle.surface_area(V, F, rho) - 4 * 2 * (size[0] * size[1] + size[1] * size[2] + size[0] * size[2])) < 1e-9
