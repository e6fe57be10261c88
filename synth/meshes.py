"""Seeded triangle-mesh generators (geometry only).

Meshes are returned as ``(V, F)`` with ``V`` float64 ``[n_v, 3]`` and ``F``
int32 ``[n_t, 3]``. Faces are oriented counter-clockwise seen from outside, so
``(v2 - v1) x (v3 - v1)`` points outward; this is the orientation the paper's
triangle notation assumes (Section 4.1.2) and the one the volume-labelled mode
needs (closed, outward-oriented surface).
"""

from __future__ import annotations

import numpy as np

_GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0

# Regular icosahedron: 12 vertices (cyclic permutations of (0, +-1, +-phi)).
_ICO_V = np.array(
    [
        [-1, _GOLDEN, 0], [1, _GOLDEN, 0], [-1, -_GOLDEN, 0], [1, -_GOLDEN, 0],
        [0, -1, _GOLDEN], [0, 1, _GOLDEN], [0, -1, -_GOLDEN], [0, 1, -_GOLDEN],
        [_GOLDEN, 0, -1], [_GOLDEN, 0, 1], [-_GOLDEN, 0, -1], [-_GOLDEN, 0, 1],
    ],
    dtype=np.float64,
)
_ICO_F = np.array(
    [
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ],
    dtype=np.int64,
)


def _orient_outward(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Flip faces of a star-shaped (about the origin) mesh so normals point away from 0."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, a + b + c) < 0
    F = F.copy()
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: the icosahedron split 1->4 ``level`` times, projected to the sphere.

    Level s has 10*4^s + 2 vertices and 20*4^s triangles.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    V = _ICO_V / np.linalg.norm(_ICO_V, axis=1, keepdims=True)
    F = _orient_outward(V, _ICO_F)
    verts = [tuple(v) for v in V]
    for _ in range(level):
        mid: dict[tuple[int, int], int] = {}

        def midpoint(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            k = mid.get(key)
            if k is None:
                p = 0.5 * (np.asarray(verts[i]) + np.asarray(verts[j]))
                p /= np.linalg.norm(p)
                verts.append(tuple(p))
                k = len(verts) - 1
                mid[key] = k
            return k

        newF = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            newF += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        F = np.asarray(newF, dtype=np.int64)
    V = np.asarray(verts, dtype=np.float64)
    return V, F.astype(np.int32)


def sphere_mesh(level: int, radius: float, center) -> tuple[np.ndarray, np.ndarray]:
    V, F = icosphere(level)
    return V * float(radius) + np.asarray(center, dtype=np.float64), F


def _real_sph_harm(l: int, m: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonic (theta polar, phi azimuth)."""
    from scipy.special import sph_harm_y

    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return np.sqrt(2.0) * (-1) ** m * np.real(y)
    return np.sqrt(2.0) * (-1) ** m * np.imag(y)


def sh_deformed_sphere(
    level: int,
    radius: float,
    center,
    lmax: int,
    coef_sigma: float,
    seed: int,
    aniso_scale=(1.0, 1.0, 1.0),
) -> tuple[np.ndarray, np.ndarray]:
    """Icosphere whose radius is r(theta, phi) = R + sum_{l<=lmax, m} c_lm Y_lm(theta, phi).

    The coefficients c_lm are i.i.d. N(0, coef_sigma^2) drawn from
    ``numpy.random.default_rng(seed)`` in (l, m) order, l = 0..lmax, m = -l..l.
    ``aniso_scale`` scales the deformed shape about its centre afterwards.
    """
    U, F = icosphere(level)
    r = sh_radius(U, radius, lmax, coef_sigma, seed)
    V = U * r[:, None] * np.asarray(aniso_scale, dtype=np.float64)
    return V + np.asarray(center, dtype=np.float64), F


def sh_radius(U: np.ndarray, radius: float, lmax: int, coef_sigma: float, seed: int) -> np.ndarray:
    """The radius r(theta, phi) of ``sh_deformed_sphere`` along unit directions U [n, 3]
    (same coefficients for the same seed), so that distances to that surface can be measured."""
    U = np.asarray(U, dtype=np.float64)
    rng = np.random.default_rng(seed)
    theta = np.arccos(np.clip(U[:, 2], -1.0, 1.0))
    phi = np.arctan2(U[:, 1], U[:, 0])
    r = np.full(U.shape[0], float(radius))
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            r += rng.normal(0.0, coef_sigma) * _real_sph_harm(l, m, theta, phi)
    return np.maximum(r, 0.2 * radius)


def box_mesh(lo, hi) -> tuple[np.ndarray, np.ndarray]:
    """Axis-aligned box [lo, hi] as 8 vertices and 12 outward triangles."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    V = np.array(
        [[(hi if (k >> a) & 1 else lo)[a] for a in range(3)] for k in range(8)],
        dtype=np.float64,
    )
    # vertex k has bit a set when coordinate a is at `hi`
    quads = [
        (0, 2, 6, 4),  # x = lo face (bits: y,z vary)
        (1, 5, 7, 3),  # x = hi
        (0, 4, 5, 1),  # y = lo
        (2, 3, 7, 6),  # y = hi
        (0, 1, 3, 2),  # z = lo
        (4, 6, 7, 5),  # z = hi
    ]
    F = []
    for a, b, c, d in quads:
        F += [[a, b, c], [a, c, d]]
    F = np.asarray(F, dtype=np.int64)
    center = 0.5 * (lo + hi)
    F = _orient_outward(V - center, F)
    return V, F.astype(np.int32)


def scale_about(V: np.ndarray, scale, center) -> np.ndarray:
    center = np.asarray(center, dtype=np.float64)
    return (V - center) * np.asarray(scale, dtype=np.float64) + center


def random_triangles(n: int, seed: int, extent: float = 1.0, center=(0.0, 0.0, 0.0)):
    """``n`` independent triangles (a triangle soup) with vertices uniform in a cube."""
    rng = np.random.default_rng(seed)
    V = rng.uniform(-0.5 * extent, 0.5 * extent, size=(3 * n, 3)) + np.asarray(center)
    F = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return V, F


def pack_cells(
    n_cells: int,
    box,
    radius_range,
    clearance: float,
    seed: int,
    max_tries: int = 20000,
):
    """Rejection-pack non-overlapping spheres (centre, radius) inside ``box`` (3 lengths).

    Radii are uniform in ``radius_range``; two cells keep ``clearance`` between
    their bounding spheres, and every cell keeps ``clearance`` from the box walls.
    """
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    cells: list[tuple[np.ndarray, float]] = []
    tries = 0
    while len(cells) < n_cells:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could only pack {len(cells)} of {n_cells} cells")
        r = rng.uniform(*radius_range)
        lo = r + clearance
        hi = box - r - clearance
        if np.any(hi <= lo):
            continue
        c = rng.uniform(lo, hi)
        if all(np.linalg.norm(c - c2) >= r + r2 + clearance for c2, r2 in cells):
            cells.append((c, r))
    return cells


def box_foam(cells=(2, 2, 1), cell_size=(6.0, 6.0, 6.0), subdiv: int = 4, origin=(0.0, 0.0, 0.0), jitter: float = 0.0,
             seed: int = 0):
    """A tissue of box cells in one non-manifold mesh: every face of the cell lattice is split into
    subdiv x subdiv quads of two triangles; a wall between two cells appears once and carries
    density 2 (two membranes), an outer face density 1. Corner positions are shared; ``jitter``
    moves every vertex by N(0, jitter^2) (seeded). Returns (V, F, rho)."""
    nc = np.asarray(cells, dtype=np.int64)
    h = np.asarray(cell_size, dtype=np.float64) / subdiv
    npts = nc * subdiv + 1  # lattice points per axis
    index = {}
    V = []

    def vid(p):
        key = tuple(int(x) for x in p)
        if key not in index:
            index[key] = len(V)
            V.append(np.asarray(origin, dtype=np.float64) + np.asarray(key, dtype=np.float64) * h)
        return index[key]

    F, rho = [], []
    for axis in range(3):
        u, w = [a for a in range(3) if a != axis]
        for plane in range(0, int(nc[axis]) + 1):
            c = plane * subdiv
            outer = plane == 0 or plane == nc[axis]
            for i in range(int(npts[u]) - 1):
                for j in range(int(npts[w]) - 1):
                    q = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = [0, 0, 0]
                        p[axis], p[u], p[w] = c, i + di, j + dj
                        q.append(vid(p))
                    F += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
                    rho += [1.0 if outer else 2.0] * 2
    V = np.array(V)
    if jitter > 0:
        V = V + np.random.default_rng(seed).normal(0.0, jitter, size=V.shape)
    return V, np.asarray(F, dtype=np.int32), np.asarray(rho, dtype=np.float64)
