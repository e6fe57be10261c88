"""FP64 CPU oracle of the renderer's hot path — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module. It shares no code with the CUDA path.

Definitions (paper section / equation, plus the readings this project takes
where the paper is silent or garbled):

* Surface density and its transform, Eq. 3-5: u_hat(xi) = S(xi) / |Lambda|,
  S(xi) = sum_T int_T exp(-i x.xi) dS (closed form Eq. 7-8, see meshft_oracle.c).
  Volume-labelled mode: S(xi) = int_V exp(-i x.xi) dV, normalised by the
  enclosed volume.
* Gaussian PSF, Eq. 2, with transfer function h_hat(xi) = exp(-1/2 xi^T Sigma xi)
  (Sigma is the spatial covariance; the printed Sigma^-1 in the transfer
  function is a typo — the Fourier transform of Eq. 2 has Sigma).
  Diagonal Sigma = diag(sigma^2) unless a full covariance is given.
* Image, Eq. 1 evaluated in Fourier space (I_hat = u_hat h_hat): on the periodic
  box of size L = N h, voxel j at x_j = origin + j h, wavevectors xi_n = 2 pi n / L
  with n on the half spectrum H = {n_x in fftfreq(N_x), n_y in fftfreq(N_y),
  n_z in 0..floor(N_z/2)} (n_z = N_z/2 is +Nyquist), Hermitian weight c_n = 1 on
  the self-conjugate planes n_z = 0 and (even N_z) n_z = N_z/2, else 2:
      I_j = (1 / (L_x L_y L_z)) sum_{n in B} c_n Re( I_hat_n exp(i xi_n . x_j) ),
  B the narrow band {n in H : h_hat(xi_n) > tau} (tau = 0 keeps all of H;
  Section 5.1 narrow band). Sum_j I_j V_vox = 1 when 0 is in B (Eq. 3's
  unit total intensity).
* Losses, Section 5.1-5.2: sum-L2 ||I - T||^2, MSE (the same divided by the voxel
  count) and the target-weighted <(I - T)^2, T>.
* Gradients: exact derivatives of the above. dL/dv by Eq. 6 (quotient rule
  through |Lambda|) with the per-triangle derivative of Eq. 9-10; dL/dsigma by
  the chain rule through h_hat.

The inverse transform uses numpy's FFT (a library primitive) on a full-grid
array, or a direct double sum over B for tiny grids (``method="dft"``).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.POINTER(ctypes.c_int32)
        L.oracle_dd.argtypes = [d, ctypes.c_int, d, d]
        L.oracle_tri_ft.argtypes = [d, d, d, d, d, d]
        L.oracle_tri_grad.argtypes = [d, d, d, d, d]
        L.oracle_mesh_ft.argtypes = [ctypes.c_int, d, ctypes.c_int64, i32, ctypes.c_int64, d, ctypes.c_int64, d, d, d]
        L.oracle_mesh_ft_adjoint.argtypes = [
            ctypes.c_int, d, ctypes.c_int64, i32, ctypes.c_int64, d, ctypes.c_int64, d, d, d, d,
        ]
        L.oracle_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ----------------------------------------------------------------------------- triangle level


def dd(nodes, m: int) -> complex:
    """Divided difference of order m of F(x) = -exp(-i x) over m+1 nodes."""
    z = np.ascontiguousarray(nodes, dtype=np.float64)
    assert z.size == m + 1
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().oracle_dd(_dp(z), m, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def tri_ft(v1, v2, v3, xi) -> complex:
    """Eq. 7-8: int_T exp(-i x.xi) dS."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (v1, v2, v3, xi)]
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().oracle_tri_ft(*[_dp(x) for x in a], ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def tri_grad(v1, v2, v3, xi) -> np.ndarray:
    """Eq. 9-10: d u_T / d v_p, shape (3 vertices, 3 axes) complex."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (v1, v2, v3, xi)]
    out = np.zeros(18, dtype=np.float64)
    lib().oracle_tri_grad(*[_dp(x) for x in a], _dp(out))
    out = out.reshape(3, 3, 2)
    return out[..., 0] + 1j * out[..., 1]


# ----------------------------------------------------------------------------- mesh level

_MODES = {"surface": 0, "volume": 1}


def _wp(weights, n_t):
    if weights is None:
        return None, None
    w = np.ascontiguousarray(weights, dtype=np.float64)
    assert w.shape == (n_t,)
    return w, _dp(w)


def mesh_ft(V, F, xi, mode: str = "surface", c0=None, weights=None) -> np.ndarray:
    """S(xi_m) = sum over triangles rho_T u_T (surface; rho = weights or 1) or signed tetrahedra about c0 (volume)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    xi = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
    c0 = np.ascontiguousarray(np.zeros(3) if c0 is None else c0, dtype=np.float64)
    w, wp = _wp(weights, F.shape[0])
    out = np.zeros((xi.shape[0], 2), dtype=np.float64)
    lib().oracle_mesh_ft(_MODES[mode], _dp(V), V.shape[0], _ip(F), F.shape[0], _dp(xi), xi.shape[0], _dp(c0), wp,
                         _dp(out))
    return out[:, 0] + 1j * out[:, 1]


def mesh_ft_adjoint(V, F, xi, Gs, mode: str = "surface", c0=None, weights=None) -> np.ndarray:
    """dV[v] = sum_m Re(conj(Gs_m) dS(xi_m)/dv)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    xi = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
    G = np.ascontiguousarray(np.stack([np.real(Gs), np.imag(Gs)], axis=1), dtype=np.float64)
    c0 = np.ascontiguousarray(np.zeros(3) if c0 is None else c0, dtype=np.float64)
    w, wp = _wp(weights, F.shape[0])
    out = np.zeros((V.shape[0], 3), dtype=np.float64)
    lib().oracle_mesh_ft_adjoint(
        _MODES[mode], _dp(V), V.shape[0], _ip(F), F.shape[0], _dp(xi), xi.shape[0], _dp(G), _dp(c0), wp, _dp(out)
    )
    return out


def surface_area(V, F, weights=None) -> float:
    """|Lambda| = sum_T rho_T A_T, A_T = |e3 x e1| / 2 (Section 4.1.2; rho = weights or 1)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    A = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    return float(np.sum(A if weights is None else np.asarray(weights) * A))


def surface_area_grad(V, F, weights=None) -> np.ndarray:
    """d|Lambda|/dv = sum over incident triangles of rho_T (-w_p / 2) = rho_T (N x e_p) / 2."""
    v = [V[F[:, k]] for k in range(3)]
    e = [v[2] - v[1], v[0] - v[2], v[1] - v[0]]  # e1, e2, e3
    n = np.cross(e[2], e[0])
    nn = np.linalg.norm(n, axis=1, keepdims=True)
    N = np.divide(n, nn, out=np.zeros_like(n), where=nn > 0)
    rho = np.ones((F.shape[0], 1)) if weights is None else np.asarray(weights, dtype=np.float64)[:, None]
    out = np.zeros_like(V)
    for p in range(3):
        np.add.at(out, F[:, p], 0.5 * rho * np.cross(N, e[p]))
    return out


def enclosed_volume(V, F) -> float:
    """Signed volume of a closed, outward-oriented mesh: sum_T v1 . (v2 x v3) / 6."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def enclosed_volume_grad(V, F) -> np.ndarray:
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    out = np.zeros_like(V)
    np.add.at(out, F[:, 0], np.cross(b, c) / 6.0)
    np.add.at(out, F[:, 1], np.cross(c, a) / 6.0)
    np.add.at(out, F[:, 2], np.cross(a, b) / 6.0)
    return out


# ----------------------------------------------------------------------------- spectral grid


def half_spectrum(n):
    """Integer frequencies of H in C order over (Nx, Ny, Nz//2+1) and their weights c_n."""
    nx, ny, nz = (int(v) for v in n)
    fx = np.fft.fftfreq(nx, d=1.0 / nx).round().astype(np.int64)
    fy = np.fft.fftfreq(ny, d=1.0 / ny).round().astype(np.int64)
    fz = np.arange(nz // 2 + 1, dtype=np.int64)
    gx, gy, gz = np.meshgrid(fx, fy, fz, indexing="ij")
    nvec = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    c = np.full(nvec.shape[0], 2.0)
    c[nvec[:, 2] == 0] = 1.0
    if nz % 2 == 0:
        c[nvec[:, 2] == nz // 2] = 1.0
    return nvec, c


def wavevectors(nvec, grid) -> np.ndarray:
    return 2.0 * np.pi * nvec.astype(np.float64) / grid.L[None, :]


def covariance(psf) -> np.ndarray:
    if getattr(psf, "cov", None) is not None:
        xx, yy, zz, xy, xz, yz = psf.cov
        return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]], dtype=np.float64)
    s = np.asarray(psf.sigma, dtype=np.float64)
    return np.diag(s * s)


def otf(xi, psf) -> np.ndarray:
    """h_hat(xi) = exp(-1/2 xi^T Sigma xi)."""
    S = covariance(psf)
    return np.exp(-0.5 * np.einsum("mi,ij,mj->m", xi, S, xi))


def band_mask(h_hat, tau: float) -> np.ndarray:
    """Section 5.1 narrow band: keep h_hat > tau * max h_hat (max = h_hat(0) = 1); tau = 0 keeps all."""
    if tau <= 0:
        return np.ones(h_hat.shape, dtype=bool)
    return h_hat > tau


def spectrum_to_image(X, nvec, c, grid, method: str = "fft") -> np.ndarray:
    """I_j = (1/(Lx Ly Lz)) sum_n c_n Re(X_n exp(i xi_n . (j h)))  (X already holds the origin phase)."""
    n = tuple(int(v) for v in grid.n)
    VL = float(np.prod(grid.L))
    if method == "dft":
        jx, jy, jz = np.meshgrid(*[np.arange(k) for k in n], indexing="ij")
        img = np.zeros(n, dtype=np.float64)
        for (a, b, d), w, x in zip(nvec, c, X):
            ph = 2 * np.pi * (a * jx / n[0] + b * jy / n[1] + d * jz / n[2])
            img += w * np.real(x * np.exp(1j * ph))
        return img / VL
    Z = np.zeros(n, dtype=np.complex128)
    Z[nvec[:, 0] % n[0], nvec[:, 1] % n[1], nvec[:, 2] % n[2]] = c * X
    return np.real(np.fft.ifftn(Z)) * (np.prod(n) / VL)


def image_adjoint(R, nvec, c, grid) -> np.ndarray:
    """G_n = dL/dRe X_n + i dL/dIm X_n = c_n/(Lx Ly Lz) * sum_j R_j exp(-i xi_n . (j h))."""
    n = tuple(int(v) for v in grid.n)
    VL = float(np.prod(grid.L))
    FR = np.fft.fftn(R)
    return c * FR[nvec[:, 0] % n[0], nvec[:, 1] % n[1], nvec[:, 2] % n[2]] / VL


# ----------------------------------------------------------------------------- render / loss / grad


def _normaliser(Vs, F, mode, weights=None):
    return surface_area(Vs, F, weights) if mode == "surface" else enclosed_volume(Vs, F)


def render(V, F, grid, psf, mode: str = "surface", method: str = "fft", weights=None):
    """Image of the mesh under the PSF; returns a dict with the image and intermediates.

    weights: optional per-triangle fluorophore density rho_T (surface mode; Section 3.3 — cell-cell
    interfaces carry density 2); the density is normalised by sum_T rho_T A_T."""
    if weights is not None and mode != "surface":
        raise ValueError("weights apply to the surface-labelled mode")
    Vs = np.asarray(V, dtype=np.float64) - np.asarray(grid.origin, dtype=np.float64)[None, :]
    nvec, c = half_spectrum(grid.n)
    xi_all = wavevectors(nvec, grid)
    h_all = otf(xi_all, psf)
    B = band_mask(h_all, psf.band_tau)
    nvec, c, xi, h = nvec[B], c[B], xi_all[B], h_all[B]
    c0 = 0.5 * grid.L
    S = mesh_ft(Vs, F, xi, mode, c0, weights)
    norm = _normaliser(Vs, F, mode, weights)
    u = S / norm
    X = u * h
    img = spectrum_to_image(X, nvec, c, grid, method)
    return dict(image=img, S=S, u=u, X=X, nvec=nvec, c=c, xi=xi, h=h, norm=norm, band=B, c0=c0, Vs=Vs,
                weights=weights)


_LOSS = {"l2": 0, "mse": 1, "weighted": 2}


def loss_value(I, T, kind: str) -> tuple[float, np.ndarray]:
    """Loss and dL/dI. l2: sum (I-T)^2; mse: mean (I-T)^2; weighted: sum T (I-T)^2."""
    d = I - T
    if kind == "l2":
        return float(np.sum(d * d)), 2.0 * d
    if kind == "mse":
        return float(np.mean(d * d)), 2.0 * d / d.size
    if kind == "weighted":
        return float(np.sum(T * d * d)), 2.0 * T * d
    raise ValueError(kind)


def render_adjoint(V, F, grid, psf, dL_dI, mode: str = "surface", fwd=None, weights=None):
    """Given dL/dI, return (dL/dV, dL/dsigma [3] or dL/dcov [6]) through the whole chain."""
    r = fwd if fwd is not None else render(V, F, grid, psf, mode, weights=weights)
    Vs, nvec, c, xi, h, S, u, X, norm, c0 = (r[k] for k in ("Vs", "nvec", "c", "xi", "h", "S", "u", "X", "norm", "c0"))
    G = image_adjoint(dL_dI, nvec, c, grid)  # dL/dX on the band
    # PSF: X = u h_hat, d h_hat / d Sigma_ab = -1/2 xi_a xi_b h_hat
    gx = np.real(np.conj(G) * X)
    if getattr(psf, "cov", None) is not None:
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        dpsf = np.array([np.sum(gx * (-0.5 * xi[:, a] * xi[:, b] * (1.0 if a == b else 2.0))) for a, b in pairs])
    else:
        s = np.asarray(psf.sigma, dtype=np.float64)
        dpsf = np.array([np.sum(gx * (-s[a] * xi[:, a] ** 2)) for a in range(3)])
    # mesh: u = S / norm (Eq. 6 quotient rule)
    Gu = G * h  # dL/du
    w = r.get("weights")
    dV_S = mesh_ft_adjoint(Vs, F, xi, Gu / norm, mode, c0, w)
    cq = float(np.sum(np.real(np.conj(Gu) * S))) / norm**2
    dnorm = surface_area_grad(Vs, F, w) if mode == "surface" else enclosed_volume_grad(Vs, F)
    dV = dV_S - cq * dnorm
    return dV, dpsf


def loss_and_grad(V, F, grid, psf, target, kind: str = "mse", mode: str = "surface", weights=None):
    r = render(V, F, grid, psf, mode, weights=weights)
    L, dI = loss_value(r["image"], target, kind)
    dV, dpsf = render_adjoint(V, F, grid, psf, dI, mode, fwd=r)
    return L, dV, dpsf, r
