"""FP64 CPU oracle of the optimisation layer around the renderer — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this module. It shares no code with the CUDA path.

What it computes (paper section, plus the readings taken where the paper is silent):

* Staggered scheme (Section 5.1, "A staggered optimization scheme"): rounds of
  (a) shape steps — the loss on the narrow band of the current PSF, vertices
  updated, PSF held — followed by (b) PSF steps — the loss on every frequency of
  the half spectrum, PSF updated, vertices held. The shape loss is the
  target-weighted <(I - T)^2, T> (Section 5.1), the PSF loss the plain
  ||I - T||^2 (Section 5.2).
* Large-steps vertex update (Section 5.1, after Nicolet et al. 2021): the paper
  writes v <- v - eta (1 + lambda L)^-2 dL/dv with the uniform-Adam optimiser and
  lambda = 50. Reading: the optimiser acts on u = (1 + lambda L) v, whose gradient
  is (1 + lambda L)^-1 dL/dv; the uniform-Adam step Delta on u moves v by
  (1 + lambda L)^-1 Delta. With the moments switched off this is exactly the
  printed (1 + lambda L)^-2 update, scaled by one number.
* L is the combinatorial graph Laplacian of the mesh edges (degree minus
  adjacency over the unique undirected edges); this reading is the common
  default of the large-steps method and needs no geometry.
* Uniform Adam (Nicolet et al. 2021): Adam's first and second moments with bias
  correction, but every coordinate is divided by the square root of the LARGEST
  second-moment estimate, so the step keeps the direction of m_hat.
* PSF step (Section 5.2): Adam on the covariance. Reading: Sigma = C C^T with C
  lower triangular (6 numbers), which keeps Sigma positive semi-definite for
  every iterate; Adam acts on C.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import oracle as _o

# order of the 6 Cholesky numbers: C00, C11, C22, C10, C20, C21
# order of the 6 covariance numbers (as in the PSF struct): xx, yy, zz, xy, xz, yz


def edges(F) -> np.ndarray:
    """Unique undirected edges (i < j) of the triangles."""
    F = np.asarray(F, dtype=np.int64)
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e = np.sort(e, axis=1)
    e = e[e[:, 0] != e[:, 1]]
    return np.unique(e, axis=0)


def laplacian(F, n_v: int) -> sp.csr_matrix:
    """Combinatorial Laplacian L = D - A over the unique edges."""
    e = edges(F)
    A = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n_v, n_v))
    A = (A + A.T).tocsr()
    return (sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A).tocsr()


def smoothing_matrix(F, n_v: int, lam: float) -> sp.csc_matrix:
    return (sp.identity(n_v) + lam * laplacian(F, n_v)).tocsc()


def smooth_solve(F, n_v: int, lam: float, B) -> np.ndarray:
    """X = (1 + lam L)^-1 B for B of shape [n_v, 3] (sparse direct solve)."""
    B = np.asarray(B, dtype=np.float64)
    X = spla.spsolve(smoothing_matrix(F, n_v, lam), B)
    return np.asarray(X).reshape(B.shape)


def adam_uniform(g, m, v, t: int, lr: float, b1: float, b2: float, eps: float):
    """One uniform-Adam step: returns (Delta, m, v); the parameter moves by -Delta."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1**t)
    vh = v / (1.0 - b2**t)
    return lr * mh / (np.sqrt(vh.max()) + eps), m, v


def adam(g, m, v, t: int, lr: float, b1: float, b2: float, eps: float):
    """One Adam step (Kingma and Ba 2014): returns (Delta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1**t)
    vh = v / (1.0 - b2**t)
    return lr * mh / (np.sqrt(vh) + eps), m, v


def chol_matrix(c) -> np.ndarray:
    c00, c11, c22, c10, c20, c21 = c
    return np.array([[c00, 0.0, 0.0], [c10, c11, 0.0], [c20, c21, c22]])


def chol_to_cov(c) -> tuple:
    S = chol_matrix(c) @ chol_matrix(c).T
    return (S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2])


def cov_to_chol(cov) -> np.ndarray:
    xx, yy, zz, xy, xz, yz = cov
    C = np.linalg.cholesky(np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]], dtype=np.float64))
    return np.array([C[0, 0], C[1, 1], C[2, 2], C[1, 0], C[2, 0], C[2, 1]])


def chol_grad(c, gcov) -> np.ndarray:
    """dL/dC from dL/d(xx, yy, zz, xy, xz, yz), where each stored off-diagonal number stands
    for both symmetric entries: dL/dC = (G + G^T) C restricted to the lower triangle, G the
    matrix with the diagonal numbers on the diagonal and half of each off-diagonal number in
    both of its places."""
    gxx, gyy, gzz, gxy, gxz, gyz = gcov
    G = np.array([[gxx, gxy / 2, gxz / 2], [gxy / 2, gyy, gyz / 2], [gxz / 2, gyz / 2, gzz]])
    D = 2.0 * G @ chol_matrix(c)
    return np.array([D[0, 0], D[1, 1], D[2, 2], D[1, 0], D[2, 0], D[2, 1]])


def _psf_full(cov, tau):
    from synth import Psf

    return Psf(sigma=(1.0, 1.0, 1.0), band_tau=tau, cov=tuple(float(x) for x in cov))


def initial_cov(psf) -> tuple:
    return tuple(float(x) for x in (psf.cov if getattr(psf, "cov", None) is not None else
                                    (psf.sigma[0] ** 2, psf.sigma[1] ** 2, psf.sigma[2] ** 2, 0.0, 0.0, 0.0)))


def fit_staggered(V, F, grid, psf, target, rounds: int, shape_steps: int, psf_steps: int, lr_vertex: float,
                  lr_psf: float, lam: float = 50.0, optimizer: str = "large_steps", shape_loss: str = "weighted",
                  psf_loss: str = "l2", beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-20,
                  mode: str = "surface", weights=None, trace=None):
    """The staggered fit. Returns (V, cov, shape_losses, psf_losses); each loss is taken before its step.
    trace (optional list): receives, for every step, the state it started from and what it evaluated there:
    dict(kind="shape" | "psf", V, cov, L, grad) with grad = dL/dV or dL/dcov."""
    V = np.array(V, dtype=np.float64)
    n_v = V.shape[0]
    c = cov_to_chol(initial_cov(psf))
    tau = float(psf.band_tau)
    mV, vV = np.zeros_like(V), np.zeros_like(V)
    mC, vC = np.zeros(6), np.zeros(6)
    ts = tp = 0
    hs, hp = [], []
    A = smoothing_matrix(F, n_v, lam) if optimizer == "large_steps" else None
    for _ in range(rounds):
        for _ in range(shape_steps):  # (a) narrow band, PSF held
            ts += 1
            L, dV, _, _ = _o.loss_and_grad(V, F, grid, _psf_full(chol_to_cov(c), tau), target, shape_loss, mode,
                                           weights=weights)
            hs.append(L)
            if trace is not None:
                trace.append(dict(kind="shape", V=V.copy(), cov=chol_to_cov(c), L=L, grad=dV.copy()))
            if optimizer == "large_steps":
                gu = np.asarray(spla.spsolve(A, dV)).reshape(dV.shape)
                d, mV, vV = adam_uniform(gu, mV, vV, ts, lr_vertex, beta1, beta2, eps)
                V = V - np.asarray(spla.spsolve(A, d)).reshape(d.shape)
            else:
                d, mV, vV = adam(dV, mV, vV, ts, lr_vertex, beta1, beta2, eps)
                V = V - d
        for _ in range(psf_steps):  # (b) full spectrum, shape held
            tp += 1
            L, _, dcov, _ = _o.loss_and_grad(V, F, grid, _psf_full(chol_to_cov(c), 0.0), target, psf_loss, mode,
                                             weights=weights)
            hp.append(L)
            if trace is not None:
                trace.append(dict(kind="psf", V=V.copy(), cov=chol_to_cov(c), L=L, grad=np.asarray(dcov).copy()))
            d, mC, vC = adam(chol_grad(c, dcov), mC, vC, tp, lr_psf, beta1, beta2, eps)
            c = c - d
    return V, chol_to_cov(c), np.array(hs), np.array(hp)
