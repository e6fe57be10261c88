"""Python binding of the C ABI: argument marshalling for torch tensors and numpy arrays.

Every computation runs in libdeltamic.so. Tensors on a CUDA device are passed as
device pointers; CPU tensors and numpy arrays as host pointers (the library
stages them). Outputs are allocated on the device of the vertex tensor.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass
class Grid:
    n: tuple  # voxels (Nx, Ny, Nz); images are C-ordered [x][y][z]
    h: tuple = (1.0, 1.0, 1.0)  # voxel size
    origin: tuple = (0.0, 0.0, 0.0)  # position of voxel (0, 0, 0)


@dataclass
class PSF:
    sigma: tuple = (1.0, 1.0, 1.0)  # Gaussian standard deviations (diagonal covariance)
    band_tau: float = 0.0  # narrow band: keep h_hat > tau; 0 keeps the whole half spectrum
    cov: tuple | None = None  # full covariance (xx, yy, zz, xy, xz, yz); overrides sigma


class DeltaMicError(RuntimeError):
    pass


def _grid(g) -> _lib.dm_grid:
    s = _lib.dm_grid()
    for a in range(3):
        s.n[a] = int(g.n[a])
        s.h[a] = float(g.h[a])
        s.origin[a] = float(getattr(g, "origin", (0.0, 0.0, 0.0))[a])
    return s


def _psf(p) -> _lib.dm_psf:
    s = _lib.dm_psf()
    cov = getattr(p, "cov", None)
    s.kind = _lib.DM_PSF_FULL if cov is not None else _lib.DM_PSF_DIAG
    for a in range(3):
        s.sigma[a] = float(p.sigma[a]) if getattr(p, "sigma", None) is not None else 1.0
    if cov is not None:
        for k in range(6):
            s.cov[k] = float(cov[k])
    s.band_tau = float(getattr(p, "band_tau", 0.0) or 0.0)
    return s


def _as_tensor(x, dtype, device=None):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(x)
    if device is not None:
        x = x.to(device)
    return x.to(dtype).contiguous()


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream, device) -> int | None:
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if device.type == "cuda":
        return torch.cuda.current_stream(device).cuda_stream
    return None


class Renderer:
    """A library context (one CUDA device, one precision).

    precision: "fp32" (FP32 mixed path: float images) or "fp64" (plain FP64 path).
    """

    def __init__(self, precision: str = "fp32", device: int = 0, graphs: bool = True):
        """graphs: fits replay one captured CUDA graph per optimisation step (False: enqueue each step's
        kernels one by one; the results are bitwise the same)."""
        self.lib = _lib.load()
        self.precision = precision
        self.real = torch.float32 if precision == "fp32" else torch.float64
        self.cplx = torch.complex64 if precision == "fp32" else torch.complex128
        opt = _lib.dm_options(_lib.DM_FP32_MIXED if precision == "fp32" else _lib.DM_FP64, int(device),
                              0 if graphs else 1)
        h = ctypes.c_void_p()
        st = self.lib.dm_create(ctypes.byref(h), ctypes.byref(opt))
        if st != _lib.DM_OK:
            raise DeltaMicError(f"dm_create failed: {_lib.STATUS.get(st, st)}")
        self.ctx = h
        self.device = torch.device("cuda", int(device))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != _lib.DM_OK:
            msg = self.lib.dm_last_error(self.ctx).decode(errors="replace")
            raise DeltaMicError(f"{what}: {_lib.STATUS.get(st, st)}: {msg}")

    def kernel_launches(self) -> int:
        return int(self.lib.dm_kernel_launches(self.ctx))

    def profile(self, enable: bool = True):
        """Enable or disable per-stage CUDA-event timing inside the library."""
        self._check(self.lib.dm_profile_enable(self.ctx, 1 if enable else 0), "dm_profile_enable")

    def profile_read(self) -> dict:
        """Synchronise and return {stage: (milliseconds, timed executions)} since the last read."""
        ms = (ctypes.c_double * len(_lib.STAGES))()
        calls = (ctypes.c_int64 * len(_lib.STAGES))()
        self._check(self.lib.dm_profile_read(self.ctx, ctypes.cast(ms, ctypes.c_void_p),
                                             ctypes.cast(calls, ctypes.c_void_p)), "dm_profile_read")
        return {k: (ms[i], calls[i]) for i, k in enumerate(_lib.STAGES)}

    def sync(self, stream=None):
        self._check(self.lib.dm_sync(self.ctx, _stream(stream, self.device)), "dm_sync")

    # ------------------------------------------------------------------ marshalling
    def _mesh(self, V, F, label, weights, device):
        V = _as_tensor(V, torch.float64, device)
        F = _as_tensor(F, torch.int32, device)
        W = None if weights is None else _as_tensor(weights, torch.float32, device)
        m = _lib.dm_mesh()
        m.V = V.data_ptr()
        m.n_v = V.shape[0]
        m.F = F.data_ptr()
        m.n_t = F.shape[0]
        m.tri_weight = _ptr(W)
        m.label = _lib.DM_VOLUME if label == "volume" else _lib.DM_SURFACE
        return m, (V, F, W)

    @staticmethod
    def _dev(V):
        return V.device if isinstance(V, torch.Tensor) else torch.device("cpu")

    # ------------------------------------------------------------------ renderer
    def check_mesh(self, V, F, label="surface", weights=None):
        """Debug check of a mesh (dm_check_mesh): raises DeltaMicError (DM_ERR_ARG, DM_ERR_DEGENERATE or
        DM_ERR_OPEN_MESH) for bad indices or values, a zero area / non-positive volume, or a volume-label
        mesh that is not closed and consistently oriented."""
        m, keep = self._mesh(V, F, label, weights, self._dev(V))  # host arrays stay on the host
        self._check(self.lib.dm_check_mesh(self.ctx, ctypes.byref(m)), "dm_check_mesh")

    def render(self, V, F, grid, psf, label="surface", weights=None, out=None, stream=None):
        dev = self._dev(V)
        m, keep = self._mesh(V, F, label, weights, dev)
        n = tuple(int(v) for v in grid.n)
        img = out if out is not None else torch.empty(n, dtype=self.real, device=dev)
        g, p = _grid(grid), _psf(psf)
        st = self.lib.dm_render(self.ctx, ctypes.byref(m), ctypes.byref(p), ctypes.byref(g), img.data_ptr(),
                                _stream(stream, dev))
        self._check(st, "dm_render")
        return img

    def loss_and_grad(self, V, F, grid, psf, target, loss="mse", label="surface", weights=None, want_image=False,
                      L_out=None, dV_out=None, dpsf_out=None, stream=None):
        """Returns (L, dV, dpsf, image). L is a float (or the given device tensor)."""
        dev = self._dev(V)
        m, keep = self._mesh(V, F, label, weights, dev)
        T = _as_tensor(target, self.real, dev if isinstance(target, torch.Tensor) and target.is_cuda else None)
        g, p = _grid(grid), _psf(psf)
        npsf = 6 if getattr(psf, "cov", None) is not None else 3
        dV = dV_out if dV_out is not None else torch.empty((m.n_v, 3), dtype=torch.float64, device=dev)
        dpsf = dpsf_out if dpsf_out is not None else torch.empty(npsf, dtype=torch.float64)
        Lh = L_out if L_out is not None else torch.empty(1, dtype=torch.float64)
        img = torch.empty(tuple(int(v) for v in grid.n), dtype=self.real, device=dev) if want_image else None
        st = self.lib.dm_loss_and_grad(self.ctx, ctypes.byref(m), ctypes.byref(p), ctypes.byref(g), T.data_ptr(),
                                       _lib.LOSSES[loss], Lh.data_ptr(), dV.data_ptr(), dpsf.data_ptr(), _ptr(img),
                                       _stream(stream, dev))
        self._check(st, "dm_loss_and_grad")
        L = Lh if L_out is not None else float(Lh[0])
        return L, dV, dpsf, img

    def render_adjoint(self, V, F, grid, psf, dL_dI, label="surface", weights=None, stream=None):
        dev = self._dev(V)
        m, keep = self._mesh(V, F, label, weights, dev)
        D = _as_tensor(dL_dI, self.real, dev if isinstance(dL_dI, torch.Tensor) and dL_dI.is_cuda else None)
        g, p = _grid(grid), _psf(psf)
        npsf = 6 if getattr(psf, "cov", None) is not None else 3
        dV = torch.empty((m.n_v, 3), dtype=torch.float64, device=dev)
        dpsf = torch.empty(npsf, dtype=torch.float64)
        st = self.lib.dm_render_adjoint(self.ctx, ctypes.byref(m), ctypes.byref(p), ctypes.byref(g), D.data_ptr(),
                                        dV.data_ptr(), dpsf.data_ptr(), _stream(stream, dev))
        self._check(st, "dm_render_adjoint")
        return dV, dpsf

    # ------------------------------------------------------------------ stages
    def meshft(self, V, F, grid, freq_n, label="surface", weights=None, stream=None):
        dev = self._dev(V)
        m, keep = self._mesh(V, F, label, weights, dev)
        fn = _as_tensor(freq_n, torch.int32, dev)
        S = torch.empty(fn.shape[0], dtype=self.cplx, device=dev)
        g = _grid(grid)
        st = self.lib.dm_meshft(self.ctx, ctypes.byref(m), ctypes.byref(g), fn.data_ptr(), fn.shape[0], S.data_ptr(),
                                _stream(stream, dev))
        self._check(st, "dm_meshft")
        return S

    def meshft_adjoint(self, V, F, grid, freq_n, G, label="surface", weights=None, stream=None):
        dev = self._dev(V)
        m, keep = self._mesh(V, F, label, weights, dev)
        fn = _as_tensor(freq_n, torch.int32, dev)
        Gt = _as_tensor(G, self.cplx, dev)
        dV = torch.empty((m.n_v, 3), dtype=torch.float64, device=dev)
        g = _grid(grid)
        st = self.lib.dm_meshft_adjoint(self.ctx, ctypes.byref(m), ctypes.byref(g), fn.data_ptr(), fn.shape[0],
                                        Gt.data_ptr(), dV.data_ptr(), _stream(stream, dev))
        self._check(st, "dm_meshft_adjoint")
        return dV

    def c2r(self, grid, spec, stream=None):
        dev = spec.device if isinstance(spec, torch.Tensor) else torch.device("cpu")
        X = _as_tensor(spec, self.cplx, dev)
        out = torch.empty(tuple(int(v) for v in grid.n), dtype=self.real, device=dev)
        g = _grid(grid)
        self._check(self.lib.dm_c2r(self.ctx, ctypes.byref(g), X.data_ptr(), out.data_ptr(), _stream(stream, dev)),
                    "dm_c2r")
        return out

    def r2c(self, grid, image, stream=None):
        dev = image.device if isinstance(image, torch.Tensor) else torch.device("cpu")
        I = _as_tensor(image, self.real, dev)
        n = tuple(int(v) for v in grid.n)
        out = torch.empty((n[0], n[1], n[2] // 2 + 1), dtype=self.cplx, device=dev)
        g = _grid(grid)
        self._check(self.lib.dm_r2c(self.ctx, ctypes.byref(g), I.data_ptr(), out.data_ptr(), _stream(stream, dev)),
                    "dm_r2c")
        return out

    def band(self, grid, psf, stream=None):
        g, p = _grid(grid), _psf(psf)
        n = tuple(int(v) for v in grid.n)
        idx = torch.empty(n[0] * n[1] * (n[2] // 2 + 1), dtype=torch.int32)
        M = ctypes.c_int64()
        st = self.lib.dm_band(self.ctx, ctypes.byref(p), ctypes.byref(g), idx.data_ptr(), ctypes.byref(M),
                              _stream(stream, self.device))
        self._check(st, "dm_band")
        return idx[: M.value].clone()

    # ------------------------------------------------------------------ optimisation
    def adam(self, param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-20, stream=None):
        st = self.lib.dm_adam(self.ctx, param.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), param.numel(),
                              lr, beta1, beta2, eps, int(step), _stream(stream, param.device))
        self._check(st, "dm_adam")

    def fit_resume(self, V, F, grid, psf, target, steps, lr_vertex, state=None, lr_psf=0.0, loss="mse",
                   label="surface", weights=None, beta1=0.9, beta2=0.999, eps=1e-20, stream=None):
        """dm_fit continued from a checkpoint. state: None (a fresh start from psf.sigma) or the dict
        returned by an earlier call (step, sigma, Adam moments). Returns (V, sigma, loss_history, state);
        a fit of a + b steps equals a fit of a steps and a resumed fit of b steps, bit for bit."""
        dev = self._dev(V)
        Vw = _as_tensor(V, torch.float64, dev).clone()
        m, keep = self._mesh(Vw, F, label, weights, dev)
        T = _as_tensor(target, self.real, dev if isinstance(target, torch.Tensor) and target.is_cuda else None)
        g, p = _grid(grid), _psf(psf)
        if state is None:
            state = {"step": 0, "sigma": tuple(p.sigma)}
        state = dict(state)
        arrays = []
        st = _lib.fit_state_struct(state, m.n_v, arrays)
        o = _lib.dm_fit_options(int(steps), _lib.LOSSES[loss], float(lr_vertex), float(lr_psf), beta1, beta2, eps)
        hist = torch.empty(int(steps), dtype=torch.float64)
        rc = self.lib.dm_fit_resume(self.ctx, ctypes.byref(m), Vw.data_ptr(), ctypes.byref(p), ctypes.byref(g),
                                    T.data_ptr(), ctypes.byref(o), ctypes.byref(st), hist.data_ptr(),
                                    _stream(stream, dev))
        self._check(rc, "dm_fit_resume")
        new_state = _lib.fit_state_dict(st, {"m_V": state["m_V"].copy(), "v_V": state["v_V"].copy()})
        return Vw, tuple(p.sigma), hist, new_state

    def smooth_solve(self, F, n_v, B, lam=50.0, X0=None, tol=0.0, max_iter=0, stream=None):
        """X = (1 + lam L)^-1 B for B [n_v, 3] (device), L the combinatorial mesh Laplacian.
        Returns (X, (total iterations, most in one column, unconverged columns))."""
        dev = B.device
        Bt = _as_tensor(B, torch.float64, dev)
        X = torch.zeros_like(Bt) if X0 is None else _as_tensor(X0, torch.float64, dev).clone()
        Ft = _as_tensor(F, torch.int32, dev)
        it = (ctypes.c_int64 * 3)()
        st = self.lib.dm_smooth_solve(self.ctx, Ft.data_ptr(), Ft.shape[0], int(n_v), float(lam), Bt.data_ptr(),
                                      X.data_ptr(), float(tol), int(max_iter), it, _stream(stream, dev))
        self._check(st, "dm_smooth_solve")
        return X, tuple(int(v) for v in it)

    def adam_uniform(self, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-20, stream=None):
        """One uniform-Adam step; m, v updated in place; returns delta (the parameter moves by -delta)."""
        delta = torch.empty_like(grad)
        st = self.lib.dm_adam_uniform(self.ctx, grad.data_ptr(), m.data_ptr(), v.data_ptr(), delta.data_ptr(),
                                      grad.numel(), lr, beta1, beta2, eps, int(step), _stream(stream, grad.device))
        self._check(st, "dm_adam_uniform")
        return delta

    def fit_staggered(self, V, F, grid, psf, target, rounds, shape_steps, psf_steps, lr_vertex, lr_psf,
                      optimizer="large_steps", lam=50.0, shape_loss="weighted", psf_loss="l2", label="surface",
                      weights=None, beta1=0.9, beta2=0.999, eps=1e-20, cg_tol=0.0, cg_max_iter=0, stream=None):
        """Staggered shape/PSF fit on the device (shape steps on the narrow band, PSF steps on the
        whole half spectrum). Returns (V_fitted, PSF with the fitted covariance, shape losses,
        PSF losses, smoothing-solve statistics)."""
        dev = self._dev(V)
        Vw = _as_tensor(V, torch.float64, dev).clone()
        m, keep = self._mesh(Vw, F, label, weights, dev)
        T = _as_tensor(target, self.real, dev if isinstance(target, torch.Tensor) and target.is_cuda else None)
        g, p = _grid(grid), _psf(psf)
        o = _lib.dm_stagger_options(int(rounds), int(shape_steps), int(psf_steps), _lib.LOSSES[shape_loss],
                                    _lib.LOSSES[psf_loss], _lib.OPTIMIZERS[optimizer], float(lr_vertex), float(lr_psf),
                                    float(lam), beta1, beta2, eps, float(cg_tol), int(cg_max_iter), 0)
        hs = torch.empty(max(1, rounds * shape_steps), dtype=torch.float64)
        hp = torch.empty(max(1, rounds * psf_steps), dtype=torch.float64)
        stats = _lib.dm_stagger_stats()
        st = self.lib.dm_fit_staggered(self.ctx, ctypes.byref(m), Vw.data_ptr(), ctypes.byref(p), ctypes.byref(g),
                                       T.data_ptr(), ctypes.byref(o), hs.data_ptr(), hp.data_ptr(), ctypes.byref(stats),
                                       _stream(stream, dev))
        self._check(st, "dm_fit_staggered")
        out_psf = PSF(sigma=tuple(p.sigma), band_tau=p.band_tau, cov=tuple(p.cov))
        cg = dict(iterations=stats.cg_iterations, max=stats.cg_max, unconverged=stats.cg_unconverged)
        return Vw, out_psf, hs[: rounds * shape_steps], hp[: rounds * psf_steps], cg

    def fit(self, V, F, grid, psf, target, steps, lr_vertex, lr_psf=0.0, loss="mse", label="surface", weights=None,
            beta1=0.9, beta2=0.999, eps=1e-20, stream=None):
        """Adam fit on the device. Returns (V_fitted, sigma_fitted, loss_history).

        eps defaults to 1e-20: rendered images have unit total intensity, so MSE gradients are
        ~1e-10 and the usual 1e-8 would dominate sqrt(v) and shrink every step.
        """
        dev = self._dev(V)
        Vw = _as_tensor(V, torch.float64, dev).clone()
        m, keep = self._mesh(Vw, F, label, weights, dev)
        T = _as_tensor(target, self.real, dev if isinstance(target, torch.Tensor) and target.is_cuda else None)
        g, p = _grid(grid), _psf(psf)
        o = _lib.dm_fit_options(int(steps), _lib.LOSSES[loss], float(lr_vertex), float(lr_psf), beta1, beta2, eps)
        hist = torch.empty(int(steps), dtype=torch.float64)
        st = self.lib.dm_fit(self.ctx, ctypes.byref(m), Vw.data_ptr(), ctypes.byref(p), ctypes.byref(g), T.data_ptr(),
                             ctypes.byref(o), hist.data_ptr(), _stream(stream, dev))
        self._check(st, "dm_fit")
        return Vw, tuple(p.sigma), hist
