"""Python front end of the continuous-batching fit server (dm_server_* in include/deltamic.h).

The engine (admission, device arena, batched persistent launches) runs in the library's own
thread; this module only copies job inputs into the C structs and reads results back.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from .api import _grid, _psf


@dataclass
class JobResult:
    job_id: int
    V: np.ndarray
    sigma: tuple
    loss_history: np.ndarray
    t_submit: float
    t_start: float
    t_end: float

    @property
    def latency(self) -> float:
        return self.t_end - self.t_submit


class FitServer:
    """Continuous-batching shape-fit server on one GPU (FP32 mixed path)."""

    def __init__(self, device: int = 0, max_jobs: int = 32, memory_bytes: int = 0, chunk_tiles: int = 0,
                 policy: str = "fifo", batch_terms: float = 0.0, max_wait_s: float = 0.0, graphs: bool = True):
        """policy "fifo": arrival order, every resident job advances every iteration; "shortest": the
        jobs with the least remaining work are admitted and advanced first, at most ``batch_terms``
        triangle-frequency terms per iteration (<= 0: no limit), a job idle for ``max_wait_s`` first.
        graphs: replay an iteration captured as a CUDA graph while the set of advanced jobs is unchanged."""
        self.lib = _lib.load()
        o = _lib.dm_server_options(int(device), int(max_jobs), int(memory_bytes), int(chunk_tiles),
                                   _lib.POLICIES[policy], float(batch_terms), float(max_wait_s), 0 if graphs else 1)
        h = ctypes.c_void_p()
        st = self.lib.dm_server_create(ctypes.byref(h), ctypes.byref(o))
        if st != _lib.DM_OK:
            raise RuntimeError(f"dm_server_create: {_lib.STATUS.get(st, st)}")
        self.h = h
        self._meta = {}

    def clock(self) -> float:
        return float(self.lib.dm_server_clock(self.h))

    def submit(self, V, F, target, grid, psf, steps: int, lr_vertex: float, lr_psf: float = 0.0, loss: str = "mse",
               label: str = "surface", beta1=0.9, beta2=0.999, eps=1e-20, optimizer: str = "adam",
               lam: float = 50.0, resume: dict | None = None, lr_decay: float = 1.0, weights=None) -> int:
        """resume: the state dict of a preempted job (see preempt); V is then that job's vertices and
        steps the steps still to take. lr_decay: step t uses lr * lr_decay^(t-1) (t continues across
        resume). weights: per-triangle densities (surface label), or None for 1."""
        V = np.ascontiguousarray(V, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.int32)
        T = np.ascontiguousarray(target, dtype=np.float32)
        j = _lib.dm_job()
        j.V = V.ctypes.data
        j.n_v = V.shape[0]
        j.F = F.ctypes.data
        j.n_t = F.shape[0]
        j.target = T.ctypes.data
        j.grid = _grid(grid)
        j.psf = _psf(psf)
        j.fit = _lib.dm_fit_options(int(steps), _lib.LOSSES[loss], float(lr_vertex), float(lr_psf), beta1, beta2, eps)
        j.label = _lib.DM_VOLUME if label == "volume" else _lib.DM_SURFACE
        j.optimizer = _lib.OPTIMIZERS[optimizer]
        j.lam = float(lam)
        j.lr_decay = float(lr_decay)
        keep = []
        if weights is not None:
            W = np.ascontiguousarray(weights, dtype=np.float32)
            if W.shape != (F.shape[0],):
                raise ValueError("weights: one value per triangle")
            keep.append(W)
            j.tri_weight = W.ctypes.data
        if resume is not None:
            st = _lib.fit_state_struct(dict(resume), V.shape[0], keep)
            keep.append(st)
            j.resume = ctypes.pointer(st)
        jid = ctypes.c_int64()
        st = self.lib.dm_server_submit(self.h, ctypes.byref(j), ctypes.byref(jid))  # copies every input
        if st != _lib.DM_OK:
            raise RuntimeError(f"dm_server_submit: {_lib.STATUS.get(st, st)}")
        self._meta[jid.value] = (V.shape[0], int(steps))
        return jid.value

    def preempt(self, job_id: int, timeout: float = -1.0):
        """Stop a queued or running job at the next iteration boundary. Returns (V, state) to resubmit with
        ``submit(..., V=V, steps=<remaining>, resume=state)``, or None if the job finished first."""
        n_v, _ = self._meta[job_id]
        V = np.empty((n_v, 3))
        arrays = {"m_V": np.empty((n_v, 3)), "v_V": np.empty((n_v, 3)), "warm": np.zeros((2, n_v, 3))}
        st = _lib.dm_fit_state()
        st.m_V, st.v_V, st.warm = (arrays[k].ctypes.data for k in ("m_V", "v_V", "warm"))
        rc = self.lib.dm_server_preempt(self.h, job_id, float(timeout), V.ctypes.data, ctypes.byref(st))
        if rc == -1:  # DM_ERR_ARG: finished first (or unknown)
            return None
        if rc != _lib.DM_OK:
            raise RuntimeError(f"dm_server_preempt: {_lib.STATUS.get(rc, rc)}")
        self._meta.pop(job_id, None)
        return V, _lib.fit_state_dict(st, arrays)

    def status(self, job_id: int) -> dict:
        s = _lib.dm_job_status()
        st = self.lib.dm_server_status(self.h, job_id, ctypes.byref(s))
        if st != _lib.DM_OK:
            raise KeyError(job_id)
        return dict(state=_lib.JOB_STATES.get(s.state, s.state), steps_done=s.steps_done, t_submit=s.t_submit,
                    t_start=s.t_start, t_end=s.t_end, last_loss=s.last_loss)

    def wait(self, job_id: int, timeout: float = -1.0) -> bool:
        st = self.lib.dm_server_wait(self.h, job_id, float(timeout))
        if st == -5:  # DM_ERR_TIMEOUT
            return False
        if st != _lib.DM_OK:
            raise RuntimeError(f"job {job_id} failed: {_lib.STATUS.get(st, st)}")
        return True

    def result(self, job_id: int) -> JobResult:
        n_v, steps = self._meta.pop(job_id)
        s = self.status(job_id)
        V = np.empty((n_v, 3))
        sig = np.empty(3)
        hist = np.empty(steps)
        st = self.lib.dm_server_result(self.h, job_id, V.ctypes.data, sig.ctypes.data, hist.ctypes.data)
        if st != _lib.DM_OK:
            raise RuntimeError(f"dm_server_result: {_lib.STATUS.get(st, st)}")
        return JobResult(job_id, V, tuple(sig), hist, s["t_submit"], s["t_start"], s["t_end"])

    def stats(self) -> dict:
        s = _lib.dm_server_stats()
        self.lib.dm_server_get_stats(self.h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def shutdown(self):
        if getattr(self, "h", None):
            self.lib.dm_server_shutdown(self.h)
            self.h = None

    def __del__(self):
        try:
            self.shutdown()
        except Exception:
            pass
