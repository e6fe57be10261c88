"""ctypes declarations of the C ABI in include/deltamic.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdeltamic.so")

c_i32, c_i64, c_f64, c_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

DM_OK = 0
STATUS = {
    0: "DM_OK",
    -1: "DM_ERR_ARG",
    -2: "DM_ERR_OOM",
    -3: "DM_ERR_DEGENERATE",
    -4: "DM_ERR_OPEN_MESH",
    -5: "DM_ERR_TIMEOUT",
    -6: "DM_ERR_CUDA",
    -7: "DM_ERR_UNSUPPORTED",
}
DM_FP64, DM_FP32_MIXED = 0, 1
DM_SURFACE, DM_VOLUME = 0, 1
LOSSES = {"l2": 0, "mse": 1, "weighted": 2}
DM_PSF_DIAG, DM_PSF_FULL = 0, 1
DM_NOALLOC_MAX_TRIANGLES = 65536
STAGES = ("params", "prep", "band", "fwd", "scatter", "c2r", "loss", "r2c", "gather", "adj", "reduce", "assemble",
          "adam", "smooth")
OPTIMIZERS = {"adam": 0, "large_steps": 1}


class dm_options(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("device", c_i32), ("no_graphs", c_i32)]


class dm_grid(ctypes.Structure):
    _fields_ = [("n", c_i32 * 3), ("h", c_f64 * 3), ("origin", c_f64 * 3)]


class dm_psf(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("sigma", c_f64 * 3), ("cov", c_f64 * 6), ("band_tau", c_f64)]


class dm_mesh(ctypes.Structure):
    _fields_ = [
        ("V", c_p),
        ("n_v", c_i64),
        ("F", c_p),
        ("n_t", c_i64),
        ("tri_weight", c_p),
        ("label", c_i32),
        ("reserved", c_i32),
    ]


class dm_fit_options(ctypes.Structure):
    _fields_ = [
        ("steps", c_i32),
        ("loss", c_i32),
        ("lr_vertex", c_f64),
        ("lr_psf", c_f64),
        ("beta1", c_f64),
        ("beta2", c_f64),
        ("eps", c_f64),
    ]


class dm_stagger_options(ctypes.Structure):
    _fields_ = [
        ("rounds", c_i32),
        ("shape_steps", c_i32),
        ("psf_steps", c_i32),
        ("shape_loss", c_i32),
        ("psf_loss", c_i32),
        ("optimizer", c_i32),
        ("lr_vertex", c_f64),
        ("lr_psf", c_f64),
        ("lam", c_f64),
        ("beta1", c_f64),
        ("beta2", c_f64),
        ("eps", c_f64),
        ("cg_tol", c_f64),
        ("cg_max_iter", c_i32),
        ("reserved", c_i32),
    ]


class dm_stagger_stats(ctypes.Structure):
    _fields_ = [("cg_iterations", c_i64), ("cg_max", c_i64), ("cg_unconverged", c_i64)]


class dm_fit_state(ctypes.Structure):
    _fields_ = [("step", c_i64), ("sigma", c_f64 * 3), ("m_sigma", c_f64 * 3), ("v_sigma", c_f64 * 3), ("m_V", c_p),
                ("v_V", c_p), ("warm", c_p)]


class dm_server_options(ctypes.Structure):
    _fields_ = [("device", c_i32), ("max_jobs", c_i32), ("memory_bytes", ctypes.c_size_t), ("chunk_tiles", c_i32),
                ("policy", c_i32), ("batch_terms", c_f64), ("max_wait_s", c_f64), ("no_graphs", c_i32)]


POLICIES = {"fifo": 0, "shortest": 1}


class dm_job(ctypes.Structure):
    _fields_ = [
        ("V", c_p),
        ("n_v", c_i64),
        ("F", c_p),
        ("n_t", c_i64),
        ("target", c_p),
        ("grid", dm_grid),
        ("psf", dm_psf),
        ("fit", dm_fit_options),
        ("label", c_i32),
        ("optimizer", c_i32),
        ("lam", c_f64),
        ("lr_decay", c_f64),
        ("tri_weight", c_p),
        ("resume", ctypes.POINTER(dm_fit_state)),
    ]


class dm_job_status(ctypes.Structure):
    _fields_ = [("state", c_i32), ("steps_done", c_i32), ("t_submit", c_f64), ("t_start", c_f64), ("t_end", c_f64),
                ("last_loss", c_f64)]


class dm_server_stats(ctypes.Structure):
    _fields_ = [("iterations", c_i64), ("jobs_done", c_i64), ("job_steps", c_i64), ("peak_active", c_i64),
                ("busy_s", c_f64), ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t),
                ("bytes_total", ctypes.c_size_t), ("graph_replays", c_i64)]


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "preempted"}


def fit_state_struct(state: dict, n_v: int, keep: list) -> "dm_fit_state":
    """A dm_fit_state over host arrays of the state dict (step, sigma, m_sigma, v_sigma, m_V, v_V, warm);
    the arrays are appended to `keep` so that they outlive the call."""
    import numpy as np

    st = dm_fit_state()
    st.step = int(state.get("step", 0))
    for a in range(3):
        st.sigma[a] = float(state["sigma"][a])
        st.m_sigma[a] = float(state.get("m_sigma", (0, 0, 0))[a])
        st.v_sigma[a] = float(state.get("v_sigma", (0, 0, 0))[a])
    for name, shape in (("m_V", (n_v, 3)), ("v_V", (n_v, 3)), ("warm", (2, n_v, 3))):
        arr = state.get(name)
        if arr is None and name == "warm":
            continue
        arr = np.ascontiguousarray(np.zeros(shape) if arr is None else arr, dtype=np.float64).reshape(shape)
        state[name] = arr
        keep.append(arr)
        setattr(st, name, arr.ctypes.data)
    return st


def fit_state_dict(st: "dm_fit_state", arrays: dict) -> dict:
    return {"step": int(st.step), "sigma": tuple(st.sigma), "m_sigma": tuple(st.m_sigma),
            "v_sigma": tuple(st.v_sigma), **arrays}

_SIGS = {
    "dm_create": (c_i32, [ctypes.POINTER(c_p), ctypes.POINTER(dm_options)]),
    "dm_destroy": (c_i32, [c_p]),
    "dm_last_error": (ctypes.c_char_p, [c_p]),
    "dm_workspace_size": (c_i32, [c_p, ctypes.POINTER(dm_grid), c_i64, c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "dm_reserve": (c_i32, [c_p, ctypes.c_size_t]),
    "dm_sync": (c_i32, [c_p, c_p]),
    "dm_check_mesh": (c_i32, [c_p, c_p]),
    "dm_kernel_launches": (c_i64, [c_p]),
    "dm_profile_enable": (c_i32, [c_p, c_i32]),
    "dm_profile_read": (c_i32, [c_p, c_p, c_p]),
    "dm_band": (c_i32, [c_p, ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p, ctypes.POINTER(c_i64), c_p]),
    "dm_meshft": (c_i32, [c_p, ctypes.POINTER(dm_mesh), ctypes.POINTER(dm_grid), c_p, c_i64, c_p, c_p]),
    "dm_meshft_adjoint": (c_i32, [c_p, ctypes.POINTER(dm_mesh), ctypes.POINTER(dm_grid), c_p, c_i64, c_p, c_p, c_p]),
    "dm_meshft_noalloc": (c_i32, [ctypes.POINTER(dm_mesh), ctypes.POINTER(dm_grid), c_p, c_i64, c_p, c_p, c_p]),
    "dm_c2r": (c_i32, [c_p, ctypes.POINTER(dm_grid), c_p, c_p, c_p]),
    "dm_r2c": (c_i32, [c_p, ctypes.POINTER(dm_grid), c_p, c_p, c_p]),
    "dm_render": (c_i32, [c_p, ctypes.POINTER(dm_mesh), ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p, c_p]),
    "dm_loss_and_grad": (
        c_i32,
        [c_p, ctypes.POINTER(dm_mesh), ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p, c_i32, c_p, c_p, c_p, c_p, c_p],
    ),
    "dm_render_adjoint": (
        c_i32,
        [c_p, ctypes.POINTER(dm_mesh), ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p, c_p, c_p, c_p],
    ),
    "dm_adam": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_i64, c_f64, c_f64, c_f64, c_f64, c_i64, c_p]),
    "dm_server_create": (c_i32, [ctypes.POINTER(c_p), ctypes.POINTER(dm_server_options)]),
    "dm_server_submit": (c_i32, [c_p, ctypes.POINTER(dm_job), ctypes.POINTER(c_i64)]),
    "dm_server_status": (c_i32, [c_p, c_i64, ctypes.POINTER(dm_job_status)]),
    "dm_server_wait": (c_i32, [c_p, c_i64, c_f64]),
    "dm_server_result": (c_i32, [c_p, c_i64, c_p, c_p, c_p]),
    "dm_server_preempt": (c_i32, [c_p, c_i64, c_f64, c_p, ctypes.POINTER(dm_fit_state)]),
    "dm_server_get_stats": (c_i32, [c_p, ctypes.POINTER(dm_server_stats)]),
    "dm_server_clock": (c_f64, [c_p]),
    "dm_server_shutdown": (c_i32, [c_p]),
    "dm_probe_wait_timeout": (c_i32, [c_i32, ctypes.c_uint64, ctypes.POINTER(c_i32)]),
    "dm_smooth_solve": (c_i32, [c_p, c_p, c_i64, c_i64, c_f64, c_p, c_p, c_f64, c_i32, c_p, c_p]),
    "dm_adam_uniform": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_i64, c_f64, c_f64, c_f64, c_f64, c_i64, c_p]),
    "dm_fit_staggered": (
        c_i32,
        [c_p, ctypes.POINTER(dm_mesh), c_p, ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p,
         ctypes.POINTER(dm_stagger_options), c_p, c_p, ctypes.POINTER(dm_stagger_stats), c_p],
    ),
    "dm_fit_resume": (
        c_i32,
        [c_p, ctypes.POINTER(dm_mesh), c_p, ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p,
         ctypes.POINTER(dm_fit_options), ctypes.POINTER(dm_fit_state), c_p, c_p],
    ),
    "dm_fit": (
        c_i32,
        [c_p, ctypes.POINTER(dm_mesh), c_p, ctypes.POINTER(dm_psf), ctypes.POINTER(dm_grid), c_p,
         ctypes.POINTER(dm_fit_options), c_p, c_p],
    ),
}

EXPORTED = tuple(_SIGS)
_LIB = None


def load():
    """Load libdeltamic.so (built in-tree by paper_2303_10440_b300/build.py); raise if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2303_10440_b300.build` "
                "(there is no CPU fallback)"
            )
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB
