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
          "adam")


class dm_options(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("device", c_i32), ("deterministic", c_i32), ("reserved", c_i32)]


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


_SIGS = {
    "dm_create": (c_i32, [ctypes.POINTER(c_p), ctypes.POINTER(dm_options)]),
    "dm_destroy": (c_i32, [c_p]),
    "dm_last_error": (ctypes.c_char_p, [c_p]),
    "dm_workspace_size": (c_i32, [c_p, ctypes.POINTER(dm_grid), c_i64, c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "dm_reserve": (c_i32, [c_p, ctypes.c_size_t]),
    "dm_sync": (c_i32, [c_p, c_p]),
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
