"""The C-ABI library builds, loads without a GPU, and exports every entry point include/deltamic.h declares."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "deltamic.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_10440_b300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dm_render", "dm_loss_and_grad", "dm_render_adjoint", "dm_meshft", "dm_meshft_adjoint",
                     "dm_c2r", "dm_r2c", "dm_band", "dm_create", "dm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_the_header(lib):
    from paper_2303_10440_b300 import _lib

    assert set(_lib.EXPORTED) == set(_declared())


def test_struct_layouts_match_the_header():
    from paper_2303_10440_b300 import _lib

    # natural C alignment: int32 n[3] is padded to 16 bytes before the doubles
    assert ctypes.sizeof(_lib.dm_grid) == 16 + 48
    assert ctypes.sizeof(_lib.dm_psf) == 8 + 24 + 48 + 8
    assert ctypes.sizeof(_lib.dm_mesh) == 48
    assert ctypes.sizeof(_lib.dm_options) == 12
    assert ctypes.sizeof(_lib.dm_fit_options) == 8 + 40
    assert ctypes.sizeof(_lib.dm_stagger_options) == 24 + 56 + 8
    assert ctypes.sizeof(_lib.dm_stagger_stats) == 24
    assert ctypes.sizeof(_lib.dm_job) == 40 + 64 + 88 + 48 + 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(_lib.dm_fit_state) == 8 + 72 + 24
    assert ctypes.sizeof(_lib.dm_server_options) == 4 + 4 + 8 + 4 + 4 + 8 + 8 + 8  # no_graphs + padding
    assert ctypes.sizeof(_lib.dm_server_stats) == 4 * 8 + 8 + 3 * 8 + 8
