"""Host-side mesh validation (dm_check_mesh without a context): the checks behind DM_ERR_ARG,
DM_ERR_DEGENERATE and DM_ERR_OPEN_MESH, on host arrays, without a GPU."""

import ctypes

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def check():
    from paper_2303_10440_b300 import _lib

    lib = _lib.load()

    def run(V, F, label="surface", W=None):
        V = np.ascontiguousarray(V, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.int32)
        m = _lib.dm_mesh()
        m.V, m.n_v, m.F, m.n_t = V.ctypes.data, V.shape[0], F.ctypes.data, F.shape[0]
        if W is not None:
            W = np.ascontiguousarray(W, dtype=np.float32)
            m.tri_weight = W.ctypes.data
        m.label = _lib.DM_VOLUME if label == "volume" else _lib.DM_SURFACE
        return _lib.STATUS.get(lib.dm_check_mesh(None, ctypes.byref(m)), "?")

    return run


def test_closed_meshes_pass(check):
    V, F = synth.sphere_mesh(2, 3.0, (1.0, 2.0, 3.0))
    assert check(V, F, "surface") == "DM_OK"
    assert check(V, F, "volume") == "DM_OK"
    Vb, Fb = synth.box_mesh((0, 0, 0), (2, 3, 4))
    assert check(Vb, Fb, "volume") == "DM_OK"


def test_open_or_misoriented_volume_meshes_are_refused(check):
    V, F = synth.sphere_mesh(2, 3.0, (0.0, 0.0, 0.0))
    assert check(V, F[:-1], "surface") == "DM_OK"  # an open surface is a valid surface
    assert check(V, F[:-1], "volume") == "DM_ERR_OPEN_MESH"
    flipped = F.copy()
    flipped[5] = flipped[5, ::-1]
    assert check(V, flipped, "volume") == "DM_ERR_OPEN_MESH"
    doubled = np.concatenate([F, F[:1]])  # a face used twice
    assert check(V, doubled, "volume") == "DM_ERR_OPEN_MESH"


def test_degenerate_meshes_are_refused(check):
    V, F = synth.sphere_mesh(1, 2.0, (0.0, 0.0, 0.0))
    assert check(V, F[:, ::-1], "volume") == "DM_ERR_DEGENERATE"  # inward: negative volume
    flat = np.repeat(V[:1], len(V), axis=0)
    assert check(flat, F, "surface") == "DM_ERR_DEGENERATE"
    assert check(V, F, "surface", W=np.zeros(len(F))) == "DM_ERR_DEGENERATE"
    # a single zero-area triangle among others is legal
    F2 = np.concatenate([F, [[0, 0, 1]]])
    assert check(V, F2, "surface") == "DM_OK"


def test_bad_values_are_refused(check):
    V, F = synth.sphere_mesh(1, 2.0, (0.0, 0.0, 0.0))
    bad = F.copy()
    bad[3, 2] = len(V)
    assert check(V, bad) == "DM_ERR_ARG"
    bad[3, 2] = -1
    assert check(V, bad) == "DM_ERR_ARG"
    Vn = V.copy()
    Vn[4, 1] = np.nan
    assert check(Vn, F) == "DM_ERR_ARG"
    assert check(V, F, "surface", W=np.full(len(F), -1.0)) == "DM_ERR_ARG"
    assert check(V, F, "volume", W=np.ones(len(F))) == "DM_ERR_ARG"
