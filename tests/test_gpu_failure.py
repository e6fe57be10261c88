"""Failure detection on the GPU without a fault: a bounded device wait that nothing completes expires,
is reported through the device error flag, and the context keeps working."""

import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_context_stays_usable():
    from paper_2303_10440_b300 import Renderer, _lib

    lib = _lib.load()
    status = ctypes.c_int32(99)
    assert lib.dm_probe_wait_timeout(0, 1_000_000, ctypes.byref(status)) == 0  # 1 ms limit
    assert status.value == -5  # DM_ERR_TIMEOUT
    # the device still renders correctly afterwards
    r = Renderer("fp32")
    grid = synth.Grid(n=(16, 16, 16), h=(1.0, 1.0, 1.0))
    V, F = synth.sphere_mesh(2, 4.0, grid.center)
    img = r.render(torch.as_tensor(V).cuda(), torch.as_tensor(F).cuda(), grid, synth.Psf(sigma=(1.0, 1.0, 1.0)))
    assert abs(float(img.sum()) * np.prod(grid.h) - 1.0) < 1e-4
    r.close()
