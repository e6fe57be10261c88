"""The allocation-free mesh transform (dm_meshft_noalloc) agrees with dm_meshft.

dm_meshft_noalloc serves callers that may not allocate device memory once they are
running (a server that reserved all of its memory at start-up, or a framework that
owns every allocation): it takes no context and keeps its scratch in a fixed device
array. Here it is called twice in a row through the C ABI, on two different meshes
and frequency lists, and each result is compared with the context-based dm_meshft
within the FP32 spectrum tolerance of the parity tests, and the second with the FP64
oracle. The first call is the warm-up (it loads the kernels' modules and looks up the
scratch); the second must leave the device's free memory unchanged.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 2e-6  # FP32 spectrum tolerance of tests/test_gpu_parity.py (relative L2)
TOL_ORACLE = 1e-5  # FP32 spectrum against the FP64 oracle (tests/test_gpu_fullsize.py)


def _mesh_struct(_lib, V, F):
    m = _lib.dm_mesh()
    m.V = V.data_ptr()
    m.n_v = V.shape[0]
    m.F = F.data_ptr()
    m.n_t = F.shape[0]
    m.tri_weight = None
    m.label = _lib.DM_SURFACE
    return m


def _grid_struct(_lib, g):
    s = _lib.dm_grid()
    for a in range(3):
        s.n[a] = g.n[a]
        s.h[a] = g.h[a]
        s.origin[a] = g.origin[a]
    return s


def test_noalloc_matches_meshft_on_two_calls_in_a_row():
    from paper_2303_10440_b300 import Renderer, _lib

    lib = _lib.load()
    r = Renderer("fp32")
    dev = torch.device("cuda", 0)
    grid = synth.Grid(n=(32, 32, 32), h=(0.5, 0.5, 1.0), origin=(0.25, 0.0, -0.5))
    cases = [
        synth.sh_deformed_sphere(3, 5.0, grid.center, lmax=4, coef_sigma=0.4, seed=11),
        synth.sh_deformed_sphere(2, 4.0, grid.center + 0.7, lmax=3, coef_sigma=0.3, seed=12),
    ]
    rng = np.random.default_rng(3)
    # every device buffer of both calls exists before the first call, so that nothing but the library
    # could take device memory between the two calls
    bufs = []
    for k, (V, F) in enumerate(cases):
        M = 3000 + 517 * k  # ragged: not a multiple of the block size
        n = np.stack([rng.integers(-16, 16, M), rng.integers(-16, 16, M), rng.integers(0, 17, M)], axis=1)
        n[0] = 0
        bufs.append(dict(V=V, F=F, n=n.astype(np.int32), M=M, Vd=torch.as_tensor(V).to(dev),
                         Fd=torch.as_tensor(F).to(dev), nd=torch.as_tensor(n.astype(np.int32)).to(dev),
                         S=torch.empty(M, dtype=torch.complex64, device=dev),
                         flags=torch.full((1,), -1, dtype=torch.int32, device=dev)))
    g = _grid_struct(_lib, grid)
    stream = torch.cuda.current_stream().cuda_stream
    free = []
    for k, b in enumerate(bufs):
        m = _mesh_struct(_lib, b["Vd"], b["Fd"])
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info(dev)[0])
        st = lib.dm_meshft_noalloc(ctypes.byref(m), ctypes.byref(g), b["nd"].data_ptr(), b["M"], b["S"].data_ptr(),
                                   b["flags"].data_ptr(), stream)
        assert st == _lib.DM_OK
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info(dev)[0])
        assert int(b["flags"].item()) == 0
    # the second call (after the warm-up call) reserved no device memory
    assert free[3] == free[2], free
    for k, b in enumerate(bufs):
        ref = r.meshft(b["Vd"], b["Fd"], grid, b["nd"])
        err = torch.linalg.norm(b["S"] - ref) / torch.linalg.norm(ref)
        assert float(err) < TOL, (k, float(err))
    b = bufs[1]
    ref = oracle.mesh_ft(b["V"] - np.asarray(grid.origin), b["F"], oracle.wavevectors(b["n"], grid))
    err = np.linalg.norm(b["S"].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < TOL_ORACLE, err
    r.close()


def test_noalloc_rejects_meshes_beyond_its_scratch():
    from paper_2303_10440_b300 import _lib

    lib = _lib.load()
    dev = torch.device("cuda", 0)
    n_t = _lib.DM_NOALLOC_MAX_TRIANGLES + 1
    V = torch.zeros((3, 3), dtype=torch.float64, device=dev)
    F = torch.zeros((n_t, 3), dtype=torch.int32, device=dev)
    nd = torch.zeros((4, 3), dtype=torch.int32, device=dev)
    S = torch.empty(4, dtype=torch.complex64, device=dev)
    m = _mesh_struct(_lib, V, F)
    g = _grid_struct(_lib, synth.Grid(n=(8, 8, 8), h=(1.0, 1.0, 1.0)))
    st = lib.dm_meshft_noalloc(ctypes.byref(m), ctypes.byref(g), nd.data_ptr(), 4, S.data_ptr(), None, None)
    assert st == -1  # DM_ERR_ARG
