"""The oracle still reproduces its frozen case-1 fixtures (tests/golden/oracle_case1.json)."""

import json
import os
import sys

import numpy as np

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
from make_golden import case1_target  # noqa: E402


def test_oracle_matches_frozen_case1():
    with open(os.path.join(HERE, "golden", "oracle_case1.json")) as f:
        g = json.load(f)
    case = synth.config_c1()
    T = case1_target(case)
    assert abs(np.linalg.norm(T) - g["target_l2_norm"]) < 1e-12 * g["target_l2_norm"]
    L, dV, dpsf, r = oracle.loss_and_grad(case.V_init, case.F, case.grid, case.psf, T, "mse")
    assert len(r["S"]) == g["band_size"]
    S = r["S"][g["spectrum_index"]]
    ref = np.array(g["spectrum_re"]) + 1j * np.array(g["spectrum_im"])
    assert np.max(np.abs(S - ref)) < 1e-12 * np.max(np.abs(ref))
    assert abs(r["image"].sum() - g["image_sum_times_voxel_volume"]) < 1e-12
    assert abs(L - g["loss_mse"]) < 1e-12 * g["loss_mse"]
    assert np.allclose(dV[g["dV_index"]], g["dV"], rtol=1e-10, atol=1e-14)
    assert np.allclose(dpsf, g["dsigma"], rtol=1e-10)
