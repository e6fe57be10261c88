"""Write oracle regression fixtures for the 32^3 icosphere case (case 1).

The paper prints no worked numeric example, so these fixtures are produced by
the FP64 oracle alone (this script imports only ``oracle`` and ``synth``). They
freeze the oracle: a later change to its arithmetic must regenerate them in a
commit that names the passage of the paper justifying the change.

Run from the repository root:  python tests/golden/make_golden.py
"""

from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def case1_target(case):
    img = oracle.render(case.V_true, case.F, case.grid, case.psf)["image"]
    return synth.add_gaussian_noise(img, case.noise["rel_sigma"], case.noise["seed"])


def main():
    case = synth.config_c1()
    T = case1_target(case)
    L, dV, dpsf, r = oracle.loss_and_grad(case.V_init, case.F, case.grid, case.psf, T, "mse")
    rng = np.random.default_rng(1234)
    sel = np.sort(rng.choice(len(r["S"]), size=48, replace=False))
    vsel = np.sort(rng.choice(case.V_init.shape[0], size=16, replace=False))
    out = {
        "source": "oracle (FP64 CPU), case 1: icosphere level 2, R=10, 32^3, h=1, sigma=(1,1,2.5), full spectrum, MSE",
        "band_size": int(len(r["S"])),
        "area": r["norm"],
        "spectrum_index": sel.tolist(),
        "spectrum_re": np.real(r["S"][sel]).tolist(),
        "spectrum_im": np.imag(r["S"][sel]).tolist(),
        "image_sum_times_voxel_volume": float(r["image"].sum()),
        "image_max": float(r["image"].max()),
        "target_l2_norm": float(np.linalg.norm(T)),
        "loss_mse": L,
        "dV_index": vsel.tolist(),
        "dV": dV[vsel].tolist(),
        "dsigma": dpsf.tolist(),
    }
    with open(os.path.join(HERE, "oracle_case1.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote oracle_case1.json", L)


if __name__ == "__main__":
    main()
