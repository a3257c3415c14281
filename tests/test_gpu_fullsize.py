"""Full-size parity of the 256x256x8 film (the benchmark workload), in the launch
configuration bench.py times (single film, CUDA graph).  Needs a B300.

Sampled outputs: m at 4096 seeded cells after 20 steps and the energies are compared with
stored oracle values (tests/golden/make_golden.py writes them from the oracle only).
Long horizon: the FP32 form is compared with the FP64 form after 1000 steps, within 10x
of how far the FP64 trajectory itself moves under an FP32-sized input perturbation.
"""
import os

import numpy as np
import pytest

from paper_2606_28113_b300 import inputs, sgspm

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "film256x256x8_20steps.npz")
W = inputs.WORKLOADS["film256x256x8_fp32"]


def handle(fp64):
    return sgspm.film(W["n"], W["h"], W["eps"], W["Q"], W["alpha"], W["dt"], u=W["u"], he=W["he"], fp64=fp64)


@pytest.mark.parametrize("fp64,tol_m,tol_e", [(True, 1e-12, 1e-12), (False, 1e-5, 1e-5)])
def test_film256x256x8_sampled_cells_match_oracle(fp64, tol_m, tol_e):
    g = np.load(GOLD)
    m0 = inputs.initial_state(W)
    H = handle(fp64)
    H.set_m(m0)
    E0 = H.energy()[0]
    H.step(int(g["steps"]))
    m = H.get_m().reshape(3, -1)[:, g["cells"]]
    E = H.energy()[0]
    H.close()
    tol = max(tol_m, 10 * float(g["ulp_sensitivity"]))
    assert np.abs(m - g["m"]).max() <= tol
    assert np.abs(E0 - g["energy"][0]).max() <= tol_e * np.abs(g["energy"][0]).max()
    assert np.abs(E - g["energy"][-1]).max() <= tol_e * np.abs(g["energy"][-1]).max()


def test_film256x256x8_fp32_vs_fp64_after_1000_steps():
    m0 = inputs.initial_state(W)
    steps = 1000
    rng = np.random.default_rng(3)
    out = {}
    for name, fp64, start in (("f32", False, m0), ("f64", True, m0),
                              ("f64p", True, m0 * (1 + 6e-8 * rng.choice([-1, 1], size=m0.shape)))):
        H = handle(fp64)
        H.set_m(start)
        H.step(steps)
        out[name] = H.get_m()
        H.close()
    err = np.abs(out["f32"] - out["f64"]).max()
    sens = np.abs(out["f64p"] - out["f64"]).max()
    print(f"fp32 vs fp64 after {steps} steps: {err:.3e}; fp64 response to 6e-8 input noise: {sens:.3e}")
    assert err <= max(1e-5, 10 * sens)
