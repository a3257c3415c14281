"""Write the stored expected values of the full-size parity tests.

Calls only the oracle (and the seeded input generators).  Run from the repo root:

    python tests/golden/make_golden.py

film256x256x8_20steps.npz: the 256x256x8 film (h = 1/256, eps = 0.016, Q = 6.2e-4 along x,
stray field on, alpha = 1e-3, h_e = (0.02, 0, 0), dt = 0.01) from the seeded smoothed random
state, advanced 20 SGSPM steps by the FP64 oracle.  Stored: m at 4096 seeded sample cells
after 20 steps, the per-step energies, and the 1-ulp sensitivity of the oracle's own
trajectory (input perturbed by 2.2e-16 relative) at the same cells.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import scheme  # noqa: E402
from paper_2606_28113_b300 import inputs  # noqa: E402


def main():
    w = inputs.WORKLOADS["film256x256x8_fp32"]
    m0 = inputs.initial_state(w)
    p = scheme.Params(n=w["n"], h=w["h"], eps=w["eps"], Q=w["Q"], alpha=w["alpha"], dt=w["dt"], u=w["u"],
                      he=w["he"], workers=os.cpu_count())
    o = scheme.Oracle(p)
    steps = 20
    rng = np.random.default_rng(12345)
    nx, ny, nz = w["n"]
    cells = rng.choice(nx * ny * nz, size=4096, replace=False)
    m = m0.copy()
    E = [o.energy(m)]
    for _ in range(steps):
        m = o.step(m, 0.0)
        E.append(o.energy(m))
    pert = m0 * (1 + 2.2e-16 * np.random.default_rng(1).choice([-1, 1], size=m0.shape))
    mp = o.run(pert, steps)
    flat = m.reshape(3, -1)[:, cells]
    sens = np.abs(mp.reshape(3, -1)[:, cells] - flat).max()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "film256x256x8_20steps.npz")
    np.savez_compressed(out, cells=cells, m=flat, energy=np.array(E), steps=steps, ulp_sensitivity=sens)
    print(out, "sensitivity", sens)


if __name__ == "__main__":
    main()
