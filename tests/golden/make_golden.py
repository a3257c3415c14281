"""Write the stored expected values of the full-size parity tests.

Calls only the oracle (and the seeded input generators).  Run from the repo root:

    python tests/golden/make_golden.py            # both files
    python tests/golden/make_golden.py 20         # the 20-step file only
    python tests/golden/make_golden.py 1000       # the 1000-step file only (about 1.5 h on 8 cores)

Both files hold the 256x256x8 film (h = 1/256, eps = 0.016, Q = 6.2e-4 along x, stray field
on, alpha = 1e-3, h_e = (0.02, 0, 0), dt = 0.01) from the seeded smoothed random state,
advanced by the FP64 oracle:

film256x256x8_20steps.npz: m at 4096 seeded sample cells after 20 SGSPM steps, the
per-step energies, and the 1-ulp sensitivity of the oracle's own trajectory (input perturbed
by 2.2e-16 relative) at the same cells.

film256x256x8_1000steps.npz: the same after 1000 steps: m at the same 4096 cells, the five
energy terms after every step (energies[k] is the energy after k steps), and the 1-ulp
sensitivity after 1000 steps.
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import scheme  # noqa: E402
from paper_2606_28113_b300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
W = inputs.WORKLOADS["film256x256x8_fp32"]


def _oracle(workers):
    w = W
    p = scheme.Params(n=w["n"], h=w["h"], eps=w["eps"], Q=w["Q"], alpha=w["alpha"], dt=w["dt"], u=w["u"],
                      he=w["he"], workers=workers)
    return scheme.Oracle(p)


def _cells():
    nx, ny, nz = W["n"]
    return np.random.default_rng(12345).choice(nx * ny * nz, size=4096, replace=False)


def _perturbed():
    m0 = inputs.initial_state(W)
    return m0 * (1 + 2.2e-16 * np.random.default_rng(1).choice([-1, 1], size=m0.shape))


def _run(args):
    """Advance `steps` oracle steps from the seeded state (or its 1-ulp perturbation)."""
    steps, perturbed, energies, workers = args
    o = _oracle(workers)
    m = _perturbed() if perturbed else inputs.initial_state(W)
    E = [o.energy(m)] if energies else []
    for k in range(steps):
        m = o.step(m, 0.0)
        if energies:
            E.append(o.energy(m))
        if (k + 1) % 50 == 0:
            print(f"{'perturbed' if perturbed else 'main'}: {k + 1}/{steps} steps", flush=True)
    return m.reshape(3, -1)[:, _cells()], np.array(E)


def make(steps, name):
    cells = _cells()
    workers = max(1, (os.cpu_count() or 2) // 2)
    # the two trajectories are independent: run them side by side in fresh processes
    with mp.get_context("spawn").Pool(2) as pool:
        (flat, E), (pflat, _) = pool.map(_run, [(steps, False, True, workers), (steps, True, False, workers)])
    sens = np.abs(pflat - flat).max()
    out = os.path.join(HERE, name)
    np.savez_compressed(out, cells=cells, m=flat, energy=E, steps=steps, ulp_sensitivity=sens)
    print(out, "sensitivity", sens)


def main():
    which = sys.argv[1:] or ["20", "1000"]
    if "20" in which:
        make(20, "film256x256x8_20steps.npz")
    if "1000" in which:
        make(1000, "film256x256x8_1000steps.npz")


if __name__ == "__main__":
    main()
