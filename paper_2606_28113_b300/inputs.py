"""Seeded synthetic inputs and workload definitions (shared by tests, bench and smoke).

This module holds no arithmetic of the method: it only draws seeded initial states
and names the workloads.  Fields are float64 arrays [3, nz, ny, nx] (x fastest).
"""
import numpy as np


def random_unit(seed, n):
    """i.i.d. Gaussian 3-vectors normalised to unit length, one per cell."""
    nx, ny, nz = n
    m = np.random.default_rng(seed).normal(size=(3, nz, ny, nx))
    return m / np.linalg.norm(m, axis=0)


def smoothed_random_unit(seed, n, sigma_cells=(20.5, 20.5, 20.5)):
    """Random unit vectors smoothed, then renormalised.

    The smoothing is a Gaussian filter (mirror boundaries) whose width equals the
    diffusion length of 20 implicit heat steps at the run's parameters,
    sqrt(2 * 20 * eps * dt) / h = sqrt(40 * 0.016 * 0.01) * 256 = 20.5 cells.
    """
    from scipy.ndimage import gaussian_filter
    m = random_unit(seed, n)
    sig = (sigma_cells[2], sigma_cells[1], sigma_cells[0])     # (z, y, x) axes of [nz, ny, nx]
    m = np.stack([gaussian_filter(m[a], sigma=sig, mode="reflect") for a in range(3)])
    return m / np.linalg.norm(m, axis=0)


def neel_wall(n, width_cells=4.0, x0_cells=None):
    """180-degree Neel wall m = (tanh((x-x0)/w), sech((x-x0)/w), 0), x in cell units."""
    nx, ny, nz = n
    x0 = nx / 2.0 if x0_cells is None else x0_cells
    xc = np.arange(nx) + 0.5
    s = (xc - x0) / width_cells
    m = np.zeros((3, nz, ny, nx))
    m[0] = np.tanh(s)
    m[1] = 1.0 / np.cosh(s)
    return m / np.linalg.norm(m, axis=0)


def cosine_profile(n, h):
    """The paper's exchange-test initial state (cos(cos pi x) sin .01, sin(cos pi x) sin .01, cos .01)."""
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) * h[0]
    x = np.broadcast_to(x, (nz, ny, nx))
    return np.stack([np.cos(np.cos(np.pi * x)) * np.sin(0.01), np.sin(np.cos(np.pi * x)) * np.sin(0.01),
                     np.full((nz, ny, nx), np.cos(0.01))])


# Workloads (names describe the film; parameters are nondimensional).
WORKLOADS = {
    "film32x32x4_fp64": dict(n=(32, 32, 4), h=(1 / 32,) * 3, eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01,
                             u=(1.0, 0.0, 0.0), he=(0.0, 0.0, 0.0), steps=200, init="random_unit", seed=0),
    "film256x256x8_fp32": dict(n=(256, 256, 8), h=(1 / 256,) * 3, eps=0.016, Q=6.2e-4, alpha=1e-3, dt=0.01,
                               u=(1.0, 0.0, 0.0), he=(0.02, 0.0, 0.0), steps=10000, init="smoothed", seed=0),
    "strip512x64x4_wall": dict(n=(512, 64, 4), h=(0.1,) * 3, eps=0.016, Q=0.1, alpha=1e-3, dt=0.005,
                               u=(1.0, 0.0, 0.0), he=(0.005, 0.0, 0.0), steps=20000, init="neel", seed=0),
    "film128x128x4_adjoint": dict(n=(128, 128, 4), h=(1 / 128,) * 3, eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01,
                                  u=(1.0, 0.0, 0.0), he=(0.0, 0.0, 0.0), steps=500, init="random_unit", seed=0),
}

ENSEMBLE_SIZES = ((64, 64, 2), (96, 64, 2), (128, 128, 4), (128, 64, 4))


def ensemble(seed=0, nfilm=256):
    """Films of uneven size for the batched workload: sizes, alpha, applied field along x."""
    rng = np.random.default_rng(seed)
    films = []
    for f in range(nfilm):
        n = ENSEMBLE_SIZES[rng.integers(len(ENSEMBLE_SIZES))]
        alpha = float(np.exp(rng.uniform(np.log(1e-4), np.log(5e-2))))
        hx = float(rng.uniform(-0.05, 0.05))
        films.append(dict(n=n, h=(1.0 / n[0],) * 3, eps=0.016, Q=6.2e-4, alpha=alpha, dt=0.01,
                          u=(1.0, 0.0, 0.0), he=(hx, 0.0, 0.0), seed=seed * 100003 + f))
    return films


def initial_state(w):
    if w["init"] == "random_unit":
        return random_unit(w["seed"], w["n"])
    if w["init"] == "smoothed":
        return smoothed_random_unit(w["seed"], w["n"])
    if w["init"] == "neel":
        return neel_wall(w["n"])
    raise ValueError(w["init"])
