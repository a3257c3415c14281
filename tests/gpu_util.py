"""Helpers shared by the GPU tests: run the same seeded workload on the oracle and on
the CUDA path (through the C ABI) and compare element by element."""
import numpy as np

from oracle import scheme
from paper_2606_28113_b300 import sgspm


def oracle_run(m0, n, h, eps, Q, alpha, dt, steps, u=(1.0, 0.0, 0.0), he=(0.0, 0.0, 0.0), stray=True,
               sch="sgspm", refresh="R1", forcing=None, energies=False):
    p = scheme.Params(n=n, h=h, eps=eps, Q=Q, alpha=alpha, dt=dt, u=u, he=he, stray=stray, scheme=sch,
                      refresh=refresh, forcing=forcing)
    o = scheme.Oracle(p)
    m = m0.copy()
    E = [o.energy(m)] if energies else None
    t = 0.0
    for _ in range(steps):
        m = o.step(m, t)
        t += dt
        if energies:
            E.append(o.energy(m))
    return (m, o, np.array(E)) if energies else (m, o)


def gpu_handle(n, h, eps, Q, alpha, dt, u=(1.0, 0.0, 0.0), he=(0.0, 0.0, 0.0), fp64=True, **kw):
    return sgspm.film(n, h, eps, Q, alpha, dt, u=u, he=he, fp64=fp64, **kw)


def gpu_run(m0, steps, chunk=None, energies=False, **kw):
    H = gpu_handle(**kw)
    H.set_m(m0)
    E = [H.energy()[0]] if energies else None
    if energies:
        for _ in range(steps):
            H.step(1)
            E.append(H.energy()[0])
    elif steps:
        H.step(steps)
    m = H.split(H.get_m())[0]
    H.close()
    return (m, np.array(E)) if energies else m


def oracle_response(m0, ref, steps, rel, seed=1, **kw):
    """How far the oracle's own trajectory (ref after `steps` steps from m0) moves when its input
    is perturbed by `rel` relative, with a random sign per entry."""
    rng = np.random.default_rng(seed)
    b, _ = oracle_run(m0 * (1 + rel * rng.choice([-1, 1], size=m0.shape)), steps=steps, **kw)
    return float(np.abs(b - ref).max())


def oracle_noise_response(m0, ref, steps, rel, seed=2, n=None, h=None, eps=None, Q=None, alpha=None, dt=None,
                          u=(1.0, 0.0, 0.0), he=(0.0, 0.0, 0.0)):
    """How far the oracle's trajectory moves when its state is perturbed by `rel` relative (random
    sign per entry) after every step: the response to rounding of that size made in every step."""
    o = scheme.Oracle(scheme.Params(n=n, h=h, eps=eps, Q=Q, alpha=alpha, dt=dt, u=u, he=he))
    rng = np.random.default_rng(seed)
    m = m0.copy()
    t = 0.0
    for _ in range(steps):
        m = o.step(m, t)
        t += dt
        m = m * (1 + rel * rng.choice([-1, 1], size=m.shape))
    return float(np.abs(m - ref).max())
