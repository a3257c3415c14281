"""SGSPM and GSPM time steps, effective field and discrete energy (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

Model (Sec. 2, Eq. (1)): m_t = -m x h_eff - alpha m x (m x h_eff),
    h_eff = eps Delta m - Q (m2 e2 + m3 e3) + h_s + h_e,   Neumann BC (Eq. (2)).

The step follows Sec. 3.2 (SGSPM) and Sec. 3.1 (GSPM) in the paper's order and
notation, with
    g_i = (I - eps dt Delta_h)^{-1} (m_i + dt f_i),   f = -Q(m2 e2 + m3 e3) + h_s + h_e.

Readings of points the paper leaves open:
  * Delta_h: cell-centred 7-point Laplacian with mirror ghosts (oracle/heat.py).
  * When f is evaluated for a g_i^*: at the newest state each time a g is formed
    ("R1", default), so h_s is refreshed at every intermediate state (the remark
    after the GSPM projection step says h_s uses the intermediate m).  "R2" freezes
    h_s at m^n for Step 1 and uses h_s(m**) for Step 2.
  * Easy axis: the paper's -Q(m2 e2 + m3 e3) is the uniaxial term with axis e1;
    it is written -Q(m - (m.u)u), which equals the paper's term for u = e1.
  * Stray field: h_s = -N * m with the Newell tensor, zero-padded (oracle/demag.py).
  * Manufactured forcing f_e (Sec. 5.1) enters as an explicit source added after
    the damping heat flow and before the projection: m*** += dt f_e(x, t_n).
  * Energy: E = eps/2 int |grad m|^2 + Q/2 int (m2^2+m3^2) - 1/2 int h_s.m - int h_e.m,
    the normalisation for which h_eff = -dE/dm holds (the printed E of Sec. 2 lacks
    the factors 1/2; with them the discrete gradient is exactly -V h_eff).

Fields are [3, nz, ny, nx]; component index 0, 1, 2 is the paper's 1, 2, 3.
"""
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import demag, heat


@dataclass
class Params:
    n: tuple                      # (nx, ny, nz) cells
    h: tuple                      # (hx, hy, hz) cell size
    eps: float
    Q: float
    alpha: float
    dt: float
    u: tuple = (1.0, 0.0, 0.0)    # easy axis
    he: object = (0.0, 0.0, 0.0)  # uniform (3,) or per cell (3, nz, ny, nx)
    stray: bool = True
    scheme: str = "sgspm"         # "sgspm" (Sec. 3.2) or "gspm" (Sec. 3.1)
    refresh: str = "R1"           # "R1" newest state for every f, "R2" frozen per step
    forcing: Optional[Callable] = None   # f_e(t) -> (3, nz, ny, nx), Sec. 5.1
    workers: Optional[int] = None


class Oracle:
    def __init__(self, p: Params):
        self.p = p
        u = np.asarray(p.u, dtype=np.float64)
        self.u = u / np.linalg.norm(u)
        he = np.asarray(p.he, dtype=np.float64)
        nx, ny, nz = p.n
        self.he = he.reshape(3, 1, 1, 1) if he.shape == (3,) else he.reshape(3, nz, ny, nx)
        self.H = demag.StrayOperator(p.n, p.h, workers=p.workers) if p.stray else None
        self.stray_evals = 0

    # ---- fields --------------------------------------------------------------------
    def h_s(self, m):
        if self.H is None:
            return np.zeros_like(m)
        self.stray_evals += 1
        return self.H(m)

    def f(self, m, hs):
        """f = -Q(m - (m.u)u) + h_s + h_e (Sec. 3.1, Step 2; anisotropy per reading above)."""
        mu = np.einsum("a...,a->...", m, self.u)
        anis = -self.p.Q * (m - mu[None] * self.u.reshape(3, 1, 1, 1))
        return anis + hs + self.he

    def S(self, r, c):
        """(I - c dt Delta_h)^{-1} r."""
        return heat.heat_solve(r, c * self.p.dt, self.p.h, workers=self.p.workers)

    def h_eff(self, m):
        lap = np.stack([heat.laplacian(m[a], self.p.h) for a in range(3)])
        return self.p.eps * lap + self.f(m, self.h_s(m))

    # ---- one time step ---------------------------------------------------------------
    def step(self, m, t):
        if self.p.scheme == "sgspm":
            mss, hs_frozen = self._step1_sgspm(m)
        elif self.p.scheme == "gspm":
            mss, hs_frozen = self._step1_gspm(m)
        else:
            raise ValueError(self.p.scheme)
        return self._step2_and_projection(mss, t)

    def _fi(self, state, i, hs_frozen):
        """Component i of f at `state` (R1: h_s(state); R2: the frozen h_s(m^n))."""
        hs = self.h_s(state) if self.p.refresh == "R1" else hs_frozen
        return self.f(state, hs)[i]

    def _step1_sgspm(self, m):
        """Sec. 3.2, Step 1: forward sweep m1* -> m2* -> m3*, backward m3** -> m2** -> m1**."""
        eps, dt = self.p.eps, self.p.dt
        m1, m2, m3 = m
        hs_n = self.h_s(m)
        fn = self.f(m, hs_n)
        g2n = self.S(m2 + dt * fn[1], eps)
        g3n = self.S(m3 + dt * fn[2], eps)
        # forward sweep
        m1s = m1 + (g2n * m3 - g3n * m2)
        g1s = self.S(m1s + dt * self._fi(np.stack([m1s, m2, m3]), 0, hs_n), eps)
        m2s = m2 + (g3n * m1s - g1s * m3)
        g2s = self.S(m2s + dt * self._fi(np.stack([m1s, m2s, m3]), 1, hs_n), eps)
        m3s = m3 + (g1s * m2s - g2s * m1s)
        # backward sweep
        m3ss = m3 + (g1s * m2s - g2s * m1s)
        g3ss = self.S(m3ss + dt * self._fi(np.stack([m1s, m2s, m3ss]), 2, hs_n), eps)
        m2ss = m2 + (g3ss * m1s - g1s * m3ss)
        g2ss = self.S(m2ss + dt * self._fi(np.stack([m1s, m2ss, m3ss]), 1, hs_n), eps)
        m1ss = m1 + (g2ss * m3ss - g3ss * m2ss)
        self.last_intermediates = dict(g2n=g2n, g3n=g3n, m1s=m1s, g1s=g1s, m2s=m2s, g2s=g2s,
                                       m3s=m3s, m3ss=m3ss, g3ss=g3ss, m2ss=m2ss, g2ss=g2ss, m1ss=m1ss)
        return np.stack([m1ss, m2ss, m3ss]), hs_n

    def _step1_gspm(self, m):
        """Sec. 3.1, Step 1: one forward sweep m1* -> m2* -> m3*."""
        eps, dt = self.p.eps, self.p.dt
        m1, m2, m3 = m
        hs_n = self.h_s(m)
        fn = self.f(m, hs_n)
        g2n = self.S(m2 + dt * fn[1], eps)
        g3n = self.S(m3 + dt * fn[2], eps)
        m1s = m1 + (g2n * m3 - g3n * m2)
        g1s = self.S(m1s + dt * self._fi(np.stack([m1s, m2, m3]), 0, hs_n), eps)
        m2s = m2 + (g3n * m1s - g1s * m3)
        g2s = self.S(m2s + dt * self._fi(np.stack([m1s, m2s, m3]), 1, hs_n), eps)
        m3s = m3 + (g1s * m2s - g2s * m1s)
        return np.stack([m1s, m2s, m3s]), hs_n

    def _step2_and_projection(self, mss, t):
        """Step 2 heat flow (I - alpha eps dt Delta_h) m*** = m** + alpha dt f**, then Step 3."""
        eps, dt, alpha = self.p.eps, self.p.dt, self.p.alpha
        fss = self.f(mss, self.h_s(mss))
        msss = np.stack([self.S(mss[i] + alpha * dt * fss[i], alpha * eps) for i in range(3)])
        if self.p.forcing is not None:
            msss = msss + dt * self.p.forcing(t)
        norm = np.sqrt(np.sum(msss * msss, axis=0))
        return msss / norm[None]

    def run(self, m, nsteps, t0=0.0):
        t = t0
        for _ in range(nsteps):
            m = self.step(m, t)
            t += self.p.dt
        return m

    # ---- energy -------------------------------------------------------------------------
    def energy(self, m):
        """[exchange, anisotropy, stray, zeeman, total] of the discrete energy (reading above).

        exchange   = V eps/2 sum over interior faces |m_c - m_c'|^2 / h_a^2
        anisotropy = V Q/2 sum_c (|m_c|^2 - (m_c.u)^2)
        stray      = -V/2 sum_c h_s,c . m_c
        zeeman     = -V sum_c h_e,c . m_c
        """
        hx, hy, hz = self.p.h
        V = hx * hy * hz
        ex = 0.0
        for axis, ha in zip((3, 2, 1), (hx, hy, hz)):
            d = np.diff(m, axis=axis)
            ex += np.sum(d * d) / ha ** 2
        ex *= 0.5 * self.p.eps * V
        mu = np.einsum("a...,a->...", m, self.u)
        an = 0.5 * self.p.Q * V * np.sum(np.sum(m * m, axis=0) - mu * mu)
        st = -0.5 * V * np.sum(self.h_s(m) * m)
        ze = -V * np.sum(self.he * m)
        return np.array([ex, an, st, ze, ex + an + st + ze])


# ---- manufactured solutions of Sec. 5.1 -------------------------------------------------------
def _X(x):
    return x * x * (1 - x) ** 2


def _dX(x):
    return 2 * x * (1 - x) * (1 - 2 * x)


def _d2X(x):
    return 2 * (1 - 6 * x + 6 * x * x)


def cell_centres(n, h):
    nx, ny, nz = n
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h[2], (np.arange(ny) + 0.5) * h[1],
                          (np.arange(nx) + 0.5) * h[0], indexing="ij")
    return x, y, z


def _phase(x, y, z, dim):
    """Phi with m_e = (cos Phi sin t, sin Phi sin t, cos t); returns Phi, |grad Phi|^2, Lap Phi."""
    if dim == 1:
        return _X(x), _dX(x) ** 2, _d2X(x)
    X, Y, Z = _X(x), _X(y), _X(z)
    dX, dY, dZ = _dX(x), _dX(y), _dX(z)
    phi = X * Y * Z
    grad2 = (dX * Y * Z) ** 2 + (X * dY * Z) ** 2 + (X * Y * dZ) ** 2
    lap = _d2X(x) * Y * Z + X * _d2X(y) * Z + X * Y * _d2X(z)
    return phi, grad2, lap


def manufactured_m(n, h, t, dim):
    """Exact solution m_e of Sec. 5.1 at the cell centres (1D: x only; 3D: XYZ)."""
    x, y, z = cell_centres(n, h)
    phi, _, _ = _phase(x, y, z, dim)
    st = np.sin(t)
    return np.stack([np.cos(phi) * st, np.sin(phi) * st, np.full_like(phi, np.cos(t))])


def manufactured_forcing(n, h, alpha, dim):
    """f_e(t) = d_t m_e + m_e x Lap m_e + alpha m_e x (m_e x Lap m_e) (Sec. 5.1), exact Laplacian."""
    x, y, z = cell_centres(n, h)
    phi, grad2, lapphi = _phase(x, y, z, dim)
    c, s = np.cos(phi), np.sin(phi)

    def fe(t):
        st, ct = np.sin(t), np.cos(t)
        me = np.stack([c * st, s * st, np.full_like(c, ct)])
        dtm = np.stack([c * ct, s * ct, np.full_like(c, -st)])
        lap = np.stack([(-s * lapphi - c * grad2) * st, (c * lapphi - s * grad2) * st, np.zeros_like(c)])
        mxl = np.cross(me, lap, axis=0)
        return dtm + mxl + alpha * np.cross(me, mxl, axis=0)
    return fe
