"""The SGSPM step (Sec. 3.2) written with plain torch FP64 ops, for reference gradients.

Test infrastructure only (see oracle/__init__.py).  Same readings as oracle/scheme.py (g-form of
the paper, f refreshed at the newest state, mirror-ghost Laplacian, Newell stray field), but
every operation is a differentiable torch op so that autograd gives d(loss)/d(h_e, alpha):

  * heat solve: orthonormal DCT-II matrices along x, y, z (dense, small grids), diagonal scale;
  * stray field: zero-padded torch.fft.rfftn / irfftn with the Newell tensor of oracle/newell.py;
  * Laplacian: replicate-padded second differences.

Fields are [3, nz, ny, nx] float64 tensors.
"""
import math

import numpy as np
import torch

from . import demag, heat


def dct_matrix(n):
    """Orthonormal DCT-II matrix C (C @ x = DCT-II of x), float64."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    C = np.cos(np.pi * k * (2 * j + 1) / (2 * n)) * math.sqrt(2.0 / n)
    C[0] /= math.sqrt(2.0)
    return torch.tensor(C, dtype=torch.float64)


class TorchSGSPM:
    def __init__(self, n, h, eps, Q, dt, u=(1.0, 0.0, 0.0), stray=True):
        self.n, self.h = tuple(n), tuple(h)
        self.eps, self.Q, self.dt = eps, Q, dt
        uu = np.asarray(u, dtype=np.float64)
        self.u = torch.tensor(uu / np.linalg.norm(uu), dtype=torch.float64)
        nx, ny, nz = n
        self.Cx, self.Cy, self.Cz = dct_matrix(nx), dct_matrix(ny), dct_matrix(nz)
        self.lam = torch.tensor(heat.eigenvalues(n, h), dtype=torch.float64)     # [nz, ny, nx]
        self.stray = stray
        if stray:
            op = demag.StrayOperator(n, h)
            self.P = op.P
            self.Khat = torch.tensor(op.Khat)                                      # complex128 [6, ...]
            self.idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4,
                        (1, 2): 5, (2, 1): 5}

    # ---- operators ----------------------------------------------------------------------------
    def S(self, r, c_dt):
        """(I - c_dt Delta_h)^{-1} r for a scalar field r[nz, ny, nx]."""
        rh = torch.einsum("ax,zyx->zya", self.Cx, r)
        rh = torch.einsum("by,zya->zba", self.Cy, rh)
        rh = torch.einsum("cz,zba->cba", self.Cz, rh)
        rh = rh / (1.0 + c_dt * self.lam)
        g = torch.einsum("cz,cba->zba", self.Cz, rh)
        g = torch.einsum("by,zba->zya", self.Cy, g)
        return torch.einsum("ax,zya->zyx", self.Cx, g)

    def h_s(self, m):
        if not self.stray:
            return torch.zeros_like(m)
        nx, ny, nz = self.n
        M = torch.fft.rfftn(m, s=self.P, dim=(1, 2, 3))
        out = []
        for a in range(3):
            acc = sum(self.Khat[self.idx[(a, b)]] * M[b] for b in range(3))
            out.append(-torch.fft.irfftn(acc, s=self.P, dim=(0, 1, 2))[:nz, :ny, :nx])
        return torch.stack(out)

    def f(self, m, he):
        mu = torch.einsum("a...,a->...", m, self.u)
        anis = -self.Q * (m - mu[None] * self.u.view(3, 1, 1, 1))
        return anis + self.h_s(m) + he

    # ---- one SGSPM step (Sec. 3.2), literal g-form --------------------------------------------
    def step(self, m, he, alpha):
        eps, dt = self.eps, self.dt
        m1, m2, m3 = m[0], m[1], m[2]
        fn = self.f(m, he)
        g2n = self.S(m2 + dt * fn[1], eps * dt)
        g3n = self.S(m3 + dt * fn[2], eps * dt)
        m1s = m1 + (g2n * m3 - g3n * m2)
        g1s = self.S(m1s + dt * self.f(torch.stack([m1s, m2, m3]), he)[0], eps * dt)
        m2s = m2 + (g3n * m1s - g1s * m3)
        g2s = self.S(m2s + dt * self.f(torch.stack([m1s, m2s, m3]), he)[1], eps * dt)
        m3s = m3 + (g1s * m2s - g2s * m1s)
        g3ss = self.S(m3s + dt * self.f(torch.stack([m1s, m2s, m3s]), he)[2], eps * dt)
        m2ss = m2 + (g3ss * m1s - g1s * m3s)
        g2ss = self.S(m2ss + dt * self.f(torch.stack([m1s, m2ss, m3s]), he)[1], eps * dt)
        m1ss = m1 + (g2ss * m3s - g3ss * m2ss)
        mss = torch.stack([m1ss, m2ss, m3s])
        fss = self.f(mss, he)
        msss = torch.stack([self.S(mss[i] + alpha * dt * fss[i], alpha * eps * dt) for i in range(3)])
        return msss / torch.sqrt(torch.sum(msss * msss, dim=0, keepdim=True))

    def run(self, m, he, alpha, steps):
        for _ in range(steps):
            m = self.step(m, he, alpha)
        return m


def loss(mT, he, reg=1e-3):
    """mean over cells of (m_x(T) - 1)^2 + reg * ||h_e||^2 (squared L2 over all 3n entries)."""
    return torch.mean((mT[0] - 1.0) ** 2) + reg * torch.sum(he * he)


def reference_gradients(model, m0, he, alpha, steps, reg=1e-3):
    """d loss / d h_e (per cell, [3, nz, ny, nx]) and d loss / d alpha by autograd."""
    he_t = torch.tensor(np.asarray(he, dtype=np.float64).copy(), requires_grad=True)
    a_t = torch.tensor(float(alpha), dtype=torch.float64, requires_grad=True)
    mT = model.run(torch.tensor(m0, dtype=torch.float64), he_t, a_t, steps)
    L = loss(mT, he_t, reg)
    L.backward()
    return float(L.detach()), he_t.grad.numpy().copy(), float(a_t.grad)
