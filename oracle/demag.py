"""Stray field h_s = -N * m on a cell grid (oracle, FP64).  Test infrastructure only.

The paper computes h_s "by FFT" (Sec. 1; Sec. 5.1 after Table 5) and evaluates it at
the intermediate magnetisation (Sec. 3.1, remark after the projection step).  Here
the convolution with the Newell tensor (oracle/newell.py) is written two ways:

* `stray_fft`: the aperiodic convolution computed exactly by zero padding every
  axis of length n > 1 to 2n and multiplying spectra (numpy real FFTs).
* `stray_direct`: the defining double sum h_a(i) = -sum_j sum_b N_ab(i - j) m_b(j),
  O(n^2), for tiny grids.

Fields are [3, nz, ny, nx] (component, z, y, x; x fastest).
"""
import numpy as np
import scipy.fft as sfft

from . import newell

_IDX = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}


def _padded_kernel(Nfull, n):
    """Place N(offset) on the periodic padded grid: offset o -> index o mod P."""
    nx, ny, nz = n
    P = tuple(2 * a if a > 1 else 1 for a in (nz, ny, nx))
    K = np.zeros((6,) + P)
    kk = np.arange(-(nz - 1), nz) % P[0]
    jj = np.arange(-(ny - 1), ny) % P[1]
    ii = np.arange(-(nx - 1), nx) % P[2]
    K[:, kk[:, None, None], jj[None, :, None], ii[None, None, :]] = Nfull
    return K, P


class StrayOperator:
    """h_s(m) for a fixed grid: holds the Newell tensor and its padded spectra."""

    def __init__(self, n, h, workers=None):
        self.n = tuple(n)
        self.h = tuple(h)
        self.N = newell.demag_tensor(self.n, self.h)
        K, self.P = _padded_kernel(self.N, self.n)
        self.Khat = sfft.rfftn(K, axes=(1, 2, 3), workers=workers)
        self.workers = workers

    def __call__(self, m):
        nx, ny, nz = self.n
        Mhat = sfft.rfftn(m, s=self.P, axes=(1, 2, 3), workers=self.workers)
        h = np.empty_like(m)
        for a in range(3):
            acc = 0.0
            for b in range(3):
                acc = acc + self.Khat[_IDX[(a, b)]] * Mhat[b]
            full = sfft.irfftn(acc, s=self.P, axes=(0, 1, 2), workers=self.workers)
            h[a] = -full[:nz, :ny, :nx]
        return h

    def component(self, m, a):
        """Only h_s component a (the cost the scheme pays when it needs one component)."""
        nx, ny, nz = self.n
        Mhat = sfft.rfftn(m, s=self.P, axes=(1, 2, 3), workers=self.workers)
        acc = 0.0
        for b in range(3):
            acc = acc + self.Khat[_IDX[(a, b)]] * Mhat[b]
        return -sfft.irfftn(acc, s=self.P, axes=(0, 1, 2), workers=self.workers)[:nz, :ny, :nx]


def stray_direct(m, Nfull):
    """Brute-force h_a(i) = -sum_j sum_b N_ab(i - j) m_b(j) (tiny grids only)."""
    _, nz, ny, nx = m.shape
    h = np.zeros_like(m)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for a in range(3):
                    s = 0.0
                    for kk in range(nz):
                        for jj in range(ny):
                            for ii in range(nx):
                                # N(target - source)
                                o = (k - kk + nz - 1, j - jj + ny - 1, i - ii + nx - 1)
                                for b in range(3):
                                    s += Nfull[_IDX[(a, b)]][o] * m[b, kk, jj, ii]
                    h[a, k, j, i] = -s
    return h
