"""Implicit heat solve (I - c dt Delta_h)^{-1} with homogeneous Neumann BC (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

The scheme's sub-problems are g = (I - eps dt Delta_h)^{-1}(m + dt f) (Sec. 3.1 and 3.2,
Step 1) and the damping heat flow (I - alpha eps dt Delta_h) m*** = m** + alpha dt f**
(Step 2), under the Neumann condition of Eq. (2).  The paper does not write Delta_h;
the reading used throughout is the cell-centred 7-point Laplacian with mirror ghost
cells (u_{-1} = u_0, u_n = u_{n-1} on every axis), which the DCT-II diagonalises
exactly with eigenvalues -(4/h^2) sin^2(pi k / (2n)), k = 0..n-1.

Fields are [nz, ny, nx] (x fastest) for one scalar component.
"""
import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla


def laplacian(u, h):
    """Mirror-ghost 7-point Laplacian of a scalar field u[nz, ny, nx]."""
    out = np.zeros_like(u)
    for axis, ha in zip((2, 1, 0), h):          # x, y, z
        if u.shape[axis] == 1:
            continue
        pad = [(0, 0)] * 3
        pad[axis] = (1, 1)
        up = np.pad(u, pad, mode="edge")        # ghost = boundary value
        sl_p = [slice(None)] * 3
        sl_m = [slice(None)] * 3
        sl_p[axis] = slice(2, None)
        sl_m[axis] = slice(0, -2)
        out += (up[tuple(sl_p)] - 2.0 * u + up[tuple(sl_m)]) / ha ** 2
    return out


def eigenvalues(n, h):
    """lambda(k_x, k_y, k_z) >= 0 with -Delta_h = C^T diag(lambda) C (C = orthonormal DCT-II)."""
    lam = 0.0
    for axis, (na, ha) in enumerate(zip(n, h)):     # n = (nx, ny, nz)
        k = np.arange(na)
        la = 4.0 / ha ** 2 * np.sin(np.pi * k / (2.0 * na)) ** 2
        shape = [1, 1, 1]
        shape[2 - axis] = na
        lam = lam + la.reshape(shape)
    return lam


def heat_solve(r, c_dt, h, workers=None):
    """(I - c_dt Delta_h)^{-1} r by orthonormal DCT-II, diagonal scaling and DCT-III."""
    nz, ny, nx = r.shape
    lam = eigenvalues((nx, ny, nz), h)
    rhat = sfft.dctn(r, type=2, norm="ortho", workers=workers)
    return sfft.idctn(rhat / (1.0 + c_dt * lam), type=2, norm="ortho", workers=workers)


def laplacian_matrix(n, h):
    """Assemble Delta_h as a dense (nx ny nz)^2 matrix, cell index i + nx (j + ny k)."""
    nx, ny, nz = n
    N = nx * ny * nz
    A = np.zeros((N, N))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * (j + ny * k)
                for (di, dj, dk, ha) in ((1, 0, 0, h[0]), (-1, 0, 0, h[0]), (0, 1, 0, h[1]),
                                         (0, -1, 0, h[1]), (0, 0, 1, h[2]), (0, 0, -1, h[2])):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        A[c, ii + nx * (jj + ny * kk)] += 1.0 / ha ** 2
                        A[c, c] -= 1.0 / ha ** 2
                    # a neighbour outside the grid is the mirror ghost: u_ghost - u_c = 0
    return A


def heat_solve_dense(r, c_dt, h):
    """Dense LU solve of (I - c_dt Delta_h) g = r (tiny grids only)."""
    nz, ny, nx = r.shape
    A = np.eye(nx * ny * nz) - c_dt * laplacian_matrix((nx, ny, nz), h)
    return sla.lu_solve(sla.lu_factor(A), r.reshape(-1)).reshape(r.shape)
