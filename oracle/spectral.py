"""Spectral radii of the Gauss-Seidel and symmetric Gauss-Seidel iteration matrices of one
step (Sec. 4), from the intermediates of an oracle step.  Test infrastructure only (see
oracle/__init__.py).

Sec. 4 takes eps = 1 and f = 0, so g_i = (I - dt Delta_h)^{-1} m_i, and writes Step 1 as a block
system in (m1, m2, m3) whose blocks are "dt Delta_h g_i^s".  The component updates it starts
from are cell by cell:  m1* = m1^n - m2^n (dt Delta_h g3^n) + m3^n (dt Delta_h g2^n), etc., so a
block multiplies a component pointwise.  Reading taken here: the block dt Delta_h g_i^s is the
diagonal matrix diag(dt (Delta_h g_i^s)_j) (the paper does not write out the blocks' entries).

With the per-cell values   a = dt Delta_h g3^n,  d = dt Delta_h g2^n,  c = dt Delta_h g1*,
b = dt Delta_h g2*,  e = dt Delta_h g3**,  f = dt Delta_h g2**  (component order 1, 2, 3):

    D - L = [[I, 0, 0], [-a, I, 0], [b, -c, I]],        U = [[0, -a, d], [0, 0, -c], [0, 0, 0]],
    (D - U)_SGS = [[I, -e, f], [0, I, -c], [0, 0, I]],  L_SGS = [[0, 0, 0], [e, 0, 0], [-b, c, 0]],
    G_GS = (D - L)^{-1} U,   G_SGS = (D - U)_SGS^{-1} L_SGS (D - L)^{-1} U,

and the spectral radius is the largest eigenvalue modulus.  Two computations are provided: the
dense 3N x 3N matrices assembled from the blocks (small N), and the per-cell 3 x 3 matrices
the block-diagonal structure reduces them to.  Parity with Tables 1-2 is unpinned: the paper
prints the radii but not its discretisation of the blocks.
"""
import numpy as np

from . import heat


def block_values(it, dt, h):
    """(a, b, c, d, e, f) per cell (flattened) from Oracle.last_intermediates of an SGSPM step."""
    L = lambda g: (dt * heat.laplacian(g, h)).reshape(-1)
    return L(it["g3n"]), L(it["g2s"]), L(it["g1s"]), L(it["g2n"]), L(it["g3ss"]), L(it["g2ss"])


def dense_matrices(vals):
    """The 3N x 3N matrices D - L, U, (D - U)_SGS and L_SGS of Sec. 4 from diagonal blocks."""
    a, b, c, d, e, f = vals
    N = a.size
    I, Z, D = np.eye(N), np.zeros((N, N)), np.diag
    DL = np.block([[I, Z, Z], [-D(a), I, Z], [D(b), -D(c), I]])
    U = np.block([[Z, -D(a), D(d)], [Z, Z, -D(c)], [Z, Z, Z]])
    DU = np.block([[I, -D(e), D(f)], [Z, I, -D(c)], [Z, Z, I]])
    Ls = np.block([[Z, Z, Z], [D(e), Z, Z], [-D(b), D(c), Z]])
    return DL, U, DU, Ls


def radii_dense(vals):
    """(rho(G_GS), rho(G_SGS)) by a dense eigen-solve of the assembled matrices."""
    DL, U, DU, Ls = dense_matrices(vals)
    Ggs = np.linalg.solve(DL, U)
    Gsgs = np.linalg.solve(DU, Ls @ Ggs)
    return np.abs(np.linalg.eigvals(Ggs)).max(), np.abs(np.linalg.eigvals(Gsgs)).max()


def cell_matrices(vals):
    """Per-cell 3 x 3 iteration matrices (N, 3, 3): G_GS and G_SGS of each cell."""
    a, b, c, d, e, f = vals
    N = a.size
    one, zero = np.ones(N), np.zeros(N)
    m = lambda rows: np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)
    DL = m([[one, zero, zero], [-a, one, zero], [b, -c, one]])
    U = m([[zero, -a, d], [zero, zero, -c], [zero, zero, zero]])
    DU = m([[one, -e, f], [zero, one, -c], [zero, zero, one]])
    Ls = m([[zero, zero, zero], [e, zero, zero], [-b, c, zero]])
    Ggs = np.linalg.solve(DL, U)
    return Ggs, np.linalg.solve(DU, Ls @ Ggs)


def radii_cellwise(vals):
    """(rho(G_GS), rho(G_SGS)): the largest eigenvalue modulus over the cells' 3 x 3 matrices."""
    Ggs, Gsgs = cell_matrices(vals)
    return np.abs(np.linalg.eigvals(Ggs)).max(), np.abs(np.linalg.eigvals(Gsgs)).max()
