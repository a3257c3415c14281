"""Newell demagnetising tensor of a uniform grid of rectangular cells (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

The paper evaluates the stray field h_s "by FFT" (Sec. 1 and Sec. 5.1, after Table 5)
without naming the kernel; the kernel used here is the cell-averaged demagnetising
tensor of Newell, Williams & Dunlop (J. Geophys. Res. 98, 1993): for two cells of
size (dx, dy, dz) whose centres differ by R,

    h_s(cell i) = - sum_j N(R_i - R_j) m_j,
    N_ab(R)     = (1/V) int_{cell_i} int_{cell_j} D_ab(x - y) dx dy,
    D_ab(r)     = (delta_ab |r|^2 - 3 r_a r_b) / (4 pi |r|^5),     V = dx dy dz.

Two independent evaluations of N_ab are written out:

* `tensor_analytic`: Newell's closed form, the triple second difference of the
  auxiliary functions f (diagonal terms) and g (off-diagonal terms).  It is exact,
  but its 27-term sum cancels catastrophically as |R| grows (relative loss of
  roughly (|R|/dx)^6 * 1e-16).
* `tensor_quadrature`: the same double cell integral reduced to one integral over
  the difference u = (x - c_i) - (y - c_j), whose density is the product of three
  triangle ("tent") functions of half-width dx, dy, dz:
      N_ab(R) = V * int T(u) D_ab(R + u) du.
  Each tent is split at 0 and integrated by q-point Gauss-Legendre on each half.
  The integrand is analytic on the tent's support once the two cells are at least
  one cell apart, and the rule then converges geometrically with no cancellation.

`tensor` picks the analytic form for the 27 touching/overlapping offsets and the
quadrature elsewhere (the closest-approach distance between the two cells decides,
and it also sets q).  Tests pin both forms against each other where both are
accurate, against sum rules (a uniformly magnetised cube of k^3 cells has mean
demagnetising factor exactly 1/3; the pair-average over a prism equals the
prism's own self term), against Laplace's trace rule and the far dipole limit.
"""
import numpy as np

PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))   # xx yy zz xy xz yz


def _safe_asinh_ratio(num, den2):
    """asinh(num / sqrt(den2)); 0 where den2 == 0 (the prefactor vanishes there)."""
    out = np.zeros(np.broadcast(num, den2).shape)
    ok = den2 > 0
    out[ok] = np.arcsinh((num * np.ones_like(out))[ok] / np.sqrt((den2 * np.ones_like(out))[ok]))
    return out


def _safe_atan_ratio(num, den):
    """atan(num / den); 0 where den == 0 (the prefactor vanishes there)."""
    out = np.zeros(np.broadcast(num, den).shape)
    ok = den != 0
    out[ok] = np.arctan((num * np.ones_like(out))[ok] / (den * np.ones_like(out))[ok])
    return out


def newell_f(x, y, z):
    """Newell's f(x, y, z), whose triple second difference gives N_xx."""
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = 0.5 * y * (z2 - x2) * _safe_asinh_ratio(y, x2 + z2)
    t = t + 0.5 * z * (y2 - x2) * _safe_asinh_ratio(z, x2 + y2)
    t = t - x * y * z * _safe_atan_ratio(y * z, x * R)
    t = t + (2.0 * x2 - y2 - z2) * R / 6.0
    return t


def newell_g(x, y, z):
    """Newell's g(x, y, z), whose triple second difference gives N_xy."""
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = x * y * z * _safe_asinh_ratio(z, x2 + y2)
    t = t + y / 6.0 * (3.0 * z2 - y2) * _safe_asinh_ratio(x, y2 + z2)
    t = t + x / 6.0 * (3.0 * z2 - x2) * _safe_asinh_ratio(y, x2 + z2)
    t = t - z2 * z / 6.0 * _safe_atan_ratio(x * y, z * R)
    t = t - z * y2 / 2.0 * _safe_atan_ratio(x * z, y * R)
    t = t - z * x2 / 2.0 * _safe_atan_ratio(y * z, x * R)
    t = t - x * y * R / 3.0
    return t


_C = {-1: -1.0, 0: 2.0, 1: -1.0}   # (2 - S^+ - S^-) along each axis


def _second_difference(fun, X, Y, Z, dx, dy, dz):
    s = 0.0
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                s = s + _C[i] * _C[j] * _C[k] * fun(X + i * dx, Y + j * dy, Z + k * dz)
    return s / (4.0 * np.pi * dx * dy * dz)


def tensor_analytic(X, Y, Z, dx, dy, dz):
    """Newell's closed form at offsets (X, Y, Z); returns [xx, yy, zz, xy, xz, yz]."""
    nxx = _second_difference(newell_f, X, Y, Z, dx, dy, dz)
    nyy = _second_difference(newell_f, Y, X, Z, dy, dx, dz)
    nzz = _second_difference(newell_f, Z, Y, X, dz, dy, dx)
    nxy = _second_difference(newell_g, X, Y, Z, dx, dy, dz)
    nxz = _second_difference(newell_g, X, Z, Y, dx, dz, dy)
    nyz = _second_difference(newell_g, Y, Z, X, dy, dz, dx)
    return np.stack(np.broadcast_arrays(nxx, nyy, nzz, nxy, nxz, nyz))


def tent_rule(half_width, q):
    """Nodes/weights integrating against the unit-mass tent (h - |u|)/h^2 on [-h, h]."""
    x, w = np.polynomial.legendre.leggauss(q)
    s = half_width * (1.0 + x) / 2.0
    ws = w * half_width / 2.0 * (half_width - s) / half_width ** 2
    return np.concatenate([-s[::-1], s]), np.concatenate([ws[::-1], ws])


def tensor_quadrature(X, Y, Z, dx, dy, dz, q):
    """V * int T(u) D_ab(R+u) du by a (2q)^3 tent-Gauss rule; [xx, yy, zz, xy, xz, yz]."""
    X, Y, Z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (X, Y, Z)))
    ux, wx = tent_rule(dx, q)
    uy, wy = tent_rule(dy, q)
    uz, wz = tent_rule(dz, q)
    acc = np.zeros((6,) + X.shape)
    for a in range(ux.size):
        for b in range(uy.size):
            for c in range(uz.size):
                w = wx[a] * wy[b] * wz[c]
                r = (X + ux[a], Y + uy[b], Z + uz[c])
                r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2]
                inv5 = 1.0 / (r2 * r2 * np.sqrt(r2))
                for p, (i, j) in enumerate(PAIRS):
                    d = -3.0 * r[i] * r[j]
                    if i == j:
                        d = d + r2
                    acc[p] += w * d * inv5
    return acc * (dx * dy * dz) / (4.0 * np.pi)


def closest_approach(X, Y, Z, dx, dy, dz):
    """Smallest |x - y| between points of the two cells, in units of the largest cell edge."""
    gx = np.maximum(0.0, np.abs(X) - dx)
    gy = np.maximum(0.0, np.abs(Y) - dy)
    gz = np.maximum(0.0, np.abs(Z) - dz)
    return np.sqrt(gx * gx + gy * gy + gz * gz) / max(dx, dy, dz)


def quadrature_order(dist):
    """Points per half-tent for a cell pair at closest-approach distance `dist` (>= 1).

    The integrand's nearest singularity sits at distance >= dist from the support, so
    the Gauss error falls geometrically in dist.  The orders below bring the rule's
    error to the float64 summation floor (~1e-14 relative), as checked against
    50-digit evaluations of the closed form.
    """
    return np.where(dist < 2, 14, np.where(dist < 3, 8, np.where(dist < 6, 7,
                    np.where(dist < 10, 6, np.where(dist < 40, 5, 4)))))


def tensor(X, Y, Z, dx, dy, dz):
    """N_ab at integer-cell offsets: closed form when the cells touch, quadrature otherwise."""
    X, Y, Z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (X, Y, Z)))
    out = np.zeros((6,) + X.shape)
    dist = closest_approach(X, Y, Z, dx, dy, dz)
    near = dist < 1.0
    if near.any():
        out[:, near] = tensor_analytic(X[near], Y[near], Z[near], dx, dy, dz)
    qs = quadrature_order(dist)
    for q in np.unique(qs[~near]):
        sel = (~near) & (qs == q)
        out[:, sel] = tensor_quadrature(X[sel], Y[sel], Z[sel], dx, dy, dz, int(q))
    return out


# parity of each component under reflection of one offset axis (x, y, z): +1 even, -1 odd
PARITY = np.array([[1, 1, 1], [1, 1, 1], [1, 1, 1],
                   [-1, -1, 1], [-1, 1, -1], [1, -1, -1]], dtype=np.float64)


def demag_tensor(n, h):
    """N_ab(i, j, k) for all offsets |i| < nx, |j| < ny, |k| < nz of an (nx, ny, nz) grid.

    Returns an array [6, 2nz-1, 2ny-1, 2nx-1]; the offset (i, j, k) sits at index
    [:, k + nz - 1, j + ny - 1, i + nx - 1].  The tensor is evaluated on the octant
    of non-negative offsets and reflected with each component's parity (D_ab(r)
    changes sign under r_a -> -r_a once for each of a, b equal to that axis, and the
    cells are mirror-symmetric), which is a property of the definition above.
    """
    nx, ny, nz = n
    dx, dy, dz = h
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    octant = tensor(I * dx, J * dy, K * dz, dx, dy, dz)          # [6, nz, ny, nx]
    full = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    for sz in (1, -1):
        for sy in (1, -1):
            for sx in (1, -1):
                sign = (PARITY[:, 0] ** (sx < 0)) * (PARITY[:, 1] ** (sy < 0)) * (PARITY[:, 2] ** (sz < 0))
                kk = nz - 1 + sz * np.arange(nz)
                jj = ny - 1 + sy * np.arange(ny)
                ii = nx - 1 + sx * np.arange(nx)
                full[:, kk[:, None, None], jj[None, :, None], ii[None, None, :]] = sign[:, None, None, None] * octant
    return full
