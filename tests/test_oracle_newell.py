"""Pins of the oracle's Newell tensor against facts fixed by the mathematics.

The stray-field kernel is the cell-averaged demagnetising tensor (Newell et al. 1993),
used for the paper's FFT stray field (Sec. 1, Sec. 5.1).  None of these checks reuses
the code under test to produce its expected value.
"""
import mpmath as mp
import numpy as np
import pytest

from oracle import newell


def test_cube_self_term_is_one_third():
    N = newell.tensor_analytic(0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
    assert np.allclose(N[:3], 1.0 / 3.0, atol=1e-15)
    assert np.allclose(N[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("d", [(1.0, 0.7, 0.3), (0.2, 1.0, 3.0), (2.0, 2.0, 0.25)])
def test_self_term_trace_is_one(d):
    N = newell.tensor_analytic(0.0, 0.0, 0.0, *d)
    assert abs(N[0] + N[1] + N[2] - 1.0) < 1e-14


@pytest.mark.parametrize("R", [(1, 0, 0), (1, 1, 0), (2, 1, 0), (3, 2, 1), (0, 0, 2)])
def test_trace_vanishes_off_the_cell(R):
    # outside the source cell the potential is harmonic: tr N = 0
    N = newell.tensor_analytic(*map(float, R), 1.0, 1.0, 1.0)
    assert abs(N[0] + N[1] + N[2]) < 1e-14


def _pair_average(Nfull, n):
    nx, ny, nz = n
    c = [na - np.abs(np.arange(-(na - 1), na)) for na in (nz, ny, nx)]
    w = c[0][:, None, None] * c[1][None, :, None] * c[2][None, None, :]
    return (Nfull * w[None]).sum(axis=(1, 2, 3)) / (nx * ny * nz)


@pytest.mark.parametrize("k", [3, 6])
def test_cube_sum_rule(k):
    # a uniformly magnetised cube of k^3 cells has mean demagnetising factor exactly 1/3
    Nf = newell.demag_tensor((k, k, k), (1.0, 1.0, 1.0))
    avg = _pair_average(Nf, (k, k, k))
    assert np.allclose(avg[:3], 1.0 / 3.0, atol=2e-14)
    assert np.allclose(avg[3:], 0.0, atol=2e-14)


@pytest.mark.parametrize("n,h", [((4, 3, 2), (1.0, 1.0, 1.0)), ((5, 2, 3), (0.5, 1.0, 0.8))])
def test_prism_pair_average_equals_prism_self_term(n, h):
    # averaging the cell tensor over all cell pairs of a prism gives the prism's own factor
    Nf = newell.demag_tensor(n, h)
    avg = _pair_average(Nf, n)
    whole = newell.tensor_analytic(0.0, 0.0, 0.0, n[0] * h[0], n[1] * h[1], n[2] * h[2])
    assert np.allclose(avg, whole, atol=5e-14)


@pytest.mark.parametrize("R", [(2, 0, 0), (2, 1, 0), (2, 2, 1), (3, 1, 1), (0, 3, 2), (4, 0, 1)])
def test_quadrature_matches_closed_form_where_both_are_exact(R):
    q = newell.tensor_quadrature(*map(float, R), 1.0, 1.0, 1.0, 14)
    a = newell.tensor_analytic(*map(float, R), 1.0, 1.0, 1.0)
    scale = np.abs(a).max()
    assert np.abs(q - a).max() < 5e-12 * scale   # closed form loses ~|R|^6 eps


# 50-digit evaluation of the closed form, independent of the float64 code paths
mp.mp.dps = 50


def _f50(x, y, z):
    x, y, z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
    R = mp.sqrt(x * x + y * y + z * z)
    t = mp.mpf(0)
    if x * x + z * z > 0:
        t += y / 2 * (z * z - x * x) * mp.asinh(y / mp.sqrt(x * x + z * z))
    if x * x + y * y > 0:
        t += z / 2 * (y * y - x * x) * mp.asinh(z / mp.sqrt(x * x + y * y))
    if x != 0 and R > 0:
        t -= x * y * z * mp.atan(y * z / (x * R))
    return t + (2 * x * x - y * y - z * z) * R / 6


def _nxx50(X, Y, Z):
    c = {-1: -1, 0: 2, 1: -1}
    s = mp.mpf(0)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                s += c[i] * c[j] * c[k] * _f50(X + i, Y + j, Z + k)
    return s / (4 * mp.pi)


@pytest.mark.parametrize("R", [(2, 0, 0), (3, 1, 0), (3, 0, 0), (6, 2, 1), (8, 0, 0), (12, 5, 3), (29, 0, 0), (41, 0, 0), (40, 31, 2)])
def test_chosen_rule_reaches_double_precision(R):
    got = newell.tensor(*map(float, R), 1.0, 1.0, 1.0)[0]
    ref = float(_nxx50(*R))
    assert abs(got - ref) <= 3e-14 * abs(ref)   # float64 summation floor of the rule


@pytest.mark.parametrize("R", [(60, 0, 0), (0, 45, 30), (50, 50, 5)])
def test_far_field_tends_to_point_dipole(R):
    R = np.array(R, dtype=float)
    N = newell.tensor(*R, 1.0, 1.0, 1.0)
    r = np.linalg.norm(R)
    dip = np.array([(1.0 if a == b else 0.0) - 3 * R[a] * R[b] / r ** 2
                    for a, b in newell.PAIRS]) / (4 * np.pi * r ** 3)
    # the cell average differs from the point dipole at relative order (h/r)^2
    assert np.abs(N - dip).max() < 2.0 / r ** 2 * np.abs(dip).max()


def test_reflected_offsets_match_direct_evaluation():
    n, h = (4, 3, 3), (1.0, 0.8, 0.6)
    Nf = newell.demag_tensor(n, h)
    for (i, j, k) in [(-3, 2, -1), (2, -2, 2), (-1, -1, -2), (0, -2, 1)]:
        direct = newell.tensor(i * h[0], j * h[1], k * h[2], *h)
        got = Nf[:, k + n[2] - 1, j + n[1] - 1, i + n[0] - 1]
        assert np.abs(got - direct).max() < 1e-13 * np.abs(direct).max()
