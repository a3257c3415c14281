"""Pins of the oracle's heat solve and stray-field convolution (CPU only)."""
import numpy as np
import pytest

from oracle import demag, heat, newell


@pytest.mark.parametrize("shape,h", [((3, 4, 5), (0.5, 0.4, 0.3)), ((1, 1, 7), (0.1, 1.0, 1.0)),
                                     ((2, 6, 1), (1.0, 0.25, 2.0)), ((1, 5, 4), (0.3, 0.3, 0.3))])
def test_dct_solve_equals_dense_lu(shape, h):
    rng = np.random.default_rng(1)
    r = rng.normal(size=shape)
    for c_dt in (1e-3, 0.7, 50.0):
        assert np.abs(heat.heat_solve(r, c_dt, h) - heat.heat_solve_dense(r, c_dt, h)).max() < 1e-13


def test_dct_eigenvalues_equal_dense_spectrum():
    n, h = (5, 3, 2), (0.3, 0.7, 1.1)
    A = heat.laplacian_matrix(n, h)
    ev = np.sort(-np.linalg.eigvalsh(A))
    lam = np.sort(heat.eigenvalues(n, h).reshape(-1))
    assert np.allclose(ev, lam, atol=1e-12)


def test_laplacian_of_quadratic_and_constant():
    nx, h = 9, 0.2
    x = (np.arange(nx) + 0.5) * h
    u = np.broadcast_to(x * x, (1, 1, nx)).copy()
    lap = heat.laplacian(u, (h, 1.0, 1.0))
    assert np.allclose(lap[0, 0, 1:-1], 2.0, atol=1e-12)       # interior: exact for quadratics
    assert np.allclose(heat.laplacian(np.ones((3, 4, 5)), (0.1, 0.2, 0.3)), 0.0)


def test_laplacian_matrix_matches_stencil():
    rng = np.random.default_rng(2)
    n, h = (4, 3, 2), (0.5, 0.3, 0.2)
    u = rng.normal(size=(2, 3, 4))
    assert np.allclose((heat.laplacian_matrix(n, h) @ u.reshape(-1)).reshape(u.shape), heat.laplacian(u, h))


@pytest.mark.parametrize("n,h", [((4, 3, 2), (1.0, 1.0, 1.0)), ((3, 1, 1), (1.0, 0.5, 0.5)),
                                 ((1, 4, 3), (0.7, 1.0, 0.3)), ((5, 4, 1), (1.0, 1.0, 0.2))])
def test_stray_fft_equals_direct_sum(n, h):
    rng = np.random.default_rng(3)
    m = rng.normal(size=(3, n[2], n[1], n[0]))
    op = demag.StrayOperator(n, h)
    hd = demag.stray_direct(m, op.N)
    assert np.abs(op(m) - hd).max() < 1e-14 * max(1.0, np.abs(hd).max())
    for a in range(3):
        assert np.abs(op.component(m, a) - hd[a]).max() < 1e-14 * max(1.0, np.abs(hd).max())


def test_uniform_prism_mean_field_is_minus_prism_factor():
    # mean stray field of a uniformly magnetised prism = -N_prism m (exact, Newell self term)
    n, h = (6, 4, 3), (1.0, 0.9, 0.5)
    op = demag.StrayOperator(n, h)
    mdir = np.array([0.3, -0.5, 0.8])
    m = np.broadcast_to(mdir.reshape(3, 1, 1, 1), (3, n[2], n[1], n[0])).copy()
    hm = op(m).mean(axis=(1, 2, 3))
    Np = newell.tensor_analytic(0.0, 0.0, 0.0, n[0] * h[0], n[1] * h[1], n[2] * h[2])
    Nmat = np.array([[Np[0], Np[3], Np[4]], [Np[3], Np[1], Np[5]], [Np[4], Np[5], Np[2]]])
    assert np.allclose(hm, -Nmat @ mdir, atol=1e-13)


def test_stray_operator_is_symmetric_and_energy_positive():
    n, h = (8, 6, 2), (1.0, 1.0, 1.0)
    rng = np.random.default_rng(4)
    a = rng.normal(size=(3, 2, 6, 8))
    b = rng.normal(size=(3, 2, 6, 8))
    op = demag.StrayOperator(n, h)
    assert abs(np.sum(op(a) * b) - np.sum(op(b) * a)) < 1e-12 * np.sum(np.abs(a))
    assert -np.sum(op(a) * a) > 0
