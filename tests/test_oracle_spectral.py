"""Pins of the spectral-radius diagnostic (Sec. 4, oracle/spectral.py).

The paper prints rho(G_GS) and rho(G_SGS) (Tables 1-2) without the entries of its blocks
"dt Delta_h g"; the values below follow the reading in oracle/spectral.py and are not compared
with the tables' digits (parity unpinned).  What is pinned:
  * the dense 3N x 3N assembly and the per-cell 3 x 3 reduction give the same radii;
  * per cell, G_GS = (D-L)^{-1} U has a zero eigenvalue (U's first block column is zero) and its
    other two eigenvalues are the roots of  l^2 - (d(ac - b) - a^2 - c^2) l + abc  (worked out by
    hand from the blocks), so a dropped sign or a misplaced block fails;
  * every block carries one factor dt, so from a fixed state the radii scale as dt^2;
  * the paper's observation rho(G_SGS) < rho(G_GS) on the Table 1 runs (1D manufactured
    solution, dx = 5e-4, T = 1, dt = 2e-2 and 1.25e-2).
"""
import numpy as np
import pytest

from oracle import scheme, spectral


def _step_values(n, h, dt, m):
    o = scheme.Oracle(scheme.Params(n=n, h=h, eps=1.0, Q=0.0, alpha=1e-3, dt=dt, stray=False))
    o.step(m, 0.0)
    return spectral.block_values(o.last_intermediates, dt, h)


def _smooth_state(n, h):
    x, y, z = scheme.cell_centres(n, h)
    phi = np.cos(np.pi * x) + 0.3 * np.sin(2 * np.pi * y) * np.cos(np.pi * z)
    m = np.stack([np.cos(phi) * np.sin(0.7), np.sin(phi) * np.sin(0.7), np.full_like(phi, np.cos(0.7))])
    return m / np.linalg.norm(m, axis=0)


def test_dense_assembly_equals_cellwise_reduction():
    n, h = (6, 4, 2), (0.2, 0.25, 0.3)
    vals = _step_values(n, h, 0.05, _smooth_state(n, h))
    gd, sd = spectral.radii_dense(vals)
    gc, sc = spectral.radii_cellwise(vals)
    assert gd > 0 and sd > 0
    assert abs(gd - gc) <= 1e-12 * gd and abs(sd - sc) <= 1e-12 * sd


def test_gauss_seidel_eigenvalues_closed_form():
    n, h = (8, 5, 3), (0.15, 0.2, 0.25)
    vals = _step_values(n, h, 0.05, _smooth_state(n, h))
    a, b, c, d, _, _ = vals
    Ggs, _ = spectral.cell_matrices(vals)
    ev = np.sort_complex(np.linalg.eigvals(Ggs))
    tr = d * (a * c - b) - a * a - c * c
    disc = np.sqrt((tr * tr - 4 * a * b * c).astype(complex))
    want = np.sort_complex(np.stack([np.zeros_like(tr, dtype=complex), (tr + disc) / 2, (tr - disc) / 2], axis=-1))
    scale = np.abs(want).max()
    assert np.abs(ev - want).max() <= 1e-12 * scale


def test_radii_scale_as_dt_squared():
    n, h = (16, 8, 4), (1 / 16, 1 / 8, 1 / 4)
    m = _smooth_state(n, h)
    r = [spectral.radii_cellwise(_step_values(n, h, dt, m)) for dt in (4e-4, 2e-4)]
    for k in range(2):
        assert 3.9 < r[0][k] / r[1][k] < 4.1


@pytest.mark.parametrize("dt,paper", [(2e-2, (5.896039e-06, 3.239712e-06)), (1.25e-2, (3.641269e-06, 1.683222e-06))])
def test_symmetric_sweep_has_the_smaller_radius_on_table1_runs(dt, paper):
    n, h = (2000, 1, 1), (5e-4, 1.0, 1.0)
    alpha = 1e-3
    p = scheme.Params(n=n, h=h, eps=1.0, Q=0.0, alpha=alpha, dt=dt, stray=False,
                      forcing=scheme.manufactured_forcing(n, h, alpha, 1))
    o = scheme.Oracle(p)
    m = scheme.manufactured_m(n, h, 0.0, 1)
    t = 0.0
    for _ in range(int(round(1.0 / dt))):
        m = o.step(m, t)
        t += dt
    g, s = spectral.radii_cellwise(spectral.block_values(o.last_intermediates, dt, h))
    print(f"dt={dt}: rho_GS {g:.6e} rho_SGS {s:.6e} (Table 1 prints {paper[0]:.6e} {paper[1]:.6e}; parity unpinned)")
    assert s < g
    assert paper[1] < paper[0]
