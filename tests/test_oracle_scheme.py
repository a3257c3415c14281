"""Pins of the oracle's SGSPM/GSPM step against what the paper and the mathematics fix."""
import numpy as np
import pytest

from oracle import heat, scheme

PAPER_TABLE3_SGSPM = {2e-2: 0.031993635118710, 1e-2: 0.016258177977747, 5e-3: 0.008198757469279,
                      2.5e-3: 0.004140400463721}            # Table 3, 1D, dx = 5e-4, alpha = 1e-3, T = 1
PAPER_TABLE5_SGSPM = {1 / 32: 2.877587588594097e-04, 1 / 64: 1.473122547213623e-04,
                      1 / 512: 2.005449155901271e-05}                    # Table 5, 3D, h = 1/16


def random_unit(rng, n):
    m = rng.normal(size=(3, n[2], n[1], n[0]))
    return m / np.linalg.norm(m, axis=0)


def full_params(n, **kw):
    h = kw.pop("h", (1.0 / n[0],) * 3)
    base = dict(n=n, h=h, eps=0.016 * 64, Q=0.3, alpha=0.05, dt=0.01, u=(0.6, 0.8, 0.0),
                he=(0.02, -0.01, 0.03), stray=True)
    base.update(kw)
    return scheme.Params(**base)


@pytest.mark.parametrize("sch", ["sgspm", "gspm"])
def test_projection_gives_unit_length(sch):
    rng = np.random.default_rng(0)
    n = (6, 5, 3)
    o = scheme.Oracle(full_params(n, scheme=sch))
    m = o.run(random_unit(rng, n), 5)
    assert np.abs(np.linalg.norm(m, axis=0) - 1.0).max() < 1e-15


def test_backward_sweep_starts_from_forward_m3():
    # Sec. 3.2: m3** has the same formula and arguments as m3*
    rng = np.random.default_rng(1)
    n = (5, 4, 2)
    o = scheme.Oracle(full_params(n))
    o.step(random_unit(rng, n), 0.0)
    it = o.last_intermediates
    assert np.array_equal(it["m3s"], it["m3ss"])


def test_gauss_seidel_updates_equal_laplacian_g_form():
    # Sec. 4: with eps = 1 and f = 0, g - m = dt Delta_h g turns every update into
    # (m_new - m_old)/dt = -m_b Delta_h g_c + m_c Delta_h g_b.
    rng = np.random.default_rng(2)
    n, h = (6, 5, 4), (0.2, 0.25, 0.3)
    p = scheme.Params(n=n, h=h, eps=1.0, Q=0.0, alpha=0.1, dt=0.01, stray=False)
    o = scheme.Oracle(p)
    m = random_unit(rng, n)
    o.step(m, 0.0)
    it = o.last_intermediates
    L = lambda g: heat.laplacian(g, h)
    m1, m2, m3 = m
    dt = p.dt
    checks = [
        ((it["m1s"] - m1) / dt, -m2 * L(it["g3n"]) + m3 * L(it["g2n"])),
        ((it["m2s"] - m2) / dt, -m3 * L(it["g1s"]) + it["m1s"] * L(it["g3n"])),
        ((it["m3s"] - m3) / dt, -it["m1s"] * L(it["g2s"]) + it["m2s"] * L(it["g1s"])),
        ((it["m3ss"] - m3) / dt, -it["m1s"] * L(it["g2s"]) + it["m2s"] * L(it["g1s"])),
        ((it["m2ss"] - m2) / dt, -it["m3ss"] * L(it["g1s"]) + it["m1s"] * L(it["g3ss"])),
        ((it["m1ss"] - m1) / dt, -it["m2ss"] * L(it["g3ss"]) + it["m3ss"] * L(it["g2ss"])),
    ]
    for lhs, rhs in checks:
        assert np.abs(lhs - rhs).max() < 1e-10 * max(1.0, np.abs(rhs).max())


def test_uniform_state_is_a_fixed_point():
    n = (5, 4, 3)
    mdir = np.array([0.48, 0.6, 0.64])
    m = np.broadcast_to(mdir.reshape(3, 1, 1, 1), (3, 3, 4, 5)).copy()
    # exchange only: g = m, all cross products vanish
    o = scheme.Oracle(scheme.Params(n=n, h=(0.2,) * 3, eps=1.0, Q=0.0, alpha=0.3, dt=0.05, stray=False))
    assert np.abs(o.run(m, 3) - m).max() < 1e-14
    # anisotropy along m and a field parallel to m keep it fixed too
    o = scheme.Oracle(scheme.Params(n=n, h=(0.2,) * 3, eps=1.0, Q=0.7, alpha=0.3, dt=0.05, stray=False,
                                    u=tuple(mdir), he=tuple(0.1 * mdir)))
    assert np.abs(o.run(m, 3) - m).max() < 1e-14


def test_energy_gradient_is_minus_volume_times_h_eff():
    rng = np.random.default_rng(3)
    n, h = (4, 3, 2), (0.3, 0.4, 0.5)
    he = rng.normal(size=(3, 2, 3, 4)) * 0.1
    o = scheme.Oracle(full_params(n, h=h, he=he))
    m = random_unit(rng, n)
    V = np.prod(h)
    heff = o.h_eff(m)
    step = 1e-6
    for (a, k, j, i) in [(0, 0, 0, 0), (1, 1, 2, 3), (2, 0, 1, 2), (0, 1, 1, 1), (2, 1, 2, 0)]:
        mp_, mm_ = m.copy(), m.copy()
        mp_[a, k, j, i] += step
        mm_[a, k, j, i] -= step
        fd = (o.energy(mp_)[4] - o.energy(mm_)[4]) / (2 * step)
        assert abs(-fd / V - heff[a, k, j, i]) < 1e-6 * max(1.0, abs(heff[a, k, j, i]))


def _m0_eq_m0_1(n, h):
    # initial state of Sec. 3.1 / Sec. 5.2 (eq-m0-1)
    x, _, _ = scheme.cell_centres(n, h)
    return np.stack([np.cos(np.cos(np.pi * x)) * np.sin(0.01), np.sin(np.cos(np.pi * x)) * np.sin(0.01),
                     np.full_like(x, np.cos(0.01))])


def _energies(sch, n, dt, steps, alpha=0.0):
    h = (1.0 / n[0],) * 3
    o = scheme.Oracle(scheme.Params(n=n, h=h, eps=1.0, Q=0.0, alpha=alpha, dt=dt, stray=False, scheme=sch))
    m = _m0_eq_m0_1(n, h)
    E = [o.energy(m)[4]]
    for _ in range(steps):
        m = o.step(m, 0.0)
        E.append(o.energy(m)[4])
    return np.array(E)


@pytest.mark.parametrize("n", [(64, 1, 1), (16, 6, 4)])
def test_sgspm_exchange_energy_decays_at_zero_damping(n):
    # Sec. 3.2 figures / Sec. 5.2: SGSPM energy decays monotonically for every alpha, incl. 0
    E = _energies("sgspm", n, 1e-2, 300)
    assert np.all(np.diff(E) <= 1e-13 * E[0])
    assert E[-1] < 0.5 * E[0]


@pytest.mark.parametrize("n", [(64, 1, 1), (16, 6, 4)])
def test_gspm_exchange_energy_rises_at_zero_damping(n):
    # Sec. 3.1 figures: GSPM energy rises (and oscillates) at alpha = 0
    E = _energies("gspm", n, 1e-2, 300)
    assert np.sum(np.diff(E) > 1e-10 * E[0]) > 10


def test_heat_and_stray_evaluation_counts():
    # cost difference between the schemes is the number of heat solves (Sec. 5.1, after Table 5)
    rng = np.random.default_rng(5)
    n = (4, 4, 2)
    counts = {}
    for sch in ("sgspm", "gspm"):
        o = scheme.Oracle(full_params(n, scheme=sch))
        calls = [0]
        S0 = o.S

        def S(r, c, S0=S0, calls=calls):
            calls[0] += 1
            return S0(r, c)
        o.S = S
        o.step(random_unit(rng, n), 0.0)
        counts[sch] = (calls[0], o.stray_evals)
    assert counts["sgspm"] == (9, 6) and counts["gspm"] == (7, 4)


def test_refresh_modes_coincide_without_stray_field():
    rng = np.random.default_rng(6)
    n = (5, 4, 2)
    m = random_unit(rng, n)
    a = scheme.Oracle(full_params(n, stray=False, refresh="R1")).run(m, 3)
    b = scheme.Oracle(full_params(n, stray=False, refresh="R2")).run(m, 3)
    assert np.array_equal(a, b)
    a = scheme.Oracle(full_params(n, refresh="R1")).run(m, 3)
    b = scheme.Oracle(full_params(n, refresh="R2")).run(m, 3)
    assert np.abs(a - b).max() > 1e-8


def _manufactured_error(n, dim, dt, alpha=1e-3, sch="sgspm"):
    h = (1.0 / n[0], 1.0 / n[1] if dim == 3 else 1.0, 1.0 / n[2] if dim == 3 else 1.0)
    p = scheme.Params(n=n, h=h, eps=1.0, Q=0.0, alpha=alpha, dt=dt, stray=False, scheme=sch,
                      forcing=scheme.manufactured_forcing(n, h, alpha, dim))
    o = scheme.Oracle(p)
    steps = int(round(1.0 / dt))
    m = o.run(scheme.manufactured_m(n, h, 0.0, dim), steps)
    return m, np.abs(m - scheme.manufactured_m(n, h, steps * dt, dim)).max()


def test_first_order_in_time_1d():
    dts = sorted(PAPER_TABLE3_SGSPM, reverse=True)
    errs = [_manufactured_error((2000, 1, 1), 1, dt)[1] for dt in dts]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 0.9) & (orders < 1.1)), orders
    for dt, e in zip(dts, errs):     # magnitude: same order as Table 3 (forcing placement is a reading)
        assert 0.5 < e / PAPER_TABLE3_SGSPM[dt] < 2.0


def test_first_order_in_time_3d():
    # Table 5 fits one order over dt = 1/32 .. 1/512 (paper: 0.9628); the spatial error
    # at h = 1/16 (~5e-6, Table 6) flattens the finest steps, so fit the same span.
    dts = (1 / 32, 1 / 64, 1 / 512)
    errs = [_manufactured_error((16, 16, 16), 3, dt)[1] for dt in dts]
    order = np.log2(errs[0] / errs[2]) / 4
    assert 0.85 < order < 1.15, errs
    for dt, e in zip(dts, errs):
        assert 0.4 < e / PAPER_TABLE5_SGSPM[dt] < 2.5


def _cauchy_space_order(ns, dim, dt):
    sols = [_manufactured_error(n, dim, dt)[0] for n in ns]
    # cell centres of a grid coincide with the centre cell of each 3-cell block one level finer
    def restrict(u, dim):
        if dim == 1:
            return u[:, :, :, 1::3]
        return u[:, 1::3, 1::3, 1::3]
    d1 = np.abs(sols[0] - restrict(sols[1], dim)).max()
    d2 = np.abs(sols[1] - restrict(sols[2], dim)).max()
    return np.log(d1 / d2) / np.log(3.0)


def test_second_order_in_space_1d():
    order = _cauchy_space_order([(10, 1, 1), (30, 1, 1), (90, 1, 1)], 1, 1e-3)
    assert 1.8 < order < 2.2, order


def test_second_order_in_space_3d():
    order = _cauchy_space_order([(4, 4, 4), (12, 12, 12), (36, 36, 36)], 3, 1e-2)
    assert 1.7 < order < 2.3, order
