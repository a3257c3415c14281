"""Pins of the states at which the oracle evaluates the stray field within one step.

Reading R1 of the scheme (Sec. 3.2, Step 1, with the remark of Sec. 3.1 that h_s is evaluated
at the intermediate m): every g_i is formed from f at the newest state, so the stray field is
refreshed at m^n, A = (m1*, m2^n, m3^n), B = (m1*, m2*, m3^n), C = (m1*, m2*, m3**),
D = (m1*, m2**, m3**) and E = m** (Step 2).  Two independent checks, with the stray field on
and an easy axis off e1 so that every term of f is non-zero:

* a recorder around the oracle's stray operator sees exactly those six states, rebuilt from
  the intermediates of the step, in that order (four for GSPM, two under reading R2);
* Gauss-Seidel means "use the newest value": a component sweep written in place over one
  state array (update m_i from the newest g_j, g_k and m_j, m_k, then re-form g_i at the
  current array) reproduces the oracle's step.  A state built with a stale component (say C
  with m3^n instead of m3**) fails both.
"""
import numpy as np
import pytest

from oracle import scheme


def _random_unit(rng, n):
    m = rng.normal(size=(3, n[2], n[1], n[0]))
    return m / np.linalg.norm(m, axis=0)


def _params(n, **kw):
    base = dict(n=n, h=(0.25, 0.2, 0.3), eps=0.9, Q=0.4, alpha=0.07, dt=0.02, u=(0.36, 0.48, 0.8),
                he=(0.05, -0.02, 0.03), stray=True)
    base.update(kw)
    return scheme.Params(**base)


class _Recorder:
    def __init__(self, op):
        self.op = op
        self.states = []

    def __call__(self, m):
        self.states.append(np.array(m, copy=True))
        return self.op(m)


def _recorded_states(sch, refresh):
    rng = np.random.default_rng(11)
    n = (5, 4, 3)
    o = scheme.Oracle(_params(n, scheme=sch, refresh=refresh))
    rec = _Recorder(o.H)
    o.H = rec
    m = _random_unit(rng, n)
    out = o.step(m, 0.0)
    return m, out, o, rec.states


def test_sgspm_r1_refreshes_at_the_six_states_of_the_two_sweeps():
    m, _, o, got = _recorded_states("sgspm", "R1")
    it = o.last_intermediates
    m1, m2, m3 = m
    want = [
        np.stack([m1, m2, m3]),                            # m^n: g2^n, g3^n
        np.stack([it["m1s"], m2, m3]),                     # A: g1*
        np.stack([it["m1s"], it["m2s"], m3]),              # B: g2*
        np.stack([it["m1s"], it["m2s"], it["m3ss"]]),      # C: g3**
        np.stack([it["m1s"], it["m2ss"], it["m3ss"]]),     # D: g2**
        np.stack([it["m1ss"], it["m2ss"], it["m3ss"]]),    # E = m**: Step 2
    ]
    assert len(got) == len(want)
    for k, (g, w) in enumerate(zip(got, want)):
        assert np.array_equal(g, w), f"stray refresh {k} at the wrong state"
    # every refresh after the first changes exactly one component of the previous state
    changed = [[a for a in range(3) if not np.array_equal(got[k][a], got[k - 1][a])] for k in range(1, 6)]
    assert changed == [[0], [1], [2], [1], [0]]


def test_gspm_r1_and_frozen_refresh_states():
    m, _, o, got = _recorded_states("gspm", "R1")
    assert len(got) == 4
    assert np.array_equal(got[0], m)
    changed = [[a for a in range(3) if not np.array_equal(got[k][a], got[k - 1][a])] for k in range(1, 4)]
    assert changed == [[0], [1], [2]]
    # R2: h_s(m^n) for all of Step 1 and h_s(m**) for Step 2
    m, out, o, got = _recorded_states("sgspm", "R2")
    it = o.last_intermediates
    assert len(got) == 2
    assert np.array_equal(got[0], m)
    assert np.array_equal(got[1], np.stack([it["m1ss"], it["m2ss"], it["m3ss"]]))


def _in_place_step(o, m, sch):
    """One step written as an in-place Gauss-Seidel component sweep over one state array."""
    p = o.p
    x = np.array(m, copy=True)
    g = [None, None, None]

    def form_g(i):
        return o.S(x[i] + p.dt * o.f(x, o.h_s(x))[i], p.eps)

    g[1], g[2] = form_g(1), form_g(2)
    order = [0, 1, 2] if sch == "gspm" else [0, 1, 2, 1, 0]
    for step, i in enumerate(order):
        j, k = (i + 1) % 3, (i + 2) % 3
        x[i] = m[i] + (g[j] * x[k] - g[k] * x[j])
        if step < len(order) - 1:
            g[i] = form_g(i)
    fss = o.f(x, o.h_s(x))
    y = np.stack([o.S(x[i] + p.alpha * p.dt * fss[i], p.alpha * p.eps) for i in range(3)])
    return y / np.sqrt(np.sum(y * y, axis=0))[None]


@pytest.mark.parametrize("sch", ["sgspm", "gspm"])
def test_oracle_step_equals_in_place_gauss_seidel_sweep(sch):
    rng = np.random.default_rng(12)
    n = (6, 5, 3)
    o = scheme.Oracle(_params(n, scheme=sch))
    m = _random_unit(rng, n)
    a = o.step(m, 0.0)
    b = _in_place_step(o, m, sch)
    assert np.abs(a - b).max() < 1e-14
    # the check has teeth: a step whose C state keeps the stale m3^n differs by far more
    if sch == "sgspm":
        it = o.last_intermediates
        bad = np.stack([it["m1s"], it["m2s"], m[2]])
        good = np.stack([it["m1s"], it["m2s"], it["m3ss"]])
        assert np.abs(o.h_s(bad) - o.h_s(good)).max() > 1e-6
