"""Pins of the reference gradient used for the adjoint (CPU only).

The torch FP64 step must reproduce the numpy oracle step, and its autograd gradient of
L = mean_c (m_x(T) - 1)^2 + 1e-3 ||h_e||^2 with respect to per-cell h_e and alpha must match
central finite differences (step 1e-6) of the numpy oracle, at 16x16x2.
"""
import numpy as np
import pytest
import torch

from oracle import scheme, torch_step
from paper_2606_28113_b300 import inputs

N, H = (16, 16, 2), (1 / 16,) * 3
KW = dict(eps=0.016, Q=6.2e-4, dt=0.01)
ALPHA = 0.01
STEPS = 8


def oracle_loss(m0, he, alpha, steps=STEPS):
    o = scheme.Oracle(scheme.Params(n=N, h=H, alpha=alpha, he=he, **KW))
    mT = o.run(m0.copy(), steps)
    return np.mean((mT[0] - 1.0) ** 2) + 1e-3 * np.sum(he * he)


@pytest.fixture(scope="module")
def setup():
    m0 = inputs.random_unit(4, N)
    he = 0.02 * np.random.default_rng(5).normal(size=(3, N[2], N[1], N[0]))
    model = torch_step.TorchSGSPM(N, H, **KW)
    return m0, he, model


def test_torch_step_equals_numpy_oracle(setup):
    m0, he, model = setup
    o = scheme.Oracle(scheme.Params(n=N, h=H, alpha=ALPHA, he=he, **KW))
    a = o.run(m0.copy(), 3)
    b = model.run(torch.tensor(m0), torch.tensor(he), ALPHA, 3).numpy()
    assert np.abs(a - b).max() < 1e-13


def test_autograd_gradient_matches_central_differences(setup):
    m0, he, model = setup
    L, g_he, g_alpha = torch_step.reference_gradients(model, m0, he, ALPHA, STEPS)
    assert abs(L - oracle_loss(m0, he, ALPHA)) < 1e-13
    step = 1e-6
    fd_a = (oracle_loss(m0, he, ALPHA + step) - oracle_loss(m0, he, ALPHA - step)) / (2 * step)
    assert abs(g_alpha - fd_a) <= 1e-6 * abs(fd_a) + 1e-12
    rng = np.random.default_rng(6)
    # individual entries
    for _ in range(6):
        idx = tuple(rng.integers(s) for s in he.shape)
        hp, hm = he.copy(), he.copy()
        hp[idx] += step
        hm[idx] -= step
        fd = (oracle_loss(m0, hp, ALPHA) - oracle_loss(m0, hm, ALPHA)) / (2 * step)
        assert abs(g_he[idx] - fd) <= 1e-5 * abs(fd) + 1e-11
    # a random direction
    v = rng.normal(size=he.shape)
    fd = (oracle_loss(m0, he + step * v, ALPHA) - oracle_loss(m0, he - step * v, ALPHA)) / (2 * step)
    assert abs(np.sum(g_he * v) - fd) <= 1e-6 * abs(fd)
