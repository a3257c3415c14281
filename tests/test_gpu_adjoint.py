"""The hand-written adjoint (sgspm_record / sgspm_grad) against reference gradients (needs a B300).

Loss L = mean_c (m_x(T) - 1)^2 + 1e-3 ||h_e||^2 (squared L2 over all 3n entries); gradients
with respect to the per-cell applied field h_e and the damping alpha.
  * 16x16x2: against autograd through the plain torch FP64 step (oracle/torch_step.py, itself
    pinned to central differences of the numpy oracle), several checkpoint segments.
  * 128x128x4, checkpoints every 50: against central differences of the FP64 GPU forward, step
    1e-8 (FD converges to the adjoint as the step shrinks; at 1e-6 it has not yet converged after
    500 steps from a random texture).  h_e along a random direction over 500 steps; alpha over
    50 steps: after 500 steps dL/dalpha is ~2e4 and FD does not converge before FP64 rounding
    takes over, so alpha is checked there against autograd at 16x16x2 instead.  Target 1e-4
    relative, for both forms after 50 steps and for the FP64 form after 500.
  * After 500 steps from the i.i.d. random texture the trajectory has passed an event whose
    outcome flips under 1e-6 per-step noise (the FP32 form's per-step error on this texture,
    whose increments are O(1) at first): the FP64 forward with such noise ends as far from the
    clean one as the FP32 form does, so the FP32 gradient cannot match the FP64 one there; a
    test measures it.  From a smooth texture (128x128x4,
    Gaussian-smoothed random state) the FP32 form tracks the FP64 trajectory, and its
    500-step gradient is held to 1e-4 of the FP64 central differences.
"""
import numpy as np
import pytest
import torch

from oracle import torch_step
from paper_2606_28113_b300 import inputs, sgspm

pytestmark = pytest.mark.gpu
REG = 1e-3


def dloss_dm(mT, ncell):
    g = np.zeros_like(mT)
    g[0] = 2.0 * (mT[0] - 1.0) / ncell
    return g


def gpu_grad(n, h, kw, alpha, m0, he, steps, K, fp64, stray=True):
    H = sgspm.film(n, h, alpha=alpha, fp64=fp64, stray=stray, **kw)
    H.set_m(m0)
    H.set_he(he)
    H.record(steps, K)
    mT = H.split(H.get_m())[0]
    ncell = int(np.prod(n))
    g_he, g_a = H.grad(dloss_dm(mT, ncell).reshape(-1))
    H.close()
    L = np.mean((mT[0] - 1.0) ** 2) + REG * np.sum(he * he)
    return L, g_he.reshape(3, n[2], n[1], n[0]) + 2 * REG * he, g_a[0]


@pytest.mark.parametrize("stray", [True, False])
def test_fp64_adjoint_matches_torch_autograd(stray):
    n, h = (16, 16, 2), (1 / 16,) * 3
    kw = dict(eps=0.016, Q=6.2e-4, dt=0.01)
    m0 = inputs.random_unit(4, n)
    he = 0.02 * np.random.default_rng(5).normal(size=(3, n[2], n[1], n[0]))
    steps, K = 12, 5
    model = torch_step.TorchSGSPM(n, h, stray=stray, **kw)
    L_ref, g_ref, a_ref = torch_step.reference_gradients(model, m0, he, 0.01, steps, REG)
    L, g, a = gpu_grad(n, h, kw, 0.01, m0, he, steps, K, True, stray)
    assert abs(L - L_ref) <= 1e-12
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    assert abs(a - a_ref) <= 1e-10 * abs(a_ref)


def test_fp32_adjoint_matches_torch_autograd():
    n, h = (16, 16, 2), (1 / 16,) * 3
    kw = dict(eps=0.016, Q=6.2e-4, dt=0.01)
    m0 = inputs.random_unit(4, n)
    he = 0.02 * np.random.default_rng(5).normal(size=(3, n[2], n[1], n[0]))
    model = torch_step.TorchSGSPM(n, h, **kw)
    L_ref, g_ref, a_ref = torch_step.reference_gradients(model, m0, he, 0.01, 12, REG)
    L, g, a = gpu_grad(n, h, kw, 0.01, m0, he, 12, 5, False)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    assert abs(a - a_ref) <= 1e-4 * abs(a_ref)


@pytest.mark.parametrize("steps,check_alpha", [(500, False), (50, True)])
def test_film128x128x4_against_central_differences(steps, check_alpha):
    w = inputs.WORKLOADS["film128x128x4_adjoint"]
    n, h = w["n"], w["h"]
    kw = dict(eps=w["eps"], Q=w["Q"], dt=w["dt"])
    alpha = w["alpha"]
    m0 = inputs.random_unit(w["seed"], n)
    he = 0.01 * np.random.default_rng(7).normal(size=(3, n[2], n[1], n[0]))
    K = 50

    def loss64(he_, alpha_):
        H = sgspm.film(n, h, alpha=alpha_, fp64=True, **kw)
        H.set_m(m0)
        H.set_he(he_)
        H.step(steps)
        mT = H.split(H.get_m())[0]
        H.close()
        return np.mean((mT[0] - 1.0) ** 2) + REG * np.sum(he_ * he_)

    v = np.random.default_rng(8).normal(size=he.shape)
    step = 1e-8
    fd_v = (loss64(he + step * v, alpha) - loss64(he - step * v, alpha)) / (2 * step)
    fd_a = (loss64(he, alpha + step) - loss64(he, alpha - step)) / (2 * step) if check_alpha else None
    for fp64 in (True, False):
        L, g, a = gpu_grad(n, h, kw, alpha, m0, he, steps, K, fp64)
        dv = float(np.sum(g * v))
        print(f"steps={steps} fp64={fp64}: directional {dv:.9e} vs FD {fd_v:.9e}; alpha {a:.9e} vs FD {fd_a}")
        if not fp64 and steps > 50:
            continue        # see test_film128x128x4_random_texture_amplifies_fp32_rounding
        assert abs(dv - fd_v) <= 1e-4 * abs(fd_v)
        if check_alpha:
            assert abs(a - fd_a) <= 1e-4 * abs(fd_a)


def _final_state(n, h, kw, alpha, m0, he, steps, fp64):
    H = sgspm.film(n, h, alpha=alpha, fp64=fp64, **kw)
    H.set_m(m0)
    H.set_he(he)
    H.step(steps)
    mT = H.split(H.get_m())[0]
    H.close()
    return mT


def test_film128x128x4_random_texture_amplifies_fp32_rounding():
    """From the i.i.d. random texture the trajectory passes, near step 420, an event whose outcome
    flips under small per-step perturbations: an FP64 run whose state is perturbed by 1e-6
    relative noise after every step ends O(1) away from the clean run, as the FP32 form does (its
    increments are O(1) in the first steps of this texture, so its per-step error is of that
    size, while 6e-8 noise leaves the outcome unchanged).  The dynamics, not the FP32 adjoint,
    set the FP32 gradient's distance from the FP64 one after 500 steps there."""
    w = inputs.WORKLOADS["film128x128x4_adjoint"]
    n, h = w["n"], w["h"]
    kw = dict(eps=w["eps"], Q=w["Q"], dt=w["dt"])
    steps = 500
    m0 = inputs.random_unit(w["seed"], n)
    he = 0.01 * np.random.default_rng(7).normal(size=(3, n[2], n[1], n[0]))
    ref = _final_state(n, h, kw, w["alpha"], m0, he, steps, True)
    rng = np.random.default_rng(9)
    H = sgspm.film(n, h, alpha=w["alpha"], fp64=True, **kw)
    H.set_m(m0)
    H.set_he(he)
    for _ in range(steps):
        H.step(1)
        m = H.get_m()
        H.set_m(m * (1 + 1e-6 * rng.choice([-1, 1], size=m.shape)))
    noisy = H.split(H.get_m())[0]
    H.close()
    d_noise = np.abs(noisy - ref).max()
    d_fp32 = np.abs(_final_state(n, h, kw, w["alpha"], m0, he, steps, False) - ref).max()
    print(f"{steps} steps, random texture: FP64 with 1e-6 noise every step vs clean {d_noise:.3e}; "
          f"FP32 form vs FP64 {d_fp32:.3e}")
    assert d_noise > 0.1                   # O(1) divergence from 1e-6 per-step noise ...
    assert d_fp32 < 10 * d_noise           # ... of the same order as the FP32 form's


def test_film128x128x4_smooth_texture_fp32_gradient_after_500_steps():
    w = inputs.WORKLOADS["film128x128x4_adjoint"]
    n, h = w["n"], w["h"]
    kw = dict(eps=w["eps"], Q=w["Q"], dt=w["dt"])
    alpha = w["alpha"]
    m0 = inputs.smoothed_random_unit(w["seed"], n, sigma_cells=(10.0, 10.0, 10.0))
    he = 0.01 * np.random.default_rng(7).normal(size=(3, n[2], n[1], n[0]))
    steps, K = 500, 50

    def loss64(he_):
        mT = _final_state(n, h, kw, alpha, m0, he_, steps, True)
        return np.mean((mT[0] - 1.0) ** 2) + REG * np.sum(he_ * he_)

    v = np.random.default_rng(8).normal(size=he.shape)
    step = 1e-8
    fd_v = (loss64(he + step * v) - loss64(he - step * v)) / (2 * step)
    for fp64 in (True, False):
        L, g, a = gpu_grad(n, h, kw, alpha, m0, he, steps, K, fp64)
        dv = float(np.sum(g * v))
        print(f"smooth texture, {steps} steps, fp64={fp64}: directional {dv:.9e} vs FD {fd_v:.9e}")
        assert abs(dv - fd_v) <= 1e-4 * abs(fd_v)


def test_autograd_function_matches_torch_reference():
    """sgspm.trajectory (torch.autograd.Function over record/grad) against autograd through the
    plain torch FP64 step: loss, dL/dh_e per cell and dL/dalpha."""
    n, h = (16, 16, 2), (1 / 16,) * 3
    kw = dict(eps=0.016, Q=6.2e-4, dt=0.01)
    m0 = inputs.random_unit(6, n)
    he0 = 0.02 * np.random.default_rng(7).normal(size=(3, n[2], n[1], n[0]))
    steps, K = 10, 4
    model = torch_step.TorchSGSPM(n, h, **kw)
    L_ref, g_ref, a_ref = torch_step.reference_gradients(model, m0, he0, 0.01, steps, REG)
    H = sgspm.film(n, h, alpha=0.03, fp64=True, **kw)   # alpha is set by the Function's input
    he = torch.tensor(he0.reshape(-1), dtype=torch.float64, device="cuda", requires_grad=True)
    alpha = torch.tensor(0.01, dtype=torch.float64, requires_grad=True)
    mT = sgspm.trajectory(H, m0, he, alpha, steps, K).reshape(3, n[2], n[1], n[0])
    L = torch.mean((mT[0] - 1.0) ** 2) + REG * torch.sum(he * he)
    L.backward()
    H.close()
    assert abs(L.item() - L_ref) <= 1e-12
    g = he.grad.cpu().numpy().reshape(3, n[2], n[1], n[0])
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    assert abs(alpha.grad.item() - a_ref) <= 1e-10 * abs(a_ref)
