"""CUDA path vs the FP64 oracle, element by element, on seeded inputs (needs a B300).

Tolerances: the FP64 GPU path must match the oracle within 1e-12 in max |dm|; the FP32
path within 1e-5 (the accuracy targets of the FP64 and FP32 forms of the hot path).
"""
import numpy as np
import pytest

from oracle import demag, scheme
from paper_2606_28113_b300 import inputs, sgspm

from gpu_util import gpu_handle, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

C1 = dict(n=(32, 32, 4), h=(1 / 32,) * 3, eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01)


def _ulp_sensitivity(m0, steps, rel=2.2e-16, **kw):
    """How far the oracle's own trajectory moves when its input is perturbed by `rel` (1 ulp)."""
    rng = np.random.default_rng(1)
    a, _ = oracle_run(m0, steps=steps, **kw)
    b, _ = oracle_run(m0 * (1 + rel * rng.choice([-1, 1], size=m0.shape)), steps=steps, **kw)
    return a, np.abs(a - b).max()


def test_fp64_film32x32x4_short_run_within_1e12():
    m0 = inputs.random_unit(0, C1["n"])
    ref, _ = oracle_run(m0, steps=40, **C1)
    got = gpu_run(m0, 40, **C1)
    assert np.abs(got - ref).max() <= 1e-12


def test_fp64_film32x32x4_200_steps_within_rounding_amplification():
    # From an i.i.d. random unit state the dynamics amplify rounding: the oracle itself moves
    # by ~5e-11 after 200 steps when its input changes by 1 ulp.  The GPU path (different
    # rounding order, delta form) must stay within 10x of that sensitivity.
    m0 = inputs.random_unit(0, C1["n"])
    ref, sens = _ulp_sensitivity(m0, 200, **C1)
    got = gpu_run(m0, 200, **C1)
    assert np.abs(got - ref).max() <= 10 * sens


@pytest.mark.xfail(strict=True, reason="unmet target: 8.6e-11 after 200 steps; the oracle itself moves 5e-11 "
                                       "under a 1-ulp change of its input, so no FP64 implementation that rounds "
                                       "differently reaches 1e-12 on this texture")
def test_fp64_film32x32x4_200_steps_at_the_1e12_target():
    # the 200-step run of the 32x32x4 film held to the stated FP64 target itself
    m0 = inputs.random_unit(0, C1["n"])
    ref, _ = oracle_run(m0, steps=200, **C1)
    got = gpu_run(m0, 200, **C1)
    assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("n", [(12, 10, 3), (24, 20, 1), (40, 1, 1), (6, 15, 5), (96, 8, 2), (5, 4, 2), (1, 9, 4)])
def test_fp64_ragged_sizes_match_oracle(n):
    # sizes with factors 3 and 5, odd and size-1 axes, and tiles with ragged tails
    kw = dict(n=n, h=(1.0 / n[0], 0.8 / n[0], 1.2 / n[0]), eps=0.02, Q=0.05, alpha=0.03, dt=0.005,
              u=(0.6, 0.0, 0.8), he=(0.01, -0.02, 0.005))
    m0 = inputs.random_unit(3, n)
    ref, _ = oracle_run(m0, steps=12, **kw)
    got = gpu_run(m0, 12, **kw)
    assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("sch,refresh,stray", [("gspm", "R1", True), ("sgspm", "R2", True), ("gspm", "R2", True),
                                               ("sgspm", "R1", False), ("gspm", "R1", False)])
def test_fp64_scheme_variants_match_oracle(sch, refresh, stray):
    n = (16, 12, 4)
    kw = dict(n=n, h=(1 / 16,) * 3, eps=0.016, Q=0.01, alpha=0.02, dt=0.01)
    m0 = inputs.random_unit(5, n)
    ref, _ = oracle_run(m0, steps=20, stray=stray, sch=sch, refresh=refresh, **kw)
    got = gpu_run(m0, 20, scheme=sch, refresh=refresh, stray=stray, **kw)
    assert np.abs(got - ref).max() <= 1e-12


def test_fp64_energy_and_stray_field_match_oracle():
    n = (20, 16, 4)
    kw = dict(n=n, h=(0.05, 0.05, 0.05), eps=0.016, Q=0.03, alpha=0.01, dt=0.01, u=(0.0, 1.0, 0.0), he=(0.02, 0.01, -0.03))
    m0 = inputs.random_unit(7, n)
    H = gpu_handle(**kw)
    H.set_m(m0)
    o = scheme.Oracle(scheme.Params(**kw))
    hs = H.split(H.get_hs())[0]
    assert np.abs(hs - o.h_s(m0)).max() <= 1e-13
    E = H.energy()[0]
    Eo = o.energy(m0)
    assert np.abs(E - Eo).max() <= 1e-12 * np.abs(Eo).max()
    H.close()


def test_fp64_per_cell_applied_field_matches_oracle():
    n = (16, 8, 2)
    rng = np.random.default_rng(11)
    he = 0.05 * rng.normal(size=(3, 2, 8, 16))
    kw = dict(n=n, h=(1 / 16,) * 3, eps=0.016, Q=0.01, alpha=0.02, dt=0.01)
    m0 = inputs.random_unit(9, n)
    ref, _ = oracle_run(m0, steps=10, he=he, **kw)
    H = gpu_handle(**kw)
    H.set_m(m0)
    H.set_he(he)
    H.step(10)
    got = H.split(H.get_m())[0]
    H.close()
    assert np.abs(got - ref).max() <= 1e-12


def test_fp64_manufactured_forcing_matches_oracle():
    for dim, n in ((1, (64, 1, 1)), (3, (8, 8, 8))):
        h = (1.0 / n[0], 1.0 / n[1] if dim == 3 else 1.0, 1.0 / n[2] if dim == 3 else 1.0)
        kw = dict(n=n, h=h, eps=1.0, Q=0.0, alpha=1e-3, dt=1e-2)
        m0 = scheme.manufactured_m(n, h, 0.0, dim)
        ref, _ = oracle_run(m0, steps=30, stray=False, forcing=scheme.manufactured_forcing(n, h, 1e-3, dim), **kw)
        H = gpu_handle(stray=False, **kw)
        H.set_forcing(sgspm.FORCE_MMS_1D if dim == 1 else sgspm.FORCE_MMS_3D)
        H.set_m(m0)
        H.step(30)
        got = H.split(H.get_m())[0]
        assert abs(H.get_time() - 0.3) < 1e-12
        H.close()
        assert np.abs(got - ref).max() <= 1e-12


def test_fp32_film32x32x4_short_run_within_1e5():
    m0 = inputs.random_unit(0, C1["n"])
    ref, _ = oracle_run(m0, steps=10, **C1)
    got = gpu_run(m0, 10, fp64=False, **C1)
    assert np.abs(got - ref).max() <= 1e-5


def test_fp32_film32x32x4_200_steps_within_rounding_amplification():
    # FP32 rounding (6e-8 relative) amplified like the oracle's own response to a 6e-8 input change
    m0 = inputs.random_unit(0, C1["n"])
    ref, sens = _ulp_sensitivity(m0, 200, rel=6e-8, **C1)
    got = gpu_run(m0, 200, fp64=False, **C1)
    assert np.abs(got - ref).max() <= 10 * sens


def test_unit_length_after_projection():
    m0 = inputs.random_unit(1, C1["n"])
    for fp64, tol in ((True, 1e-15), (False, 1e-6)):
        got = gpu_run(m0, 10, fp64=fp64, **C1)
        assert np.abs(np.linalg.norm(got, axis=0) - 1).max() <= tol


def test_graph_and_direct_launch_agree_bitwise():
    m0 = inputs.random_unit(2, C1["n"])
    a = gpu_run(m0, 7, fp64=False, graph=True, **C1)
    b = gpu_run(m0, 7, fp64=False, graph=False, **C1)
    assert np.array_equal(a, b)


def test_batch_of_uneven_films_matches_per_film_oracle():
    films = [dict(n=(16, 8, 2), h=(1 / 16,) * 3, eps=0.016, Q=6.2e-4, alpha=0.02, dt=0.01, he=(0.03, 0, 0)),
             dict(n=(12, 12, 4), h=(1 / 12,) * 3, eps=0.02, Q=0.01, alpha=0.001, dt=0.01, he=(-0.02, 0, 0)),
             dict(n=(24, 8, 1), h=(1 / 24,) * 3, eps=0.016, Q=6.2e-4, alpha=0.05, dt=0.005, he=(0.0, 0.01, 0))]
    H = sgspm.Handle(films, fp64=True)
    m0s = [inputs.random_unit(20 + i, f["n"]) for i, f in enumerate(films)]
    H.set_m(np.concatenate([m.reshape(-1) for m in m0s]))
    H.step(8)
    gots = H.split(H.get_m())
    E = H.energy()
    H.close()
    for f, m0, got, e in zip(films, m0s, gots, E):
        ref, o = oracle_run(m0, steps=8, **f)
        assert np.abs(got - ref).max() <= 1e-12
        assert np.abs(e - o.energy(ref)).max() <= 1e-12 * np.abs(e).max()


def test_nonfinite_input_is_reported():
    n = (8, 8, 2)
    H = gpu_handle(n=n, h=(0.1,) * 3, eps=0.016, Q=0.0, alpha=0.01, dt=0.01)
    bad = inputs.random_unit(0, n)
    bad[:, 0, 0, 0] = 0.0
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_m(bad)
    assert e.value.code == sgspm.ERR_ARG
    H.set_m(inputs.random_unit(0, n))
    he = np.zeros((3, 2, 8, 8))
    he[1, 1, 3, 4] = np.nan
    H.set_he(he)
    H.step(2)
    with pytest.raises(sgspm.SGSPMError) as e:
        H.sync()
    assert e.value.code == sgspm.ERR_NONFINITE
    H.close()


def test_step_before_set_field_is_a_state_error():
    H = gpu_handle(n=(8, 8, 2), h=(0.1,) * 3, eps=0.016, Q=0.0, alpha=0.01, dt=0.01)
    with pytest.raises(sgspm.SGSPMError) as e:
        H.step(1)
    assert e.value.code == sgspm.ERR_STATE
    H.close()


def test_fp32_batch_with_misaligned_film_matches_oracle():
    # the compile-time slab kernels move four cells per access; a power-of-two film whose pool
    # offset is not a multiple of four (it follows a 15-cell film) runs the runtime-length kernel
    films = [dict(n=(32, 8, 2), h=(1 / 32,) * 3, eps=0.016, Q=0.01, alpha=0.02, dt=0.01, he=(0.02, 0, 0)),
             dict(n=(5, 3, 1), h=(0.2,) * 3, eps=0.016, Q=0.01, alpha=0.05, dt=0.01, he=(0.0, 0.01, 0)),
             dict(n=(16, 8, 2), h=(1 / 16,) * 3, eps=0.02, Q=0.01, alpha=0.001, dt=0.01, he=(-0.02, 0, 0))]
    H = sgspm.Handle(films, fp64=False)
    m0s = [inputs.random_unit(40 + i, f["n"]) for i, f in enumerate(films)]
    H.set_m(np.concatenate([m.reshape(-1) for m in m0s]))
    H.step(6)
    gots = H.split(H.get_m())
    H.close()
    for f, m0, got in zip(films, m0s, gots):
        ref, _ = oracle_run(m0, steps=6, **f)
        assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("fp64", [True, False])
def test_host_pinned_and_device_buffers_give_the_pageable_results(fp64):
    # set_field / get_field read and write page-locked host and device buffers in place (the
    # copy kernels' own loads and stores) and pageable ones through a staging copy: every route
    # must give the same bits, per-film offsets of an uneven batch included
    import torch
    films = [dict(n=(16, 8, 2), h=(1 / 16,) * 3, eps=0.016, Q=6.2e-4, alpha=0.02, dt=0.01, he=(0.03, 0, 0)),
             dict(n=(5, 3, 1), h=(0.2,) * 3, eps=0.016, Q=0.01, alpha=0.05, dt=0.01, he=(0.0, 0.01, 0))]
    m0 = np.concatenate([inputs.random_unit(60 + i, f["n"]).reshape(-1) for i, f in enumerate(films)])
    H = sgspm.Handle(films, fp64=fp64)
    ref = {}
    for dt in (np.float64, np.float32):
        H.set_m(m0.astype(dt))
        H.step(3)
        ref[dt] = H.get_m()
    tdt = {np.float64: torch.float64, np.float32: torch.float32}
    for dt in (np.float64, np.float32):
        src = torch.from_numpy(m0.astype(dt))
        for buf in (src.pin_memory(), src.cuda()):
            H.set_m(buf)
            H.step(3)
            for out in (torch.empty(m0.size, dtype=torch.float64).pin_memory(),
                        torch.empty(m0.size, dtype=torch.float64, device="cuda")):
                assert np.array_equal(H.get_m(out).cpu().numpy(), ref[dt])
            o32 = H.get_m(torch.empty(m0.size, dtype=torch.float32).pin_memory()).numpy()
            assert np.array_equal(o32, H.get_m(np.empty(m0.size, dtype=np.float32)))
            assert np.array_equal(H.get_m(), ref[dt])
    bad = torch.from_numpy(m0.copy())
    bad[7] = float("nan")
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_m(bad.pin_memory())
    assert e.value.code == sgspm.ERR_ARG
    H.close()
