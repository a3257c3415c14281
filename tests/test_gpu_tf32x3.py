"""The TF32X3 precision form (needs a B300): the short-axis (z) DCTs of the FP32 form as dense
GEMMs on the tensor cores (tcgen05, 3xTF32 split, FP32 accumulation), everything else FP32.

The split keeps ~22 of the 24 bits of each operand, so the form is held to the FP32 form's
bar: within 1e-5 of the FP64 oracle in max |dm| (short runs, and sampled cells of the
256x256x8 film after 20 steps).  Its results must also differ from the FP32 form's (else the
tensor-core path did not run) by no more than FP32-level rounding.
"""
import os

import numpy as np
import pytest

from paper_2606_28113_b300 import inputs, sgspm

from gpu_util import oracle_run

pytestmark = pytest.mark.gpu

BASE = dict(eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01, he=(0.02, 0.0, 0.0))


def run(m0, steps, f, **kw):
    H = sgspm.film(f["n"], f["h"], f["eps"], f["Q"], f["alpha"], f["dt"], u=f.get("u", (1.0, 0.0, 0.0)),
                   he=f["he"], fp64=False, **kw)
    H.set_m(m0)
    H.step(steps)
    m = H.split(H.get_m())[0]
    H.close()
    return m


@pytest.mark.parametrize("n,h", [((128, 16, 4), 1 / 128), ((256, 8, 8), 1 / 256), ((256, 16, 2), 1 / 256),
                                 ((512, 8, 3), 1 / 256)])
def test_tf32x3_matches_oracle_and_differs_from_fp32(n, h):
    f = dict(BASE, n=n, h=(h,) * 3)
    m0 = inputs.random_unit(31, n)
    ref, _ = oracle_run(m0, steps=5, **{k: f[k] for k in ("n", "h", "eps", "Q", "alpha", "dt", "he")})
    a = run(m0, 5, f, tf32x3=True)
    b = run(m0, 5, f)
    assert np.abs(a - ref).max() <= 1e-5
    assert np.abs(b - ref).max() <= 1e-5
    assert not np.array_equal(a, b)
    assert np.abs(a - b).max() <= 1e-5


def test_tf32x3_batch_mixes_tensor_core_and_fp32_classes():
    """One handle with films whose slab pass runs the tensor-core transforms (nx 128, 256) and
    films that keep the FP32 path (nx 96; nz 1)."""
    films = [dict(BASE, n=(128, 8, 4), h=(1 / 128,) * 3), dict(BASE, n=(96, 8, 2), h=(1 / 96,) * 3, alpha=0.03),
             dict(BASE, n=(256, 4, 8), h=(1 / 256,) * 3, he=(-0.01, 0.0, 0.0)), dict(BASE, n=(128, 8, 1), h=(1 / 128,) * 3)]
    m0s = [inputs.random_unit(40 + i, f["n"]) for i, f in enumerate(films)]
    H = sgspm.Handle(films, tf32x3=True)
    H.set_m(np.concatenate([m.reshape(-1) for m in m0s]))
    H.step(4)
    got = H.split(H.get_m())
    H.close()
    for f, m0, g in zip(films, m0s, got):
        ref, _ = oracle_run(m0, steps=4, **{k: f[k] for k in ("n", "h", "eps", "Q", "alpha", "dt", "he")})
        assert np.abs(g - ref).max() <= 1e-5, f["n"]


def test_tf32x3_film256x256x8_sampled_cells_match_oracle():
    gold = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "film256x256x8_20steps.npz"))
    W = inputs.WORKLOADS["film256x256x8_fp32"]
    H = sgspm.film(W["n"], W["h"], W["eps"], W["Q"], W["alpha"], W["dt"], u=W["u"], he=W["he"], tf32x3=True)
    H.set_m(inputs.initial_state(W))
    H.step(int(gold["steps"]))
    m = H.get_m().reshape(3, -1)[:, gold["cells"]]
    E = H.energy()[0]
    H.close()
    assert np.abs(m - gold["m"]).max() <= 1e-5
    assert np.abs(E - gold["energy"][-1]).max() <= 1e-5 * np.abs(gold["energy"][-1]).max()


def test_tf32x3_strip_short_run_matches_oracle():
    W = dict(inputs.WORKLOADS["strip512x64x4_wall"], alpha=1e-2)
    m0 = inputs.neel_wall(W["n"])
    ref, _ = oracle_run(m0, steps=5, **{k: W[k] for k in ("n", "h", "eps", "Q", "alpha", "dt", "u", "he")})
    got = run(m0, 5, W, tf32x3=True)
    assert np.abs(got - ref).max() <= 1e-5


def test_tf32x3_expired_tensor_core_wait_is_reported():
    """Failure detection without a fault: with the test switch set, the slab passes issue no MMA
    and no commit, so every bounded mbarrier wait runs out with nothing in flight; the handle
    then reports SGSPM_ERR_TIMEOUT at the next synchronising call, and the device stays usable."""
    f = dict(BASE, n=(128, 8, 4), h=(1 / 128,) * 3)
    m0 = inputs.random_unit(33, f["n"])
    H = sgspm.film(f["n"], f["h"], f["eps"], f["Q"], f["alpha"], f["dt"], he=f["he"], tf32x3=True)
    H.set_m(m0)
    H.step(1)
    H.sync()
    H.test_tc_timeout(True, wait_limit=1000)
    H.step(1)
    with pytest.raises(sgspm.SGSPMError) as e:
        H.sync()
    assert e.value.code == sgspm.ERR_TIMEOUT
    H.test_tc_timeout(False)
    H.close()
    # a fresh handle on the same device computes correct results
    ref, _ = oracle_run(m0, steps=3, **{k: f[k] for k in ("n", "h", "eps", "Q", "alpha", "dt", "he")})
    assert np.abs(run(m0, 3, f, tf32x3=True) - ref).max() <= 1e-5


def test_tc_timeout_switch_needs_the_tensor_core_form():
    f = dict(BASE, n=(16, 8, 2), h=(1 / 16,) * 3)
    H = sgspm.film(f["n"], f["h"], f["eps"], f["Q"], f["alpha"], f["dt"], he=f["he"])
    with pytest.raises(sgspm.SGSPMError) as e:
        H.test_tc_timeout(True)
    assert e.value.code == sgspm.ERR_STATE
    H.close()
