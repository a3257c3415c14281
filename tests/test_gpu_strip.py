"""The 512x64x4 strip with a 180-degree Neel wall under an applied field along +x (needs a B300).

m = (tanh((x - x0)/w), sech((x - x0)/w), 0) with w = 4 cells: m_x = -1 on the left, +1 on the
right.  A field along +x favours the right-hand domain, so the wall moves toward -x.  The wall
position is the zero of the y,z-averaged m_x(x), by linear interpolation between cell centres.
  * short runs of both forms against the FP64 oracle (1e-12 FP64, 1e-5 FP32);
  * 60 steps at the least and the most damped alpha of the workload (1e-4, 1e-2) against the
    oracle, at the accuracy targets (1e-12 FP64, 1e-5 FP32; measured 1.7e-14 and 1.9e-8: the
    smooth wall does not amplify rounding);
  * 2000 steps: the wall moves toward -x at every checkpoint, and the FP32 form's position
    agrees with the FP64 form's.
"""
import numpy as np
import pytest

from paper_2606_28113_b300 import inputs, sgspm

from gpu_util import gpu_run, oracle_run

pytestmark = pytest.mark.gpu

W = dict(inputs.WORKLOADS["strip512x64x4_wall"])
KW = {k: W[k] for k in ("n", "h", "eps", "Q", "dt", "u", "he")}


def wall_position(m):
    """Zero of <m_x>_{y,z}(x) in cell units (cell centres at i + 1/2)."""
    mx = m[0].mean(axis=(0, 1))
    s = np.nonzero(np.sign(mx[:-1]) != np.sign(mx[1:]))[0]
    assert len(s) == 1, "expected exactly one sign change of <m_x>"
    i = int(s[0])
    return i + 0.5 + mx[i] / (mx[i] - mx[i + 1])


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_strip_short_run_matches_oracle(fp64, tol):
    m0 = inputs.neel_wall(W["n"])
    ref, _ = oracle_run(m0, steps=5, alpha=1e-2, **KW)
    got = gpu_run(m0, 5, fp64=fp64, alpha=1e-2, **KW)
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("alpha", [1e-4, 1e-2])
def test_strip_60_steps_match_oracle(alpha):
    steps = 60
    m0 = inputs.neel_wall(W["n"])
    ref, _ = oracle_run(m0, steps=steps, alpha=alpha, **KW)
    e64 = np.abs(gpu_run(m0, steps, fp64=True, alpha=alpha, **KW) - ref).max()
    e32 = np.abs(gpu_run(m0, steps, fp64=False, alpha=alpha, **KW) - ref).max()
    print(f"alpha {alpha}: fp64 {e64:.3e}, fp32 {e32:.3e}")
    assert e64 <= 1e-12
    assert e32 <= 1e-5


def test_wall_moves_toward_minus_x():
    m0 = inputs.neel_wall(W["n"])
    x0 = wall_position(m0)
    pos = {}
    for fp64 in (True, False):
        H = sgspm.film(W["n"], W["h"], W["eps"], W["Q"], 1e-2, W["dt"], u=W["u"], he=W["he"], fp64=fp64)
        H.set_m(m0)
        track = []
        for _ in range(4):
            H.step(500)
            track.append(wall_position(H.split(H.get_m())[0]))
        H.close()
        pos[fp64] = np.array(track)
    xs = np.concatenate([[x0], pos[True]])
    assert np.all(np.diff(xs) < 0), xs
    assert x0 - pos[True][-1] > 1.0, xs
    assert np.abs(pos[False] - pos[True]).max() < 1e-2, (pos[False], pos[True])
