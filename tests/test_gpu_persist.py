"""The persistent ensemble step (SGSPM_PERSISTENT, needs a B300): one launch per step runs every
pass for every film, taking work items from one queue in program order; an item waits only for
its own film's earlier passes (bounded waits on per-film completion counters).

  * The items are the per-pass kernels' own work items, so the step is bitwise the per-pass step,
    for any slab packing and heat tile, with and without the CUDA graph.
  * The 256-film ensemble after 100 steps: spot films (one of each size class) against the FP64
    oracle run on its own.  Random unit textures amplify rounding (their first increments are
    O(1)), so each form is held to the larger of its target (1e-12 FP64, 1e-5 FP32) and ten times
    the oracle's own response to rounding of that form's size: for FP64 a relative change of 2^-52
    of the input (random sign per entry; the rule of the 200-step and 1000-step film tests), for
    FP32 a relative change of 2^-24 after every step, since the FP32 form rounds its state and
    increments in every step.  The FP32 form runs persistent, the FP64 form per-pass.
  * A withheld work item makes the waits behind it run out: the step is abandoned on every CTA,
    the handle reports SGSPM_ERR_TIMEOUT, and the device stays usable.
"""
import numpy as np
import pytest

from paper_2606_28113_b300 import inputs, sgspm

from gpu_util import oracle_noise_response, oracle_response, oracle_run

pytestmark = pytest.mark.gpu

# padded y lengths 64..256 (the register stray pass); x lengths of the 64, runtime (96) and 128 classes
FILMS = [dict(n=(64, 32, 2), h=(1 / 64,) * 3, eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01, he=(0.02, 0, 0)),
         dict(n=(96, 32, 2), h=(1 / 96,) * 3, eps=0.016, Q=6.2e-4, alpha=0.002, dt=0.01, he=(-0.01, 0, 0)),
         dict(n=(128, 64, 4), h=(1 / 128,) * 3, eps=0.016, Q=6.2e-4, alpha=0.03, dt=0.01, he=(0.0, 0.01, 0)),
         dict(n=(64, 64, 2), h=(1 / 64,) * 3, eps=0.016, Q=6.2e-4, alpha=0.001, dt=0.01, he=(0.05, 0, 0))]


def _m0(films, seed0=70):
    return np.concatenate([inputs.random_unit(seed0 + i, f["n"]).reshape(-1) for i, f in enumerate(films)])


def _run(films, m0, steps, setup=None, **kw):
    H = sgspm.Handle(films, **kw)
    H.set_m(m0)
    if setup:
        setup(H)
    H.step(steps)
    m = H.get_m()
    launches = H.launches_per_step()
    H.close()
    return m, launches


def test_persistent_step_is_bitwise_the_per_pass_step():
    m0 = _m0(FILMS)
    base, n_pass = _run(FILMS, m0, 10)
    got, n_pers = _run(FILMS, m0, 10, persistent=True)
    assert n_pass == 24 and n_pers == 1
    assert np.array_equal(got, base)
    nograph, _ = _run(FILMS, m0, 10, persistent=True, graph=False)
    assert np.array_equal(nograph, base)
    packed, _ = _run(FILMS, m0, 10, setup=lambda H: H.set_packing([4] * len(H.xz_classes())), persistent=True)
    assert np.array_equal(packed, base)
    tiled, _ = _run(FILMS, m0, 10, setup=lambda H: H.set_heat_tile(4), persistent=True)
    assert np.array_equal(tiled, base)
    # without the graph, packing and tile changes between steps rebuild the item tables
    H = sgspm.Handle(FILMS, persistent=True, graph=False)
    H.set_m(m0)
    H.step(3)
    H.set_packing([2] * len(H.xz_classes()))
    H.set_packing_threads([64] * len(H.xz_classes()))
    H.step(4)
    H.set_heat_tile(6)
    H.step(3)
    assert H.xz_classes()[0][1] == 2
    assert np.array_equal(H.get_m(), base)
    H.close()


def test_persistent_step_rejects_what_it_does_not_run():
    for kw in (dict(fp64=True), dict(tf32x3=True)):
        with pytest.raises(sgspm.SGSPMError) as e:
            sgspm.Handle(FILMS, persistent=True, **kw)
        assert e.value.code == sgspm.ERR_UNSUPPORTED
    big = dict(FILMS[0], n=(64, 256, 2))                     # padded y length 512
    with pytest.raises(sgspm.SGSPMError) as e:
        sgspm.Handle([big], persistent=True)
    assert e.value.code == sgspm.ERR_UNSUPPORTED
    H = sgspm.Handle(FILMS, persistent=True)
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_forcing(sgspm.FORCE_MMS_3D)
    assert e.value.code == sgspm.ERR_UNSUPPORTED
    H.close()


def _spot_films(films):
    first = {}
    for i, f in enumerate(films):
        first.setdefault(tuple(f["n"]), i)
    return sorted(first.values())


def test_ensemble256_persistent_spot_films_match_oracle_after_100_steps():
    steps = 100
    films = inputs.ensemble(seed=0, nfilm=256)
    m0s = [inputs.random_unit(f["seed"], f["n"]) for f in films]
    m0 = np.concatenate([m.reshape(-1) for m in m0s])
    out = {}
    for name, kw in (("fp32_persistent", dict(persistent=True)), ("fp64", dict(fp64=True))):
        H = sgspm.Handle(films, **kw)
        H.set_m(m0)
        H.step(steps)
        out[name] = H.split(H.get_m())
        H.close()
    keys = ("n", "h", "eps", "Q", "alpha", "dt", "u", "he")
    for i in _spot_films(films):
        kw = {k: films[i][k] for k in keys}
        ref = oracle_run(m0s[i], steps=steps, **kw)[0]
        # the oracle's own response to relative input changes of the two forms' rounding sizes
        s64 = oracle_response(m0s[i], ref, steps, 2.0 ** -52, **kw)
        s32 = oracle_noise_response(m0s[i], ref, steps, 2.0 ** -24, **kw)
        e32 = np.abs(out["fp32_persistent"][i] - ref).max()
        e64 = np.abs(out["fp64"][i] - ref).max()
        print(f"film {i} {films[i]['n']}: fp32 persistent {e32:.3e} (oracle response to 2^-24 every step: {s32:.3e}), "
              f"fp64 {e64:.3e} (oracle response to 2^-52: {s64:.3e})")
        assert e32 <= max(1e-5, 10 * s32)
        assert e64 <= max(1e-12, 10 * s64)


def test_withheld_item_makes_the_waits_run_out():
    m0 = _m0(FILMS)
    H = sgspm.Handle(FILMS, persistent=True)
    H.set_m(m0)
    H.step(1)
    H.sync()
    H.test_persist_wait(withhold=0, wait_limit=20_000_000)   # about 10 ms of clock cycles
    H.step(2)
    with pytest.raises(sgspm.SGSPMError) as e:
        H.sync()
    assert e.value.code == sgspm.ERR_TIMEOUT
    H.close()
    # the device and a new handle are unaffected
    base, _ = _run(FILMS, m0, 3)
    got, _ = _run(FILMS, m0, 3, persistent=True)
    assert np.array_equal(got, base)
