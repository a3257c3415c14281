"""The batched workload: 256 films of uneven size in one handle (needs a B300).

Every launch of a step covers all films through its work list, with per-film eps, Q, alpha,
dt and applied field.  Spot checks: two films of each size class against the FP64 oracle,
run on its own, after a few steps of the whole batch.  The FP64 form must match within 1e-12,
the FP32 form within 1e-5 (the accuracy targets of the two forms).
"""
import numpy as np
import pytest

from paper_2606_28113_b300 import inputs, sgspm

from gpu_util import oracle_run

pytestmark = pytest.mark.gpu

STEPS = 3


def _spot_films(films):
    """Indices of the first two films of every size class."""
    picked = {}
    for i, f in enumerate(films):
        picked.setdefault(tuple(f["n"]), [])
        if len(picked[tuple(f["n"])]) < 2:
            picked[tuple(f["n"])].append(i)
    assert len(picked) == len(inputs.ENSEMBLE_SIZES)
    return sorted(i for v in picked.values() for i in v)


@pytest.fixture(scope="module")
def ensemble():
    films = inputs.ensemble(seed=0, nfilm=256)
    m0s = [inputs.random_unit(f["seed"], f["n"]) for f in films]
    refs = {i: oracle_run(m0s[i], steps=STEPS, **{k: films[i][k] for k in ("n", "h", "eps", "Q", "alpha", "dt",
                                                                            "u", "he")})[0]
            for i in _spot_films(films)}
    return films, m0s, refs


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_ensemble256_spot_films_match_oracle(ensemble, fp64, tol):
    films, m0s, refs = ensemble
    H = sgspm.Handle(films, fp64=fp64)
    H.set_m(np.concatenate([m.reshape(-1) for m in m0s]))
    H.step(STEPS)
    got = H.split(H.get_m())
    H.close()
    for i, ref in refs.items():
        err = np.abs(got[i] - ref).max()
        assert err <= tol, (i, films[i]["n"], err)
    # every film of the batch still has unit-length magnetisation
    for m in got:
        assert np.abs(np.sqrt((m * m).sum(axis=0)) - 1).max() < (1e-13 if fp64 else 1e-6)


def test_packing_and_autotune_leave_results_unchanged():
    """Packing several y rows per slab CTA is a launch-shape choice: results are bitwise the same
    for every packing, and the autotuner restores m (and the step count) after its timing runs."""
    films = [dict(n=(64, 16, 2), h=(1 / 64,) * 3, eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01, he=(0.02, 0, 0)),
             dict(n=(96, 12, 2), h=(1 / 96,) * 3, eps=0.016, Q=6.2e-4, alpha=0.002, dt=0.01, he=(-0.01, 0, 0)),
             dict(n=(128, 8, 4), h=(1 / 128,) * 3, eps=0.016, Q=6.2e-4, alpha=0.03, dt=0.01, he=(0.0, 0.01, 0))]
    m0 = np.concatenate([inputs.random_unit(60 + i, f["n"]).reshape(-1) for i, f in enumerate(films)])

    def run(setup):
        H = sgspm.Handle(films)
        H.set_m(m0)
        info = setup(H)
        H.step(6)
        m = H.get_m()
        H.close()
        return m, info

    base, cls = run(lambda H: H.xz_classes())
    assert all(r == 1 for _, r in cls)
    for rows in (2, 4, 8):
        got, _ = run(lambda H: H.set_packing([rows] * len(cls)))
        assert np.array_equal(got, base), rows
    for rows, th in ((4, 64), (4, 128), (1, 64), (2, 32)):
        def packed(H):
            H.set_packing([rows] * len(cls))
            H.set_packing_threads([th] * len(cls))
            return H.packing_threads()
        got, info = run(packed)
        assert info == [th] * len(cls)
        assert np.array_equal(got, base), (rows, th)
    for tx in (4, 6, 16):
        got, _ = run(lambda H: H.set_heat_tile(tx))
        assert np.array_equal(got, base), tx
    tuned, choice = run(lambda H: H.autotune(2))
    assert np.array_equal(tuned, base)
    assert len(choice) == len(cls) and all(r in (1, 2, 4, 8) for r in choice)


def test_tuning_calls_validate_their_arguments():
    f = dict(n=(64, 16, 2), h=(1 / 64,) * 3, eps=0.016, Q=6.2e-4, alpha=0.01, dt=0.01, he=(0.0, 0, 0))
    g = dict(f, n=(512, 8, 2), h=(1 / 512,) * 3)
    H = sgspm.Handle([f, g])
    with pytest.raises(sgspm.SGSPMError) as e:
        H.autotune(2)                          # m not set
    assert e.value.code == sgspm.ERR_STATE
    H.set_m(np.concatenate([inputs.random_unit(1, f["n"]).reshape(-1), inputs.random_unit(2, g["n"]).reshape(-1)]))
    cls = H.xz_classes()
    assert sorted(k for k, _ in cls) == [64, 512]
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_packing([2] * (len(cls) + 1))    # one entry per class
    assert e.value.code == sgspm.ERR_ARG
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_packing([9] * len(cls))          # rows in 1..8
    assert e.value.code == sgspm.ERR_ARG
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_packing([1 if k == 64 else 2 for k, _ in cls])   # the nx 512 class runs one row per CTA
    assert e.value.code == sgspm.ERR_UNSUPPORTED
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_packing_threads([96] * len(cls))   # 32, 64, 128 or 256
    assert e.value.code == sgspm.ERR_ARG
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_packing_threads([128])             # one entry per class
    assert e.value.code == sgspm.ERR_ARG
    assert H.packing_threads() == [256] * len(cls)
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_packing_threads([64 if k == 64 else 128 for k, _ in cls])   # the nx 512 class cannot be packed
    assert e.value.code == sgspm.ERR_UNSUPPORTED
    with pytest.raises(sgspm.SGSPMError) as e:
        H.set_heat_tile(17)
    assert e.value.code == sgspm.ERR_ARG
    with pytest.raises(sgspm.SGSPMError) as e:
        H.autotune(0)
    assert e.value.code == sgspm.ERR_ARG
    H.close()
