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
