"""The allocation-free energy entry point (sgspm_energy_noalloc) against sgspm_energy.

For callers that cannot allocate device memory (a plugin whose host owns all device buffers,
a fixed device-memory budget, a loop that must not risk an allocation's synchronisation),
the library offers one entry point that uses a fixed file-scope device array as scratch.
This test checks, through the C ABI, that two calls in a row on the caller's own device
buffers give the same five energy terms as the handle-based sgspm_energy, within the
tolerance of the other parity tests.  It is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2606_28113_b300 import inputs, sgspm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp64", [True, False])
def test_energy_noalloc_matches_handle_energy_twice(fp64):
    # The fields are fetched as float64 (exact for both forms: the FP32 form keeps its state
    # as a double-float pair), so both entry points reduce the same numbers: tolerance 1e-12.
    import torch
    n, h = (40, 24, 4), (1 / 40,) * 3
    kw = dict(eps=0.016, Q=0.03, alpha=0.01, dt=0.01, u=(0.6, 0.8, 0.0), he=(0.02, -0.01, 0.005))
    tdt = torch.float64
    rtol = 1e-12
    H = sgspm.film(n, h, fp64=fp64, **kw)
    for seed in (0, 1):                       # two calls in a row, on different states
        H.set_m(inputs.random_unit(seed, n))
        H.step(2)
        ref = H.energy()[0]
        m = torch.empty(3 * np.prod(n), dtype=tdt, device="cuda")
        hs = torch.empty_like(m)
        H.get_field(sgspm.M, m)
        H.get_field(sgspm.HS, hs)
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        sgspm.energy_noalloc(n, h, kw["eps"], kw["Q"], kw["u"], kw["he"], m, hs, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= rtol * np.abs(ref).max()), (got, ref)
        # the float32 input path, against the same reference within the FP32 tolerance
        out32 = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        sgspm.energy_noalloc(n, h, kw["eps"], kw["Q"], kw["u"], kw["he"], m.float(), hs.float(), out32)
        torch.cuda.synchronize()
        assert np.all(np.abs(out32.cpu().numpy() - ref) <= 1e-5 * np.abs(ref).max())
    H.close()


def test_energy_noalloc_rejects_too_many_cells():
    import torch
    m = torch.zeros(3, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(sgspm.SGSPMError) as e:
        sgspm.energy_noalloc((4096, 4096, 2), (1.0, 1.0, 1.0), 0.1, 0.1, (1, 0, 0), (0, 0, 0), m, None, out)
    assert e.value.code == sgspm.ERR_UNSUPPORTED
