"""The C-ABI library loads, exports every symbol include/sgspm.h declares, and rejects bad
arguments on the host before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_28113_b300 import sgspm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sgspm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgspm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = sgspm.lib()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s


def test_version():
    assert sgspm.lib().sgspm_version() == 102


def _create(grid, eps=0.1, Q=0.1, alpha=0.1, dt=0.01, u=(1.0, 0.0, 0.0)):
    L = sgspm.lib()
    g = sgspm.Grid(*grid)
    ua = np.ascontiguousarray(u, dtype=np.float64)
    h = ctypes.c_void_p()
    rc = L.sgspm_create(ctypes.byref(g), eps, Q, alpha, dt, ua.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        0, None, ctypes.byref(h))
    return rc, h, L.sgspm_last_error(None).decode()


@pytest.mark.parametrize("grid,kw,msg", [
    ((0, 4, 4, 1.0, 1.0, 1.0), {}, "cell counts"),
    ((4, 4, 4, 0.0, 1.0, 1.0), {}, "cell sizes"),
    ((4, 4, 4, 1.0, 1.0, 1.0), {"dt": 0.0}, "dt"),
    ((4, 4, 4, 1.0, 1.0, 1.0), {"alpha": -1.0}, "alpha"),
    ((4, 4, 4, 1.0, 1.0, 1.0), {"u": (0.0, 0.0, 0.0)}, "easy axis"),
    ((4, 4, 4, 1.0, 1.0, 1.0), {"eps": float("nan")}, "eps"),
])
def test_create_rejects_bad_arguments_on_host(grid, kw, msg):
    rc, h, err = _create(grid, **kw)
    assert rc == sgspm.ERR_ARG and h.value is None and msg in err


def test_null_handle_calls_are_rejected():
    L = sgspm.lib()
    assert L.sgspm_step(None, 1) == sgspm.ERR_ARG
    assert L.sgspm_sync(None) == sgspm.ERR_ARG
    assert L.sgspm_destroy(None) == sgspm.OK
    assert L.sgspm_create(None, 0.1, 0.1, 0.1, 0.1, None, 0, None, None) == sgspm.ERR_ARG


def test_null_handle_tuning_and_parameter_calls_are_rejected():
    L = sgspm.lib()
    a = (ctypes.c_double * 1)(0.01)
    r = (ctypes.c_int * 1)(1)
    assert L.sgspm_set_alpha(None, a) == sgspm.ERR_ARG
    assert L.sgspm_xz_classes(None, None, None, 0) == sgspm.ERR_ARG
    assert L.sgspm_set_packing(None, r, 1) == sgspm.ERR_ARG
    assert L.sgspm_xz_threads(None, None, 0) == sgspm.ERR_ARG
    assert L.sgspm_set_packing_threads(None, r, 1) == sgspm.ERR_ARG
    assert L.sgspm_autotune(None, 1, None, 0) == sgspm.ERR_ARG
    assert L.sgspm_heat_tile(None) == sgspm.ERR_ARG
    assert L.sgspm_set_heat_tile(None, 6) == sgspm.ERR_ARG
    assert L.sgspm_test_tc_timeout(None, 1, 0) == sgspm.ERR_ARG
