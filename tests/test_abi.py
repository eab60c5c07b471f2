"""The C ABI on any host: the library loads, exports every function declared in
include/lbm.h, and its host-only validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_2608_13437_gb300 import build, lbm
    build.build()
    return lbm.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_population_bytes_layout(L):
    from paper_2608_13437_gb300 import inputs, lbm
    p = lbm.make_params(inputs.tgv_params(32), "f32")
    assert L.lbm_population_bytes(ctypes.byref(p)) == 98 * 32 ** 3 * 4
    p = lbm.make_params(inputs.tgv_params(32), "f16")
    assert L.lbm_population_bytes(ctypes.byref(p)) == 98 * 32 ** 3 * 2
    # whole tiles of 32 cells
    q = dict(inputs.tgv_params(8))
    q.update(nx=5, ny=3, nz=1)
    p = lbm.make_params(q, "f32")
    assert L.lbm_population_bytes(ctypes.byref(p)) == 98 * 32 * 4
    q.update(nx=33)
    assert L.lbm_population_bytes(ctypes.byref(lbm.make_params(q, "bf16"))) == 4 * 98 * 32 * 2
    q.update(nx=0)
    assert L.lbm_population_bytes(ctypes.byref(lbm.make_params(q, "f32"))) == 0


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 0, "every size"), ("dx", -1.0, "dx"), ("gamma", 1.0, "gamma"),
    ("tau_R", 0.0, "tau_R"), ("omega_min", 2.5, "omega_min"), ("store", 7, "store"),
    ("J_min", -1.0, "J_min"), ("mu", float("nan"), "mu"),
])
def test_create_rejects_invalid_params_before_any_cuda_call(L, field, value, msg):
    from paper_2608_13437_gb300 import inputs, lbm
    q = dict(inputs.tgv_params(8))
    store = "f32"
    if field == "store":
        store = value
    else:
        q[field] = value
    p = lbm.make_params(q, store)
    h = ctypes.c_void_p()
    st = L.lbm_create(ctypes.byref(p), ctypes.byref(h))
    assert st == lbm.LBM_E_INVAL
    assert not h.value
    assert msg in L.lbm_last_error().decode()


def test_null_arguments_are_rejected(L):
    from paper_2608_13437_gb300 import lbm
    assert L.lbm_step(None, 1) == lbm.LBM_E_INVAL
    assert L.lbm_step_diag(None, 1, ctypes.byref(lbm.LbmDiag())) == lbm.LBM_E_INVAL
    assert L.lbm_destroy(None) == lbm.LBM_OK
    assert L.lbm_status_string(4) == b"LBM_E_NONFINITE"
    assert L.lbm_batch_create(0, None, ctypes.byref(ctypes.c_void_p())) == lbm.LBM_E_INVAL
