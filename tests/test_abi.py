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
    ("J_min", -1.0, "J_min"), ("mu", float("nan"), "mu"), ("streaming", 2, "streaming"),
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
    assert L.lbm_status_string(7) == b"LBM_E_TIMEOUT"
    assert L.lbm_batch_create(0, None, ctypes.byref(ctypes.c_void_p())) == lbm.LBM_E_INVAL


def test_every_entry_point_rejects_a_null_handle(L):
    """No entry point dereferences a NULL handle or output pointer: each returns
    LBM_E_INVAL (lbm_destroy and lbm_batch_destroy accept NULL) before any CUDA call."""
    from paper_2608_13437_gb300 import lbm
    V = None
    buf = ctypes.create_string_buffer(64)
    d3 = (ctypes.c_double * 3)(1.0, 0.0, 1.0)
    calls = {
        "lbm_get_info": (V, V), "lbm_init_tgv": (V, 1.0, 1.25, 1.0),
        "lbm_init_riemann": (V, 0, 1, d3, d3), "lbm_init_fields": (V, buf, 0, 0),
        "lbm_init_state": (V, buf, 0, 0), "lbm_step": (V, 1), "lbm_synchronize": (V,),
        "lbm_moments": (V, 0, buf, 0, 0), "lbm_sensor": (V, buf, 0, 0), "lbm_diag": (V, V),
        "lbm_step_diag": (V, 1, V), "lbm_diag_static": (V, V),
        "lbm_populations_get": (V, buf, 0, 0), "lbm_populations_set": (V, buf, 0, 0),
        "lbm_save": (V, b"x"), "lbm_load": (V, b"x"), "lbm_autotune": (V, 1, V),
        "lbm_set_kernel_config": (V, 64, 0), "lbm_set_prefetch": (V, 0), "lbm_test_skip_copy": (V,),
        "lbm_plane_get": (V, 0, 0, buf, 0), "lbm_plane_set": (V, 0, 0, buf, 0),
        "lbm_batch_init_tgv": (V, d3, d3, d3), "lbm_batch_step": (V, 1),
        "lbm_batch_step_sequential": (V, 1), "lbm_batch_synchronize": (V,),
        "lbm_batch_moments": (V, 0, 0, buf, 0, 0), "lbm_batch_info": (V, V, 0, V),
        "lbm_batch_autotune": (V, 1, V, V, V, V), "lbm_batch_set_prefetch": (V, 0),
        "lbm_test_encode": (1, 0, V, V, V, 4, V),
        "lbm_check_count": (V, V), "lbm_batch_check_count": (V, V),
        "lbm_batch_diag": (V, 0, V),
    }
    for name, args in calls.items():
        fn = getattr(L, name)
        fn.restype = ctypes.c_int
        assert fn(*args) == lbm.LBM_E_INVAL, name
    assert L.lbm_destroy(None) == lbm.LBM_OK
    assert L.lbm_batch_destroy(None) == lbm.LBM_OK
    declared = set(_declared())
    untested = declared - set(calls) - {"lbm_create", "lbm_destroy", "lbm_batch_create",
                                        "lbm_batch_destroy", "lbm_population_bytes",
                                        "lbm_last_error", "lbm_status_string"}
    assert not untested, untested


def test_encode_hook_validates_before_any_cuda_call(L):
    """lbm_test_encode refuses FP32 storage, a bad rounding mode, a bad count and NULL
    buffers with LBM_E_INVAL; zero pairs is a no-op."""
    from paper_2608_13437_gb300 import lbm
    buf = ctypes.create_string_buffer(64)
    assert L.lbm_test_encode(0, 0, buf, buf, buf, 4, None) == lbm.LBM_E_INVAL
    assert L.lbm_test_encode(1, 2, buf, buf, buf, 4, None) == lbm.LBM_E_INVAL
    assert L.lbm_test_encode(2, 0, buf, buf, buf, -1, None) == lbm.LBM_E_INVAL
    assert L.lbm_test_encode(1, 1, buf, None, buf, 4, None) == lbm.LBM_E_INVAL
    assert L.lbm_test_encode(1, 1, None, None, None, 0, None) == lbm.LBM_OK


def test_batch_and_params_reject_invalid_stochastic_rounding(L):
    """stochastic_round is 0 or 1, and a batch takes one rounding mode for all its
    domains; both are refused before any CUDA call."""
    from paper_2608_13437_gb300 import inputs, lbm
    q = dict(inputs.tgv_params(8), stochastic_round=2)
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(lbm.make_params(q, "f16")), ctypes.byref(h)) == lbm.LBM_E_INVAL
    arr = (lbm.LbmParams * 2)(lbm.make_params(inputs.tgv_params(8), "f16"),
                              lbm.make_params(dict(inputs.tgv_params(8), stochastic_round=1), "f16"))
    b = ctypes.c_void_p()
    assert L.lbm_batch_create(2, arr, ctypes.byref(b)) == lbm.LBM_E_INVAL
    assert b"one rounding mode" in L.lbm_last_error()


def test_batch_rejects_mixed_streaming_maps(L):
    """A batch takes one streaming map for all its domains (its persistent kernel is
    compiled per map): mixed maps are refused before any CUDA call."""
    from paper_2608_13437_gb300 import inputs, lbm
    arr = (lbm.LbmParams * 2)(lbm.make_params(inputs.tgv_params(8), "f32"),
                              lbm.make_params(dict(inputs.tgv_params(8), streaming=1), "f32"))
    b = ctypes.c_void_p()
    assert L.lbm_batch_create(2, arr, ctypes.byref(b)) == lbm.LBM_E_INVAL
    assert not b.value
    assert b"one streaming map" in L.lbm_last_error()


def test_batch_rejects_more_domains_or_wider_rows_than_its_tile_records_hold(L):
    """The batched kernel's per-tile records hold 16-bit domain indices and
    coordinates: a batch of more than 65535 domains, or a domain with nx > 65535, is
    refused before any CUDA call."""
    from paper_2608_13437_gb300 import inputs, lbm
    one = (lbm.LbmParams * 1)(lbm.make_params(inputs.tgv_params(8), "f32"))
    b = ctypes.c_void_p()
    assert L.lbm_batch_create(65536, one, ctypes.byref(b)) == lbm.LBM_E_INVAL
    assert not b.value
    assert b"65535 domains" in L.lbm_last_error()
    wide = dict(inputs.tgv_params(8), nx=65536, ny=1, nz=1)
    arr = (lbm.LbmParams * 2)(lbm.make_params(inputs.tgv_params(8), "f32"),
                              lbm.make_params(wide, "f32"))
    assert L.lbm_batch_create(2, arr, ctypes.byref(b)) == lbm.LBM_E_INVAL
    assert not b.value
    assert b"nx <= 65535" in L.lbm_last_error()


def test_header_compiles_as_c_and_binding_layouts_match(tmp_path):
    """include/lbm.h is plain C (gcc -std=c99) and C++, and the ctypes structures of the
    binding have the sizes and field offsets of the header's structs."""
    import shutil
    import subprocess

    from paper_2608_13437_gb300 import lbm
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"lbm_params": lbm.LbmParams, "lbm_info_t": lbm.LbmInfo,
               "lbm_tune_t": lbm.LbmTune, "lbm_diag_t": lbm.LbmDiag}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe)], check=True)
    cxx = shutil.which("g++")
    if cxx:
        subprocess.run([cxx, "-x", "c++", "-fsyntax-only", "-Wall", "-Werror", "-I", inc, str(src)],
                       check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)
