"""lbm_diag_static: diagnostics for callers that cannot allocate device memory at
the time they sample them. It must give the same results as lbm_diag, call after
call, from its fixed scratch array, and refuse domains larger than that array.

Kept in a file of its own, collected after the other test files."""
import ctypes

import pytest

from paper_2608_13437_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("sum_rho", "sum_mx", "sum_my", "sum_mz", "sum_E", "ek_mean", "eps_s_raw", "eps_d_raw",
          "max_mach", "max_cfl", "min_rho", "min_T", "nonfinite", "step", "time")


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13437_gb300 import build, lbm as L
    build.build()
    L.lib()
    return L


def _diag(lbm, fn, dom):
    d = lbm.LbmDiag()
    st = getattr(lbm.lib(), fn)(dom.handle, ctypes.byref(d))
    assert st == lbm.LBM_OK, lbm.lib().lbm_last_error().decode()
    return {n: getattr(d, n) for n in FIELDS}


def _same(a, b):
    """Tolerances of the diagnostics tests: 2e-6 relative on sums and extrema,
    1e-4 on the dissipation integrals (here both paths run the same kernels on the
    same state, so the values agree far more closely)."""
    for k in FIELDS:
        rel = 1e-4 if k.startswith("eps") else 2e-6
        assert a[k] == pytest.approx(b[k], rel=rel, abs=1e-300), k


@pytest.mark.parametrize("shape,store", [((40, 36, 20), "f32"), ((64, 64, 64), "f16")])
def test_static_diag_matches_lbm_diag_on_consecutive_calls(lbm, shape, store):
    nx, ny, nz = shape
    p = inputs.tgv_params(32)
    p.update(nx=nx, ny=ny, nz=nz)
    if (nx, ny, nz) != (64, 64, 64):
        p.update(dx=2 * 3.141592653589793 / 40, sutherland=0, f_mu=0.3, tau_R=0.05, tau_q=0.05)
        s = inputs.random_smooth_state(nx, ny, nz, seed=29, amp=0.1)
    dom = lbm.Domain(p, store=store)
    if (nx, ny, nz) == (64, 64, 64):
        dom.init_tgv(1.0, 1.25, 1.0)
    else:
        dom.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"])
    dom.step(7)
    first = _diag(lbm, "lbm_diag_static", dom)
    _same(first, _diag(lbm, "lbm_diag", dom))
    dom.step(5)  # a different state: nothing of the previous call may leak through
    second = _diag(lbm, "lbm_diag_static", dom)
    ref = _diag(lbm, "lbm_diag", dom)
    _same(second, ref)
    assert second["step"] == 12 and first["step"] == 7
    assert second["ek_mean"] != first["ek_mean"]
    dom.close()


def test_static_diag_rejects_domains_above_its_limit(lbm):
    p = inputs.tgv_params(32)
    p.update(nx=65, ny=64, nz=64)
    dom = lbm.Domain(p)
    dom.init_tgv(1.0, 1.25, 1.0)
    d = lbm.LbmDiag()
    st = lbm.lib().lbm_diag_static(dom.handle, ctypes.byref(d))
    assert st == lbm.LBM_E_INVAL
    assert "at most 262144 cells" in lbm.lib().lbm_last_error().decode()
    dom.close()


def test_static_diag_allocates_no_device_memory(lbm):
    """The entry point's contract itself: on a fresh handle that lbm_diag has never
    touched (so its O(cells) scratch does not exist), a call after a first one (which
    may load the kernels and looks up the array's address) leaves the free device
    memory unchanged, while lbm_diag's first call then takes its scratch."""
    import torch
    p = inputs.tgv_params(32)
    p.update(nx=64, ny=64, nz=64)
    dom = lbm.Domain(p)
    dom.init_tgv(1.0, 1.25, 1.0)
    dom.step(3)
    first = _diag(lbm, "lbm_diag_static", dom)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    second = _diag(lbm, "lbm_diag_static", dom)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert second == first
    _same(_diag(lbm, "lbm_diag", dom), second)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1  # lbm_diag allocated its 4 MB of scratch
    dom.close()
