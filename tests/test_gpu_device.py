"""Handles and batches are bound to the CUDA device that was current when they were
created: every call makes that device current while it runs and gives the caller's
current device back afterwards.

With one GPU the binding is exercised from a second host thread (whose CUDA state is
its own) and by checking that the caller's current device is left as it was; with two
or more GPUs a handle on device 1 is driven while device 0 is current."""
import threading

import numpy as np
import pytest

from paper_2608_13437_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13437_gb300 import build, lbm as L
    build.build()
    L.lib()
    return torch, L


def _run(dom, steps):
    dom.init_tgv(1.0, 1.25, 1.0)
    dom.step(steps)
    d = dom.diag()
    return dom.populations("native").view(np.uint32), d


def test_handle_reports_its_device_and_runs_from_another_thread(env):
    torch, lbm = env
    p = inputs.tgv_params(16)
    a = lbm.Domain(p)
    assert a.info()["device"] == torch.cuda.current_device()
    ref_pop, ref_diag = _run(a, 9)
    b = lbm.Domain(p)
    out = {}

    def worker():
        try:
            out["res"] = _run(b, 9)
            st = lbm.LbmDiag()
            out["static"] = lbm.lib().lbm_diag_static(b.handle, st)
            out["eps"] = st.eps_s_raw
        except Exception as e:  # reported to the main thread
            out["err"] = e

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "err" not in out, out.get("err")
    pop, diag = out["res"]
    assert np.array_equal(pop, ref_pop)
    assert diag["eps_s_raw"] == ref_diag["eps_s_raw"]
    assert out["static"] == lbm.LBM_OK and out["eps"] == ref_diag["eps_s_raw"]
    assert torch.cuda.current_device() == a.info()["device"]
    a.close()
    b.close()


def test_batch_runs_from_another_thread(env):
    torch, lbm = env
    pl = [inputs.tgv_params(n) for n in (16, 24)]
    ref = lbm.Batch(pl)
    ref.init_tgv([1.0, 1.0], [1.25, 0.8], [1.0, 1.0])
    ref.step(6)
    want = [ref.moments(d) for d in range(2)]
    ref.close()
    b = lbm.Batch(pl)
    out = {}

    def worker():
        try:
            b.init_tgv([1.0, 1.0], [1.25, 0.8], [1.0, 1.0])
            b.step(6)
            out["got"] = [b.moments(d) for d in range(2)]
        except Exception as e:
            out["err"] = e

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "err" not in out, out.get("err")
    for g, w in zip(out["got"], want):
        assert np.array_equal(g, w)
    b.close()


def test_handle_on_second_device_while_first_is_current(env):
    torch, lbm = env
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    p = inputs.tgv_params(16)
    ref = lbm.Domain(p, device="cuda:0")
    ref_pop, ref_diag = _run(ref, 5)
    ref.close()
    h = lbm.Domain(p, device="cuda:1")  # makes device 1 current while creating
    assert h.info()["device"] == 1
    torch.cuda.set_device(0)
    pop, diag = _run(h, 5)
    assert torch.cuda.current_device() == 0  # the caller's device is given back
    assert np.array_equal(pop, ref_pop)
    assert diag["eps_s_raw"] == ref_diag["eps_s_raw"]
    h.close()
