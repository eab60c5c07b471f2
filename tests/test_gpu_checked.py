"""The checked build of the library (liblbm_checked.so, compiled with LBM_CHECKED): every
population tile and ghost address its kernels form is tested against the buffer before
use, and one outside would be counted (lbm_check_count) instead of faulting. Every entry
point that moves populations runs on ragged, whole-tile-row, held-x, one-cell,
stochastically rounded, esoteric-twist and batched domains; the count must stay zero and the results
must equal the production build's bit for bit (each build in a child process of its
own)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes, json, os, sys, tempfile
import numpy as np
from paper_2608_13437_gb300 import inputs, lbm

arrays, counts = {}, {}


def count(name, fn, obj):
    c = ctypes.c_ulonglong(0)
    st = fn(obj, ctypes.byref(c))
    counts[name] = int(c.value) if st == lbm.LBM_OK else -st


def domain_case(name, p, store, init, steps, sround=0, prefetch=None):
    d = lbm.Domain(dict(p, stochastic_round=sround), store=store)
    if prefetch is not None:
        d.set_prefetch(prefetch)
    init(d)
    d.step(steps)
    d.step_diag(3)
    d.step(1)  # an odd count of direct steps, then graph replays
    d.step(6)
    diag = d.diag()
    if d.ncell <= 262144:
        st = lbm.LbmDiag()
        lbm.check(lbm.lib().lbm_diag_static(d.handle, ctypes.byref(st)))
    arrays[name + "_pop"] = d.populations("native").view(np.uint16 if store != "f32" else np.uint32)
    arrays[name + "_mom"] = d.moments()
    th, chi, om = d.sensor()
    arrays[name + "_sensor"] = np.stack([th, chi, om])
    arrays[name + "_diag"] = np.array([diag[k] for k in lbm.DIAG_FIELDS])
    if not p.get("streaming"):  # slot planes follow the AA maps
        plane = d.plane_get(0, 5, np.empty((14, d.ny, d.nx), dtype=d.plane_dtype(numpy=True)))
        d.plane_set(0, 5, plane)
    f = d.populations()
    d.set_populations(f)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ck")
        d.save(path)
        d.load(path)
    d.step(2)
    arrays[name + "_end"] = d.populations("native").view(np.uint16 if store != "f32" else np.uint32)
    count(name, lbm.lib().lbm_check_count, d.handle)
    d.close()


tgv = lambda d: d.init_tgv(1.0, 1.25, 1.0)
p = inputs.tgv_params(16)
p.update(nx=37, ny=5, nz=3, dx=2 * np.pi / 37, sutherland=0, f_mu=0.3, J_min=1e-3, tau_R=0.05, tau_q=0.05)
s = inputs.random_smooth_state(37, 5, 3, seed=61, amp=0.15)
domain_case("ragged_f32", p, "f32", lambda d: d.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"]), 7)
q = inputs.tgv_params(16)
q.update(nx=64, ny=8, nz=4, dx=2 * np.pi / 64)
domain_case("rows_f16", q, "f16", tgv, 9, prefetch=3)
domain_case("rows_bf16_sr", q, "bf16", tgv, 5, sround=1)
domain_case("rows_f16_twist", dict(q, streaming=1), "f16", tgv, 9, prefetch=3)
domain_case("ragged_f32_twist", dict(p, streaming=1), "f32",
            lambda d: d.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"]), 7)
domain_case("sod_bf16", inputs.sod_params(64), "bf16",
            lambda d: d.init_riemann(0, 32, inputs.SOD_LEFT, inputs.SOD_RIGHT), 11)
domain_case("sod_f32_twist", dict(inputs.sod_params(64), streaming=1), "f32",
            lambda d: d.init_riemann(0, 32, inputs.SOD_LEFT, inputs.SOD_RIGHT), 11)
one = inputs.tgv_params(16)
one.update(nx=1, ny=1, nz=1)
domain_case("one_cell", one, "f32", tgv, 3)
domain_case("one_cell_twist", dict(one, streaming=1), "f32", tgv, 3)
pl = [inputs.tgv_params(n) for n in (16, 24, 32)]
b = lbm.Batch(pl)
b.init_tgv([1.0] * 3, [1.25, 0.9, 0.6], [1.0] * 3)
b.step(4)
b.step_sequential(3)
for j in range(3):
    arrays[f"batch_{j}"] = b.moments(j)
count("batch", lbm.lib().lbm_batch_check_count, b._h)
b.close()
b = lbm.Batch([dict(q, streaming=1) for q in pl], store="f16")
b.init_tgv([1.0] * 3, [1.25, 0.9, 0.6], [1.0] * 3)
b.set_prefetch(2)
b.step(5)
b.step_sequential(2)
for j in range(3):
    arrays[f"batch_twist_{j}"] = b.moments(j)
count("batch_twist", lbm.lib().lbm_batch_check_count, b._h)
b.close()
np.savez(sys.argv[1], **arrays)
print(json.dumps(counts))
"""


@pytest.fixture(scope="module")
def libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13437_gb300 import build
    build.build()
    build.build(variant="checked")


def _run(variant, out):
    env = dict(os.environ, PYTHONPATH=ROOT)
    env.pop("LBM_LIBRARY", None)
    if variant:
        env["LBM_LIBRARY"] = variant
    r = subprocess.run([sys.executable, "-c", SCRIPT, out], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_finds_no_bad_address_and_matches(libs, tmp_path):
    checked = _run("checked", str(tmp_path / "checked.npz"))
    plain = _run("", str(tmp_path / "plain.npz"))
    assert checked and all(v == 0 for v in checked.values()), checked
    assert all(v == -5 for v in plain.values()), plain  # LBM_E_STATE: not a checked build
    a = np.load(tmp_path / "checked.npz")
    b = np.load(tmp_path / "plain.npz")
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k], equal_nan=True), k
