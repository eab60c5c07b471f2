"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: every entry point
on small and degenerate grids (one cell, one-cell axes, ragged sizes, held x ends),
in a child process that preloads the ASan runtime and aborts on the first finding."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
from conftest import make_oracle
from paper_2608_13437_gb300 import inputs
from oracle import becker, oracle
assert oracle._SANITIZED
for shape in ((1, 1, 1), (5, 4, 3), (7, 1, 2), (1, 6, 1)):
    p = inputs.tgv_params(8)
    p.update(nx=shape[0], ny=shape[1], nz=shape[2])
    o = make_oracle(p)
    o.init_tgv(1.0, 1.25, 1.0)
    o.step(3)
    o.diag(); o.moments(); o.primitives(); o.sensor()
    f = o.populations()
    o.set_populations(f)
    s = inputs.random_smooth_state(*shape, seed=3, amp=0.1)
    o.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"])
    o.step(2)
    o.diag()
for n in (1, 2, 9):
    o = make_oracle(inputs.sod_params(n, ny=1, nz=2))
    o.init_riemann(0, n // 2, inputs.SOD_LEFT, inputs.SOD_RIGHT)
    o.step(4)
    o.diag(); o.primitives()
b = becker.paper_case()
o = make_oracle(inputs.becker_params(16, ny=1, nz=1))
o.init_state(becker.initial_moments(b, 16, 1, 1, inputs.BECKER_X0))
o.step(5)
o.diag()
Q = np.zeros(14); Q[0] = 1.2; Q[1] = 0.1; Q[4] = 3.0; Q[5:] = 0.01
o.equilibrium_of(Q); o.flux_of(Q); o.closure_of(Q); o.chi_of(0.05)
o.collide_of(o.equilibrium_of(Q))
print("sanitized oracle ok")
"""


def test_oracle_clean_under_asan_and_ubsan():
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True,
                          text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    env = dict(os.environ, LBM_ORACLE_SANITIZED="1", LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1",
               PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    build = subprocess.run([sys.executable, "-c", "from oracle import oracle; oracle.build()"],
                           cwd=ROOT, env=dict(env, LD_PRELOAD=""), capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr
    assert "sanitized oracle ok" in r.stdout
