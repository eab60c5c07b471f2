"""The esoteric twist (lbm_params.streaming = 1) on the GPU, through the C ABI.

Under the twist the slots of the -x, -y, -z directions of every cell are stored with
the cell one step along +x, +y, +z; the step kernels read and write the own cell and
one slot of each of the neighbours x + e_x, x + e_y, x + e_z at both parities. The
stored buffer is therefore a fixed permutation of the AA buffer, and everything
computed from it (canonical populations, moments, sensor, diagnostics separate and in
the step) must equal the AA handle's results bit for bit, on whole-tile rows, ragged
rows, held x ends, degenerate widths, every storage type and both rounding modes. The
raw buffers are decoded from the documented tiled layout here and compared through the
permutation itself.
"""
import os
import tempfile

import numpy as np
import pytest

from conftest import make_oracle
from paper_2608_13437_gb300 import inputs

pytestmark = pytest.mark.gpu

NF, NQ, KTILE = 14, 7, 32


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13437_gb300 import build, lbm as L
    build.build()
    L.lib()
    return L


def decode_raw(lbm, dom):
    """Stored elements [k][slot][z][y][x] of the raw buffer: 32-cell tiles of 7 slots,
    each slot holding fields 0-3, 4-7, 8-11 as [lane][4] and fields 12-13 as [lane][2]."""
    wide = dom.store == lbm.STORE_F32
    raw = dom.buffer.cpu().numpy().view(np.uint32 if wide else np.uint16)
    ntile = -(-dom.ncell // KTILE)
    t = raw[: ntile * NQ * NF * KTILE].reshape(ntile, NQ, NF * KTILE)
    out = np.empty((NF, NQ, ntile * KTILE), dtype=raw.dtype)
    for g in range(3):
        blk = t[:, :, g * 4 * KTILE:(g + 1) * 4 * KTILE].reshape(ntile, NQ, KTILE, 4)
        for j in range(4):
            out[4 * g + j] = blk[..., j].transpose(1, 0, 2).reshape(NQ, -1)
    blk = t[:, :, 12 * KTILE:].reshape(ntile, NQ, KTILE, 2)
    for j in range(2):
        out[12 + j] = blk[..., j].transpose(1, 0, 2).reshape(NQ, -1)
    return out[:, :, : dom.ncell].reshape(NF, NQ, dom.nz, dom.ny, dom.nx)


def bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


def run_case(lbm, p, store, init, streaming, sround=0, prefetch=None, tune=False, use_graphs=True):
    d = lbm.Domain(dict(p, stochastic_round=sround, streaming=streaming), store=store,
                   use_graphs=use_graphs)
    if prefetch is not None:
        d.set_prefetch(prefetch)
    init(d)
    r = {}
    d.step(7)  # graph pairs, then a direct odd step
    r["step_diag"] = d.step_diag(3)
    d.step(1)
    if tune:
        d.autotune(1)
    d.step(6)
    d.synchronize()
    r["step"] = d.step_count
    r["pop"] = bits(d.populations("native"))
    r["mom"] = d.moments()
    r["sensor"] = np.stack(d.sensor())
    r["diag"] = d.diag()
    r["raw"] = decode_raw(lbm, d)
    d.close()
    return r


def tgv(d):
    d.init_tgv(1.0, 1.25, 1.0)


def smooth(nx, ny, nz, seed):
    s = inputs.random_smooth_state(nx, ny, nz, seed=seed, amp=0.15)
    return lambda d: d.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"])


def _params(nx, ny, nz, **kw):
    p = inputs.tgv_params(16)
    p.update(nx=nx, ny=ny, nz=nz, dx=2 * np.pi / nx, **kw)
    return p


CASES = {
    "rows_f32_tuned": (lambda: _params(64, 8, 4), "f32", tgv, dict(tune=True)),
    "rows_f32_direct": (lambda: _params(64, 8, 4), "f32", tgv, dict(use_graphs=False)),
    "ragged_f32": (lambda: _params(37, 5, 3, sutherland=0), "f32", smooth(37, 5, 3, 61), {}),
    "rows_f16_prefetch": (lambda: _params(64, 8, 4), "f16", tgv, dict(prefetch=3)),
    "rows_f16_stochastic": (lambda: _params(64, 8, 4), "f16", tgv, dict(sround=1)),
    "rows_bf16": (lambda: _params(96, 4, 4), "bf16", tgv, {}),
    "ragged_bf16_stochastic": (lambda: _params(37, 5, 3), "bf16", smooth(37, 5, 3, 62), dict(sround=1)),
    "thin_row_f32": (lambda: _params(32, 1, 1), "f32", tgv, {}),
    "one_cell_f32": (lambda: _params(1, 1, 1), "f32", tgv, {}),
    "held_x_f32": (lambda: inputs.sod_params(64), "f32",
                   lambda d: d.init_riemann(0, 32, inputs.SOD_LEFT, inputs.SOD_RIGHT), {}),
    "held_x_bf16": (lambda: inputs.sod_params(64), "bf16",
                    lambda d: d.init_riemann(0, 32, inputs.SOD_LEFT, inputs.SOD_RIGHT), {}),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_twist_equals_aa_bit_for_bit(lbm, name):
    mk, store, init, kw = CASES[name]
    p = mk()
    aa = run_case(lbm, p, store, init, 0, **kw)
    eso = run_case(lbm, p, store, init, 1, **kw)
    assert aa["step"] == eso["step"]
    for key in ("pop", "mom", "sensor"):
        assert np.array_equal(aa[key], eso[key]), (name, key)
    for key in ("diag", "step_diag"):
        for f in lbm.DIAG_FIELDS:
            assert aa[key][f] == eso[key][f], (name, key, f)
    # the raw buffers differ exactly by the twist's relabelling
    ra, re_ = aa["raw"], eso["raw"]
    for s in (0, 1, 3, 5):
        assert np.array_equal(re_[:, s], ra[:, s]), (name, s)
    for s, axis in ((2, 3), (4, 2), (6, 1)):  # [k][z][y][x]: x is axis 3
        assert np.array_equal(re_[:, s], np.roll(ra[:, s], 1, axis=axis)), (name, s)
    if min(p["nx"], p["ny"], p["nz"]) > 1:
        assert not np.array_equal(re_, ra)  # the layouts do differ


def test_twist_tgv_against_oracle(lbm, oracle_mod):
    """32^3 supersonic TGV, 100 steps under the twist: within the FP32 bar of the
    FP64 oracle (rel-L2 1e-5 on rho, u, T)."""
    p = inputs.tgv_params(32)
    d = lbm.Domain(dict(p, streaming=1))
    d.init_tgv(1.0, 1.25, 1.0)
    d.step(100)
    gpu = d.primitives()
    d.close()
    o = make_oracle(p)
    o.init_tgv(1.0, 1.25, 1.0)
    o.step(100)
    ref = o.primitives()
    for j, name in ((0, "rho"), (4, "T")):
        err = np.linalg.norm(gpu[j] - ref[j]) / np.linalg.norm(ref[j])
        assert err < 1e-5, (name, err)
    err = np.linalg.norm(gpu[1:4] - ref[1:4]) / np.linalg.norm(ref[1:4])
    assert err < 1e-5, ("u", err)


def test_checkpoints_cross_between_the_maps(lbm):
    """Checkpoints hold canonical populations: a state saved under the twist resumes
    under the AA maps (and back) exactly as an uninterrupted run."""
    p = _params(64, 4, 4)
    ref = lbm.Domain(p)
    ref.init_tgv(1.0, 1.25, 1.0)
    ref.step(9)
    want = bits(ref.populations("native"))
    ref.close()
    a = lbm.Domain(dict(p, streaming=1))
    a.init_tgv(1.0, 1.25, 1.0)
    a.step(5)
    b = lbm.Domain(p)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ck")
        a.save(path)
        b.load(path)
        b.step(2)
        b.save(path)
        a.load(path)
    a.step(2)
    assert np.array_equal(bits(a.populations("native")), want)
    a.close()
    b.close()


def test_populations_set_under_the_twist(lbm):
    """lbm_populations_set writes canonical populations through the twist's map (at the
    handle's own parity): a state copied from an AA handle three steps ahead steps on
    identically."""
    p = _params(37, 5, 3)
    a = lbm.Domain(p)
    a.init_tgv(1.0, 1.25, 1.0)
    a.step(3)
    e = lbm.Domain(dict(p, streaming=1))
    e.init_tgv(1.0, 1.25, 1.0)  # the same Q_ref and storage scales; counter at 0
    e.set_populations(a.populations("native"), native=True)
    a.step(4)
    e.step(4)
    assert np.array_equal(bits(a.populations("native")), bits(e.populations("native")))
    a.close()
    e.close()


@pytest.mark.parametrize("store,sround", [("f32", 0), ("f16", 1), ("bf16", 0)])
def test_batch_under_the_twist_equals_aa_batch(lbm, store, sround):
    """A batch under the twist (TGV cubes with whole-tile rows, 32 and 64; ragged rows,
    20, 33 and 48; rows shorter than a tile, 8) steps bit-identically to the same batch
    under the AA maps, in its persistent launch and in per-domain launches, and its
    diagnostics agree."""
    sizes = [32, 20, 64, 33, 48, 8]
    params, ic = [], []
    for j, n in enumerate(sizes):
        M0 = 0.4 + 0.12 * j
        p = inputs.tgv_params(n, M0=M0, Re=300.0 + 100 * j)
        p.update(stochastic_round=sround)
        params.append(p)
        ic.append(inputs.tgv_init(M0=M0))
    args = ([c["U0"] for c in ic], [c["M0"] for c in ic], [c["rho0"] for c in ic])
    out = {}
    for mode in (0, 1):
        for how in ("persistent", "sequential"):
            b = lbm.Batch([dict(p, streaming=mode) for p in params], store=store)
            b.init_tgv(*args)
            if how == "persistent":
                b.set_prefetch(2)
                b.step(9)
            else:
                b.step_sequential(9)
            b.synchronize()
            out[mode, how] = ([b.moments(d) for d in range(len(sizes))],
                              [b.diag(d) for d in range(len(sizes))])
            b.close()
    ref_q, ref_d = out[0, "persistent"]
    for key, (qs, ds) in out.items():
        for d in range(len(sizes)):
            assert np.array_equal(qs[d], ref_q[d]), (key, d)
            for f in ("sum_rho", "sum_E", "ek_mean", "max_mach", "min_T", "eps_s_raw"):
                assert ds[d][f] == ref_d[d][f], (key, d, f)


def test_twist_refuses_slot_planes_and_staged_forms(lbm):
    d = lbm.Domain(dict(_params(64, 4, 4), streaming=1))
    d.init_tgv(1.0, 1.25, 1.0)
    with pytest.raises(lbm.LbmError, match="INVAL"):
        d.plane_get(0, 5)
    with pytest.raises(lbm.LbmError, match="INVAL"):
        d.set_kernel_config(64, 2)
    d.set_kernel_config(64, 1)  # the plain forms stay available
    d.step(2)
    d.synchronize()
    d.close()
