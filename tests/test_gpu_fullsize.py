"""Full-size and convergence checks on the GPU:
  * 512^3 TGV in the benchmark's launch configuration against the oracle on a light
    cone: after n steps a cell depends only on cells within n lattice steps, so the
    oracle recomputes a (B + 2n)^3 window of the same initial field and its central
    B^3 cells must match the GPU's (sampled outputs at full size), for FP32 and the
    FP16 and BF16 storage modes;
  * the largest cubes that fit (840^3 FP32, 1024^3 FP16) on light cones, interior and
    across the periodic corner;
  * 512^3: the TMA-staged step form against the plain kernel (bit for bit, on the
    device) and the in-step diagnostics against the separate pass;
  * 512^3: the plain step with and without its L2 prefetch (bit for bit, FP32 and
    FP16, both streaming maps), and the esoteric twist against the AA maps;
  * dissipation time series per storage type against the oracle (64^3, 400 steps),
    and the 16-bit modes' kinetic-energy drift over 5000 steps (128^3) with and without
    stochastic rounding;
  * Sod at 256..2048 cells: shock position, first-order thickness, L1 falling;
  * reduced storage at 128^3 against the FP64 oracle and the FP32 GPU path;
  * Becker's viscous shock against the exact profile, the oracle and Table 3;
  * spectral diagnostics against the oracle's;
  * the paper's TGV (Re 1600) at 256^3: dissipation peak times against Sec. 3.2.
"""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2608_13437_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13437_gb300 import build, lbm as L
    build.build()
    L.lib()
    return L


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("steps,store,bound", [(40, "f32", 1e-5), (41, "f32", 1e-5),
                                               (40, "f16", 2e-3), (41, "bf16", 2e-2)])
def test_tgv_512_light_cone_matches_oracle(lbm, oracle_mod, steps, store, bound):
    """FP32 within the parity bar; the 16-bit storage modes (the bench's FP16 and BF16
    legs) within the bounds their 32^3 error tests state. The benchmark's configuration:
    esoteric-twist streaming, autotuned kernel form."""
    import torch
    n, B = 512, 12
    origin = (100, 250, 400)
    p = inputs.tgv_params(n)
    dom = lbm.Domain(dict(p, streaming=1), store=store)
    dom.init_tgv(1.0, 1.25, 1.0)
    dom.autotune(pairs_per_trial=2)  # the benchmark's configuration; re-init after
    dom.init_tgv(1.0, 1.25, 1.0)
    dom.step(steps)
    dom.synchronize()
    prim = dom.moments_device(lbm.MOM_PRIM, torch.float64)
    x0, y0, z0 = origin
    g = prim[:, z0:z0 + B, y0:y0 + B, x0:x0 + B].cpu().numpy()
    del prim
    dom.close()
    torch.cuda.empty_cache()
    side = B + 2 * steps
    q = dict(p)
    q.update(nx=side, ny=side, nz=side)
    o = make_oracle(q)
    o.init_tgv(1.0, 1.25, 1.0, gn=n, origin=(x0 - steps, y0 - steps, z0 - steps))
    o.step(steps)
    r = o.primitives()[:, steps:steps + B, steps:steps + B, steps:steps + B]
    errs = {"rho": rel_l2(g[0], r[0]), "u": rel_l2(g[1:4], r[1:4]), "T": rel_l2(g[4], r[4])}
    print(f"512^3 {store} light cone after {steps} steps: {errs}")
    assert max(errs.values()) < bound, errs


@pytest.mark.parametrize("store,n,streaming,bound", [("f32", 840, 0, 1e-5), ("f32", 840, 1, 1e-5),
                                                      ("f16", 1024, 1, 2e-3)])
def test_largest_domain_matches_oracle_on_light_cones(lbm, oracle_mod, store, n, streaming, bound):
    """The largest cubes whose populations and a primitive readback fit on the GPU with
    a margin: FP32 at 840^3 (392 B per cell, 216 GiB: 593 M cells, 5.8e10 stored
    values) under either streaming map, and 16-bit storage at 1024^3 (196 B per cell,
    196 GiB: 2^30 cells, 1.05e11 stored values). After 9 steps, windows in the interior
    and across the periodic corner (the highest cell indices, wrapping to the lowest)
    match the oracle's light-cone recomputation at the FP32 tolerance (FP16: the bound of
    the 512^3 light cone). Skipped when the free device memory is short."""
    import torch
    B, steps = 10, 9
    torch.cuda.empty_cache()
    need = n ** 3 * ((392 if store == "f32" else 196) + 6 * 4) + (8 << 30)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB free, {free / 2**30:.0f} GiB available")
    p = inputs.tgv_params(n)
    dom = lbm.Domain(dict(p, streaming=streaming), store=store)
    dom.init_tgv(1.0, 1.25, 1.0)
    dom.step(steps)
    dom.synchronize()
    prim = dom.moments_device(lbm.MOM_PRIM)
    origins = [(400, 123, 777), (n - 4, n - 6, n - 3)]  # interior; across the corner
    got = []
    for x0, y0, z0 in origins:
        ix, iy, iz = [torch.arange(o, o + B, device=prim.device) % n for o in (x0, y0, z0)]
        w = prim.index_select(3, ix).index_select(2, iy).index_select(1, iz)
        got.append(w.double().cpu().numpy())
    del prim
    dom.close()
    torch.cuda.empty_cache()
    side = B + 2 * steps
    q = dict(p)
    q.update(nx=side, ny=side, nz=side)
    for (x0, y0, z0), g in zip(origins, got):
        o = make_oracle(q)
        o.init_tgv(1.0, 1.25, 1.0, gn=n, origin=(x0 - steps, y0 - steps, z0 - steps))
        o.step(steps)
        r = o.primitives()[:, steps:steps + B, steps:steps + B, steps:steps + B]
        errs = {"rho": rel_l2(g[0], r[0]), "u": rel_l2(g[1:4], r[1:4]), "T": rel_l2(g[4], r[4])}
        print(f"{store} {n}^3 light cone at {(x0, y0, z0)}: {errs}")
        assert max(errs.values()) < bound, ((x0, y0, z0), errs)


def test_512_staged_form_and_in_step_diagnostics(lbm):
    """At the benchmark's size (512^3, 134 M cells, 13.2 G population elements, so
    64-bit addressing throughout): the TMA-staged form of the step equals the plain
    kernel bit for bit after an odd number of steps (compared on the device), and the
    diagnostics computed inside a step equal the separate pass on the same state."""
    import torch
    n = 512
    p = inputs.tgv_params(n)
    a = lbm.Domain(p)
    b = lbm.Domain(p)
    b.set_kernel_config(64, 2)
    for d in (a, b):
        d.init_tgv(1.0, 1.25, 1.0)
        d.step(3)
        d.synchronize()
    assert torch.equal(a._buf, b._buf)
    b.close()
    del b
    torch.cuda.empty_cache()
    ref = a.diag()
    got = a.step_diag(1)
    for k in ("max_mach", "max_cfl", "min_rho", "min_T", "nonfinite", "eps_s_raw", "eps_d_raw",
              "step"):
        assert got[k] == ref[k], k
    for k in ("sum_rho", "sum_E", "ek_mean"):
        assert got[k] == pytest.approx(ref[k], rel=1e-11), k
    a.close()


@pytest.mark.parametrize("store,pf,streaming", [("f32", 512, 0), ("f16", 1024, 0),
                                                ("f32", 512, 1), ("f16", 1024, 1)])
def test_512_prefetch_form_is_bitwise_equal(lbm, store, pf, streaming):
    """At 512^3 the plain step with its L2 prefetch (the distance the autotuner picks
    for this size) equals the step without it bit for bit after an odd number of
    steps, compared on the device, under either streaming map."""
    import torch
    p = dict(inputs.tgv_params(512), streaming=streaming)
    a = lbm.Domain(p, store=store)
    b = lbm.Domain(p, store=store)
    a.set_kernel_config(64, 0)
    b.set_kernel_config(64, 0)
    a.set_prefetch(0)
    b.set_prefetch(pf)
    for d in (a, b):
        d.init_tgv(1.0, 1.25, 1.0)
        d.step(3)
        d.synchronize()
    assert torch.equal(a._buf, b._buf)
    a.close()
    b.close()
    del a, b
    torch.cuda.empty_cache()


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_512_twist_equals_aa(lbm, store):
    """At 512^3, each map in its autotuned form, the esoteric twist gives the AA maps'
    zeroth moments (compared on the device) and diagnostics (in the step and separate)
    bit for bit after an odd number of steps."""
    import torch
    p = inputs.tgv_params(512)
    res = []
    for mode in (0, 1):
        d = lbm.Domain(dict(p, streaming=mode), store=store)
        d.init_tgv(1.0, 1.25, 1.0)
        d.autotune(pairs_per_trial=1)
        d.init_tgv(1.0, 1.25, 1.0)
        d.step(5)
        in_step = d.step_diag(2)
        d.synchronize()
        res.append((d.moments_device(lbm.MOM_Q), in_step, d.diag()))
        d.close()
        del d
        torch.cuda.empty_cache()
    (qa, ia, sa), (qe, ie, se) = res
    assert torch.equal(qa, qe)
    for f in lbm.DIAG_FIELDS:
        assert ia[f] == ie[f] and sa[f] == se[f], f
    del res, qa, qe
    torch.cuda.empty_cache()


def test_stochastic_rounding_removes_the_long_run_drift(lbm):
    """Supersonic TGV 128^3 over 5000 steps (t_c 6.8, into the shocklet phase), E_k
    sampled inside the step every 250 steps, against the FP32 path: the largest
    deviation of the 16-bit curves divided by the curve's largest value. Observed:
    FP16 4.9e-3 rounding to nearest, 1.45e-4 with stochastic rounding; BF16 1.4e-2 and
    5.3e-3."""
    from paper_2608_13437_gb300 import tgv_series
    curves = {}
    for store, sr in (("f32", 0), ("f16", 0), ("f16", 1), ("bf16", 0), ("bf16", 1)):
        res = tgv_series.run(128, 5000, 250, store, overrides={"stochastic_round": sr})
        curves[store, sr] = [x["E_k"] for x in res["samples"]]
    ref = curves["f32", 0]
    dev = {k: max(abs(a - b) for a, b in zip(v, ref)) / max(ref) for k, v in curves.items()}
    print("E_k deviation from FP32 over 5000 steps:", dev)
    assert dev["f16", 1] < 5e-4
    assert dev["f16", 0] < 2e-2 and dev["f16", 1] < dev["f16", 0] / 10
    assert dev["bf16", 1] < dev["bf16", 0] < 5e-2


def test_dissipation_curves_per_storage_type(lbm, oracle_mod):
    """Time series of E_k, eps_s and eps_d (Eq. 7), sampled inside the step every 50
    steps over 400 steps of the 64^3 TGV, for each storage type against the FP64
    oracle's; the error is the largest deviation over the curve divided by the curve's
    largest value. Observed: FP32 1e-7..4e-7, FP16 7e-5..2.4e-4, BF16 1.7e-3..1.4e-2."""
    n, every, steps = 64, 50, 400
    p = inputs.tgv_params(n)
    o = make_oracle(p)
    o.init_tgv(1.0, 1.25, 1.0)
    ref = []
    for k in range(steps // every + 1):
        ref.append(o.diag())
        if k < steps // every:
            o.step(every)
    bounds = {"f32": 2e-6, "f16": 1e-3, "bf16": 5e-2}
    for store, bound in bounds.items():
        d = lbm.Domain(p, store=store)
        d.init_tgv(1.0, 1.25, 1.0)
        got = [d.step_diag(every) for _ in range(steps // every)] + [d.diag()]
        d.close()
        assert [g["step"] for g in got] == [r["step"] for r in ref]
        for key in ("ek_mean", "eps_s_raw", "eps_d_raw"):
            a = np.array([g[key] for g in got])
            b = np.array([r[key] for r in ref])
            err = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            assert err < bound, (store, key, err)


def test_sod_convergence_gpu(lbm):
    """Sec. 3.1, Tables 2 and 4: the captured shock thickness holds a fixed number of
    cells (w proportional to dx, first order), the shock sits within 1e-3 of the exact
    position and L1(rho) falls with the mesh."""
    from oracle import riemann
    L = riemann.State(*inputs.SOD_LEFT)
    R = riemann.State(*inputs.SOD_RIGHT)
    st = riemann.solve_star(L, R)
    res = []
    for n in (256, 512, 1024, 2048):
        p = inputs.sod_params(n)
        dom = lbm.Domain(p)
        dom.init_riemann(0, n // 2, inputs.SOD_LEFT, inputs.SOD_RIGHT)
        steps = inputs.sod_steps(dom.dt)
        dom.step(steps)
        dom.synchronize()
        rho = dom.primitives()[0, 0, 0]
        t = steps * dom.dt
        dom.close()
        x = (np.arange(n) + 0.5) / n
        re, _, _ = riemann.sample(L, R, (x - 0.5) / t)
        right = x[:-1] > 0.5 + st.u * t + 0.05
        w = (st.rho_R - R.rho) / (np.abs(np.diff(rho)) * n)[right].max()
        mid = 0.5 * (st.rho_R + R.rho)
        i = np.where(right & (rho[:-1] >= mid) & (rho[1:] < mid))[0][-1]
        xs = x[i] + (rho[i] - mid) / (rho[i] - rho[i + 1]) / n
        res.append(dict(n=n, w=w, xs=xs, xe=riemann.shock_position(L, R, t, 0.5),
                        l1=float(np.mean(np.abs(rho - re)))))
    for a, b in zip(res, res[1:]):
        assert 1.6 < a["w"] / b["w"] < 2.5, res
        assert b["l1"] < 0.8 * a["l1"], res
    for r in res[1:]:
        assert abs(r["xs"] - r["xe"]) < 1e-3, res
        assert 3.0 < r["w"] * r["n"] < 9.0, res
    print(res)


def test_reduced_storage_at_128(lbm, oracle_mod):
    """FP16 / BF16 shifted storage with FP32 arithmetic against the FP64 oracle and the
    FP32 GPU path, TGV 128^3 after 60 steps; errors of rho, u, T and of the
    diagnostics are stated (printed) and bounded."""
    n, steps = 128, 60
    p = inputs.tgv_params(n)
    o = make_oracle(p)
    o.init_tgv(1.0, 1.25, 1.0)
    o.step(steps)
    ref = o.primitives()
    dref = o.diag()
    out = {}
    for store in ("f32", "f16", "bf16"):
        d = lbm.Domain(p, store=store)
        d.init_tgv(1.0, 1.25, 1.0)
        d.step(steps)
        g = d.primitives()
        dg = d.diag()
        d.close()
        out[store] = {"rho": rel_l2(g[0], ref[0]), "u": rel_l2(g[1:4], ref[1:4]),
                      "T": rel_l2(g[4], ref[4]),
                      "ek": abs(dg["ek_mean"] / dref["ek_mean"] - 1),
                      "eps_s": abs(dg["eps_s_raw"] / dref["eps_s_raw"] - 1),
                      "eps_d": abs(dg["eps_d_raw"] / dref["eps_d_raw"] - 1)}
    print(out)
    assert max(out["f32"][k] for k in ("rho", "u", "T")) < 1e-5
    assert max(out["f16"][k] for k in ("rho", "u", "T")) < 2e-3
    assert max(out["bf16"][k] for k in ("rho", "u", "T")) < 2e-2
    assert out["f16"]["ek"] < 1e-3 and out["bf16"]["ek"] < 1e-2


def test_becker_gpu_convergence_and_paper_table3(lbm, oracle_mod):
    """Becker's shock on 750, 1500, 3000 x 4 x 4 cells (x ends held): the GPU profile
    matches the oracle's at N = 750 (shock position, mean difference); L1(rho) and L1(p)
    within 25 % of Table 3 at N = 750 and no larger than the paper's beyond; the excess
    thickness w / w_ex - 1 falls at least at first order (Table 2). (At N = 6000 the
    stress and heat-flux relaxation waves, whose speed grows as dt^-1/2 with
    tau_R = tau_q = 5 dt, reach 0.87 of the lattice sound speed under the CFL reading
    used here, and oracle and GPU both diverge.)"""
    import json
    import os

    from oracle import becker
    b = becker.paper_case()
    wex = b.thickness()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    res = []
    for n in (750, 1500, 3000):
        p = inputs.becker_params(n)
        dom = lbm.Domain(p)
        dom.init_state(becker.initial_moments(b, n, 4, 4, inputs.BECKER_X0))
        dt = dom.dt
        steps = int(round(0.2 / dt))
        dom.step(steps)
        dom.synchronize()
        P = dom.primitives()
        dom.close()
        rho = P[0, 0, 0]
        t = steps * dt
        x = (np.arange(n) + 0.5) / n
        rho_e, _, _, _, _, _ = b.lab(x, t, inputs.BECKER_X0)
        w = (b.downstream()[0] - b.rho1) / np.max(np.abs(np.diff(rho)) * n)
        paper = next(r for r in gold["becker_conv"] if r["N"] == n)
        _, _, p_e, _, _, _ = b.lab(x, t, inputs.BECKER_X0)
        res.append(dict(n=n, l1=float(np.mean(np.abs(rho - rho_e))), excess=w / wex - 1,
                        l1p=float(np.mean(np.abs(P[5, 0, 0] - p_e))), paper_l1=paper["L1_rho"],
                        paper_l1p=paper["L1_p"]))
        if n == 750:
            # shocked flow: parity is the shock position (within 1e-3, as for Sod) and a
            # small mean difference; at omega = 2 the undamped modes carry FP32 and FP64
            # rounding apart locally near the front
            o = make_oracle(inputs.becker_params(n, ny=1, nz=1))
            o.init_state(becker.initial_moments(b, n, 1, 1, inputs.BECKER_X0))
            o.step(steps)
            rho_o = o.primitives()[0, 0, 0]
            mid = 0.5 * (b.rho1 + b.downstream()[0])

            def front(r):
                i = np.where((r[:-1] >= mid) & (r[1:] < mid))[0][-1]
                return x[i] + (r[i] - mid) / (r[i] - r[i + 1]) / n

            res[-1]["front_gpu_minus_oracle"] = front(rho) - front(rho_o)
            res[-1]["mean_abs_diff_oracle"] = float(np.mean(np.abs(rho - rho_o)))
            assert abs(front(rho) - front(rho_o)) < 1e-3
            assert np.mean(np.abs(rho - rho_o)) < 1e-3
    print(res)
    assert res[0]["l1"] == pytest.approx(res[0]["paper_l1"], rel=0.25), res
    assert res[0]["l1p"] == pytest.approx(res[0]["paper_l1p"], rel=0.25), res
    for r in res[1:]:
        assert r["l1"] <= 1.25 * r["paper_l1"], r
    for a, c in zip(res, res[1:]):
        assert a["excess"] / c["excess"] > 1.8, res
        assert c["l1"] < 0.7 * a["l1"], res



def test_spectral_diagnostics_match_oracle(lbm, oracle_mod):
    """Device spectral eps_s, eps_d and E(k) (torch.fft on lbm_moments output) of the
    GPU TGV state after 100 steps at 32^3 against the oracle's numpy versions on the
    oracle state."""
    import torch

    from oracle import spectral as ospec
    from paper_2608_13437_gb300 import spectral
    p = inputs.tgv_params(32)
    dom = lbm.Domain(p)
    dom.init_tgv(1.0, 1.25, 1.0)
    dom.step(100)
    prim = dom.moments_device(lbm.MOM_PRIM, torch.float64)
    es, ed = spectral.dissipation(prim, p["mu"], p["T_ref"], True, 1.0)
    k, E = spectral.energy_spectrum(prim[1:4])
    dom.close()
    o = make_oracle(p)
    o.init_tgv(1.0, 1.25, 1.0)
    o.step(100)
    P = o.primitives()
    es_o, ed_o = ospec.dissipation(P[1:4], P[4], p["mu"], p["T_ref"], True, 1.0)
    _, E_o = ospec.energy_spectrum(P[1:4])
    assert es == pytest.approx(es_o, rel=1e-5)
    assert ed == pytest.approx(ed_o, rel=1e-4)
    E = E.cpu().numpy()
    # shells far down the tail sit at the FP32 state's rounding floor (about 1e-10 of
    # the peak for a 1e-7 relative velocity error summed over a shell)
    assert np.allclose(E[:len(E_o)], E_o, rtol=1e-4, atol=1e-9 * E_o.max())


def test_tgv_re1600_dissipation_peaks_match_paper(lbm):
    """Sec. 3.2 at the paper's own TGV parameters (Re 1600, M0 1.25, 256^3, C_sigma 40,
    f_mu 1e-2), run to t_c = 10 with the diagnostics computed inside the step every 50
    steps and Eq. 7 also taken spectrally every 50 steps, as the paper evaluates it: the
    dilatational dissipation peaks near t_c = 2.5 and near t_c = 6.5 and the solenoidal
    one near t_c = 9, the times the paper states (within 0.3, 0.3 and 0.5 t_c). The
    curves ring from sample to sample by up to 10 % (spectral) as shocklets cross the
    grid, so each is averaged over +-0.15 t_c before its peak is located. The ratio of
    the two dilatational peaks depends on how sharply the shocklets are captured and is
    reported, not pinned."""
    import json
    import os

    from paper_2608_13437_gb300 import tgv_series
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")) as fh:
        paper = json.load(fh)["tgv_peaks"]
    res = tgv_series.run(256, 0, 50, Re=1600.0, spectral_every=50, t_end=10.0)

    def peak(samples, key, lo, hi):
        t = [s["t_c"] for s in samples]
        v = tgv_series.moving_average(t, [s[key] for s in samples], 0.15)
        i = max((j for j in range(len(t)) if lo <= t[j] <= hi), key=lambda j: v[j])
        assert lo < t[i] < hi, (key, lo, hi, t[i])  # a maximum inside the window, not at its edge
        return t[i], v[i]

    for name in ("spectral", "samples"):  # spectral (the paper's) and in-step FD
        (t1, e1), (t2, e2) = peak(res[name], "eps_d", 1.5, 4.5), peak(res[name], "eps_d", 4.5, 8.0)
        print(f"{name}: eps_d peaks at t_c {t1:.2f}, {t2:.2f}; early/late {e1 / e2:.3f} "
              f"(paper, spectral: {paper['eps_d_early_over_late']['256']})")
        assert abs(t1 - paper["eps_d_peak_tc"][0]) <= 0.3, (name, t1)
        assert abs(t2 - paper["eps_d_peak_tc"][1]) <= 0.3, (name, t2)
    ts, _ = peak(res["samples"], "eps_s", 6.0, 9.99)
    print(f"eps_s peak at t_c {ts:.2f}")
    assert abs(ts - paper["eps_s_peak_tc"]) <= 0.5, ts
