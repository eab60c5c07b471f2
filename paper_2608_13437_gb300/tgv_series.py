"""Time series of the supersonic Taylor-Green vortex (Sec. 3.2): kinetic energy and
the solenoidal and dilatational dissipation rates (Eq. 7), computed inside the step
every `every` steps (lbm_step_diag; FP64 global sums).

    python -m paper_2608_13437_gb300.tgv_series --n 256 --steps 20000 --every 100 \
        [--store f32] [--M0 1.25] [--Re 1000] [--spectral-every K] [--t-end T]
        [--param NAME=VALUE ...] [--out series.json]

Prints one JSON object: the workload, and per sample the step, convective time
t_c = t U0 / L, E_k / (rho0 U0^2), eps_s and eps_d divided by rho_ref = rho0, the
largest Mach number and the largest (|u| + a) dt / dx. With --spectral-every K, every
K steps (K a multiple of `every`) eps_s and eps_d are also taken spectrally, as the
paper evaluates them (curl and divergence by FFT of the primitive fields, mu_local per
cell). --t-end sets the number of steps to reach that convective time.
"""
from __future__ import annotations

import argparse
import json
import time


def run(n: int, steps: int, every: int, store: str = "f32", M0: float = 1.25, Re: float = 1000.0,
        U0: float = 1.0, rho0: float = 1.0, spectral_every: int = 0, t_end: float = 0.0,
        overrides: dict | None = None) -> dict:
    import math

    import torch

    from paper_2608_13437_gb300 import inputs, lbm, spectral
    torch.cuda.set_device(0)
    p = inputs.tgv_params(n, M0=M0, Re=Re, U0=U0, rho0=rho0)
    p.update(overrides or {})
    dom = lbm.Domain(p, store=store)
    dom.init_tgv(U0, M0, rho0)
    if t_end > 0:
        steps = int(math.ceil(t_end / (dom.dt * U0)))
    samples, spec = [], []

    def spectral_sample(step):
        prim = dom.moments_device(lbm.MOM_PRIM, torch.float64)
        es, ed = spectral.dissipation(prim, p["mu"], p["T_ref"], p["sutherland"], rho0)
        spec.append({"step": step, "t_c": step * dom.dt * U0, "eps_s": es, "eps_d": ed})
        del prim

    def sample(d):
        if d["status"] != lbm.LBM_OK:
            raise RuntimeError(f"non-finite state at step {d['step']:.0f}")
        samples.append({"step": int(d["step"]), "t_c": d["time"] * U0 / 1.0,
                        "E_k": d["ek_mean"] / (rho0 * U0 * U0),
                        "eps_s": d["eps_s_raw"] / rho0, "eps_d": d["eps_d_raw"] / rho0,
                        "max_mach": d["max_mach"], "max_cfl": d["max_cfl"]})

    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        if spectral_every and done % spectral_every == 0:
            spectral_sample(done)
        # the first of these k steps also computes the diagnostics of the state it reads
        sample(dom.step_diag(k))
        done += k
    sample(dom.diag())  # the final state
    if spectral_every:
        spectral_sample(done)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    info = dom.info()
    dom.close()
    out = {"workload": f"supersonic TGV {n}^3, M0 {M0}, Re {Re}, store {store}"
                       + "".join(f", {k} {v}" for k, v in (overrides or {}).items()),
           "dt": info["dt"], "steps": steps, "wall_s": round(wall, 2),
           "mlups_including_diagnostics": round(n ** 3 * steps / wall / 1e6, 1),
           "samples": samples}
    if spectral_every:
        out["spectral"] = spec
    return out


def moving_average(t, v, half):
    """Each sample replaced by the mean of the samples within +-half of its time: takes
    out the sample-to-sample ringing of the dissipation curves (shocklets crossing the
    grid) before peaks are located."""
    out = []
    for ti in t:
        near = [vj for tj, vj in zip(t, v) if abs(tj - ti) <= half]
        out.append(sum(near) / len(near))
    return out


def local_maxima(t, v, window):
    """(t, v) of the samples that are the largest within +-window of t: the peaks of a
    sampled curve, robust to sample-to-sample noise narrower than the window."""
    peaks = []
    for i, (ti, vi) in enumerate(zip(t, v)):
        near = [vj for tj, vj in zip(t, v) if abs(tj - ti) <= window]
        if vi == max(near) and 0 < i < len(t) - 1:
            peaks.append((ti, vi))
    return peaks


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--store", default="f32", choices=("f32", "f16", "bf16"))
    ap.add_argument("--M0", type=float, default=1.25)
    ap.add_argument("--Re", type=float, default=1000.0)
    ap.add_argument("--spectral-every", type=int, default=0)
    ap.add_argument("--t-end", type=float, default=0.0)
    ap.add_argument("--param", action="append", default=[], metavar="NAME=VALUE",
                    help="override one domain parameter (e.g. sensor_mode=1, C_sigma=20)")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    overrides = {}
    for item in a.param:
        name, value = item.split("=", 1)
        overrides[name] = int(value) if value.lstrip("-").isdigit() else float(value)
    res = run(a.n, a.steps, a.every, a.store, a.M0, a.Re, spectral_every=a.spectral_every,
              t_end=a.t_end, overrides=overrides)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
