"""Time series of the supersonic Taylor-Green vortex (Sec. 3.2): kinetic energy and
the solenoidal and dilatational dissipation rates (Eq. 7), computed inside the step
every `every` steps (lbm_step_diag; FP64 global sums).

    python -m paper_2608_13437_gb300.tgv_series --n 256 --steps 20000 --every 100 \
        [--store f32] [--M0 1.25] [--Re 1000] [--out series.json]

Prints one JSON object: the workload, and per sample the step, convective time
t_c = t U0 / L, E_k / (rho0 U0^2), eps_s and eps_d divided by rho_ref = rho0, the
largest Mach number and the largest (|u| + a) dt / dx.
"""
from __future__ import annotations

import argparse
import json
import time


def run(n: int, steps: int, every: int, store: str = "f32", M0: float = 1.25, Re: float = 1000.0,
        U0: float = 1.0, rho0: float = 1.0) -> dict:
    import torch

    from paper_2608_13437_gb300 import inputs, lbm
    torch.cuda.set_device(0)
    p = inputs.tgv_params(n, M0=M0, Re=Re, U0=U0, rho0=rho0)
    dom = lbm.Domain(p, store=store)
    dom.init_tgv(U0, M0, rho0)
    samples = []

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
        # the first of these k steps also computes the diagnostics of the state it reads
        sample(dom.step_diag(k))
        done += k
    sample(dom.diag())  # the final state
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    info = dom.info()
    dom.close()
    return {"workload": f"supersonic TGV {n}^3, M0 {M0}, Re {Re}, store {store}",
            "dt": info["dt"], "steps": steps, "wall_s": round(wall, 2),
            "mlups_including_diagnostics": round(n ** 3 * steps / wall / 1e6, 1),
            "samples": samples}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--store", default="f32", choices=("f32", "f16", "bf16"))
    ap.add_argument("--M0", type=float, default=1.25)
    ap.add_argument("--Re", type=float, default=1000.0)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    res = run(a.n, a.steps, a.every, a.store, a.M0, a.Re)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
