"""Times every form of the fused step kernel on one TGV domain (the candidates the
autotuner chooses from): variants 0 and 1 at blocks of 64 and 128 threads, each with
L2 prefetch distances of 0, 512, 1024 and 2048 tiles, and the shared-memory-staged
variants 2-4 where the domain allows them.

    python -m paper_2608_13437_gb300.forms [--n 512] [--stores f16,f32] [--steps 40]
        [--form VARIANT,BLOCK,PREFETCH]   (time that one form only)

Prints one JSON line: milliseconds per step for each (storage, variant, block).
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--stores", default="f16,f32")
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--form", default="", help="VARIANT,BLOCK,PREFETCH: time this form only")
    a = ap.parse_args(argv)
    import torch
    from . import build, inputs, lbm
    build.build()
    p = inputs.tgv_params(a.n)
    out = {"n": a.n, "steps": a.steps, "ms_per_step": {}}
    forms = [(v, bx, pf) for v in (0, 1) for bx in (64, 128) for pf in (0, 512, 1024, 2048)]
    forms += [(2, 0, 0), (3, 0, 0), (4, 0, 0)]
    if a.form:
        forms = [tuple(int(v) for v in a.form.split(","))]
    for store in a.stores.split(","):
        d = lbm.Domain(p, store=store)
        d.init_tgv(1.0, 1.25, 1.0)
        for var, bx, pf in forms:
            if var >= 2 and a.n % 32:
                continue
            d.set_kernel_config(bx or 64, var)
            d.set_prefetch(pf)
            d.step(a.warmup)
            d.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(d.stream)
            d.step(a.steps)
            t1.record(d.stream)
            torch.cuda.synchronize()
            d.synchronize()
            key = f"{store} variant {var}" + (f" block {bx} prefetch {pf}" if var < 2 else "")
            out["ms_per_step"][key] = round(t0.elapsed_time(t1) / a.steps, 4)
        d.close()
        del d
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
