"""Benchmark of the fused compressible-NSF D3Q7 time step (supersonic TGV, 512^3).

python bench.py [--gpus N] [--steps K] [--warmup W] [--n 512] [--store f32] [--impl reference]

One step = one pass of the whole hot path over the grid: per cell, load 98
populations, moments, closure, sensor, collision, store 98 populations in place
(one kernel launch, replayed from CUDA graphs). Inputs (52.6 GB of populations
at 512^3 FP32) are far larger than the 129 MB L2, so no flush is needed between
steps. Prints one JSON line (rank 0).

Multi-GPU: the path has no exchange step between independent problems here, so
N ranks run N replicas (weak scaling): barrier + synchronize around the timed
region, the max time over ranks, value = all ranks' cell updates / that time.

--impl reference times the FP64 CPU oracle on host cores on a bounded sample of
the same workload (a window of the 512^3 TGV per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and achieved HBM GB/s vs peak, 512^3 TGV; FP32 vs FP16-store at stated err"
BYTES_PER_CELL = {"f32": 784, "f16": 392, "bf16": 392}
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ("paper_2608_13437_gb300/csrc/lbm_device.cuh",
                  "paper_2608_13437_gb300/csrc/step_impl.cuh")


def bench_config(n, store, world, streaming=0):
    """The workload as both arms name it (the reference arm runs the oracle on a window
    of this workload per step; its cpu_baseline says which)."""
    ncell = n ** 3
    return {"workload": workload_name(n, streaming), "n": n, "cells": ncell, "store": store,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "populations (%.1f GB) exceed the 129 MB L2; no flush between steps"
                  % (BYTES_PER_CELL[store] / 2 * ncell / 1e9)}


def workload_name(n, streaming=0):
    return (f"supersonic Taylor-Green vortex {n}^3 periodic [0,2pi)^3, gamma 1.4, Pr 0.71, M0 1.25, "
            "Re 1000, uniform T0, Sutherland, C_sigma 40, J_min 1e-2, omega_min 1.987, "
            "tau_R = tau_q = 5e-3, CFL 0.1, 14 fields x D3Q7, in-place "
            + ("esoteric-twist" if streaming else "AA") + " streaming")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(store, ncell, streaming=0):
    """DRAM bytes per launch at ncell cells from the committed ncu counters of a smaller
    capture: the reads per cell scale with the cells, and the in-place step writes back
    every line it reads once its state exceeds L2 (at the small capture part of the
    writes is still dirty in L2 when the kernel ends), so writes = reads. None when the
    kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    ent = d.get(store + ("_esoteric_twist" if streaming else ""))
    if not ent or ent.get("kernel_hash") != kernel_hash():
        return None
    return 2.0 * ent["dram_read_bytes_per_cell"] * ncell


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def reduce_max(x, dist, device):
    """Maximum of a per-rank number over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ncell, steps, ms_max):
    """Whole-job MLUPS: all ranks' cell updates over the slowest rank's time."""
    return world * ncell * steps / (ms_max * 1e-3) / 1e6


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- CPU oracle
def time_oracle(n_global, side, steps, warmup, threads=None):
    """Runs the FP64 oracle on a side^3 window of the n_global^3 TGV; returns
    (MLUPS, seconds, threads)."""
    from oracle.oracle import Oracle, get_threads, set_threads
    from paper_2608_13437_gb300 import inputs
    if threads:
        set_threads(threads)
    p = inputs.tgv_params(n_global)
    p.update(nx=side, ny=side, nz=side)
    q = dict(p)
    o = Oracle(q.pop("nx"), q.pop("ny"), q.pop("nz"), q.pop("dx"), **q)
    o.init_tgv(1.0, 1.25, 1.0, gn=n_global, origin=(0, 0, 0))
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return side ** 3 * steps / dt / 1e6, dt, get_threads()


CPU_WINDOW = 160  # side of the oracle's window of the TGV, as in the reference arm


def cpu_baseline(n_global, budget_s=15.0):
    """Bounded sample: time one step of a 160^3 window (the reference arm's largest
    window), then that window for as many steps as fit in about budget_s seconds."""
    side = CPU_WINDOW
    _, one_step, thr = time_oracle(n_global, side, 1, 0)
    steps = max(1, min(50, int(budget_s / max(one_step, 1e-3))))
    mlups, secs, thr = time_oracle(n_global, side, steps, 1)
    # the same code on one core, on a 64^3 window for about 3 s
    from oracle.oracle import set_threads
    r1, _, _ = time_oracle(n_global, 32, 1, 0, threads=1)
    s1 = max(1, min(20, int(3.0 * r1 * 1e6 / 64 ** 3)))
    one, secs1, _ = time_oracle(n_global, 64, s1, 0, threads=1)
    set_threads(thr)
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
            "sample": f"FP64 oracle, {side}^3 window of the {n_global}^3 TGV, {steps} steps "
                      f"({secs:.1f} s) after 1 warm-up step, OpenMP over z-planes, in a fresh "
                      "process started before any CUDA work (no torch loaded)",
            "single_core": {"value": round(one, 3), "unit": "MLUPS",
                            "sample": f"64^3 window, {s1} steps ({secs1:.1f} s), 1 thread"}}


def cpu_baseline_subprocess(n_global):
    """cpu_baseline() in a fresh interpreter that loads neither torch nor CUDA, run to
    completion before the GPU legs start, so the oracle has the host cores to itself."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only",
                        "--n", str(n_global)], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"CPU baseline failed:\n{r.stdout}\n{r.stderr}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    rate, _, thr = time_oracle(args.n, 32, 2, 0)
    total = args.steps + args.warmup
    side = int((90.0 * rate * 1e6 / max(total, 1)) ** (1.0 / 3.0))
    side = max(8, min(side, 160))
    mlups, secs, thr = time_oracle(args.n, side, args.steps, args.warmup)
    ms = secs * 1e3 / max(args.steps, 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.n, args.store, world, args.streaming),
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
                         "sample": f"FP64 oracle (two-buffer pull streaming, FP64 arithmetic) on a "
                                   f"{side}^3 window of the {args.n}^3 TGV per step"},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def stated_error(store, n=32, steps=100, sround=0):
    """rel-L2 of rho, u, T against the FP64 oracle after `steps` TGV steps at n^3."""
    import numpy as np

    from oracle.oracle import Oracle
    from paper_2608_13437_gb300 import inputs, lbm
    p = inputs.tgv_params(n)
    d = lbm.Domain(dict(p, stochastic_round=sround), store=store)
    d.init_tgv(1.0, 1.25, 1.0)
    d.step(steps)
    g = d.primitives()
    d.close()
    q = dict(p)
    o = Oracle(q.pop("nx"), q.pop("ny"), q.pop("nz"), q.pop("dx"), **q)
    o.init_tgv(1.0, 1.25, 1.0)
    o.step(steps)
    r = o.primitives()

    def rel(a, b):
        return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

    return {"rho": rel(g[0], r[0]), "u": rel(g[1:4], r[1:4]), "T": rel(g[4], r[4]),
            "case": f"TGV {n}^3, {steps} steps, vs FP64 oracle"}


LONG_RUN = (128, 5000, 250)  # TGV size, steps, diagnostic interval of the drift statement


def long_run_curves(store, sround=0):
    """E_k, eps_s, eps_d every LONG_RUN[2] steps over LONG_RUN[1] steps of the TGV at
    LONG_RUN[0]^3, computed inside the step."""
    from paper_2608_13437_gb300 import tgv_series
    n, steps, every = LONG_RUN
    res = tgv_series.run(n, steps, every, store, overrides={"stochastic_round": sround})
    return {k: [x[k] for x in res["samples"]] for k in ("E_k", "eps_s", "eps_d")}


def long_run_error(curves, ref):
    """Largest deviation from the FP32 path's curves over the run, divided by the
    curve's largest value."""
    n, steps, every = LONG_RUN
    out = {k: round(max(abs(a - b) for a, b in zip(curves[k], ref[k])) / max(ref[k]), 8)
           for k in ref}
    out["case"] = (f"TGV {n}^3, {steps} steps, E_k / eps_s / eps_d every {every} steps "
                   "vs the FP32 path (largest deviation / largest value)")
    return out


def time_steps(torch, dom, steps, warmup, dist=None, sampler_index=None):
    stream = dom.stream
    dom.step(warmup)
    dom.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(sampler_index) if sampler_index is not None else None
    if sampler:
        sampler.__enter__()
    a.record(stream)
    dom.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__()
        clocks = sampler.summary()
    if dist:
        dist.barrier()
    ms = a.elapsed_time(b)
    dom.synchronize()
    return ms, clocks


def diag_costs(torch, dom, ms_step, reps=8):
    """GPU time of one separate FP64 diagnostic pass (lbm_diag) and of a step that
    computes the diagnostics itself, against plain steps. lbm_step_diag blocks the
    caller until the diagnostics are on the host: with n = 2 the second step is queued
    behind them and keeps the GPU busy meanwhile (in_step_extra_ms, the GPU cost of the
    diagnostics); with n = 1 the GPU also idles while the host wakes up and issues the
    next call (in_step_extra_with_host_wait_ms)."""
    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record(dom.stream)
        for _ in range(reps):
            fn()
        b.record(dom.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    sep = timed(dom.diag)
    fused = timed(lambda: dom.step_diag(1))
    one = timed(lambda: dom.step(1))  # single plain steps, launched the same way
    fused2 = timed(lambda: dom.step_diag(2))
    two = timed(lambda: dom.step(2))
    return {"plain_step_ms": round(ms_step, 4), "single_plain_step_ms": round(one, 4),
            "separate_diag_ms": round(sep, 4), "step_with_diag_ms": round(fused, 4),
            "two_steps_ms": round(two, 4), "two_steps_first_with_diag_ms": round(fused2, 4),
            "in_step_extra_ms": round(fused2 - two, 4),
            "in_step_extra_with_host_wait_ms": round(fused - one, 4)}


def parity_times(torch, dom, pairs=10):
    """Mean GPU time of the even and of the odd steps (single launches, a CUDA event
    between consecutive steps on the handle's stream)."""
    dom.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * pairs + 1)]
    first_odd = dom.step_count & 1
    ev[0].record(dom.stream)
    for j in range(2 * pairs):
        dom.step(1)
        ev[j + 1].record(dom.stream)
    torch.cuda.synchronize()
    t = [ev[j].elapsed_time(ev[j + 1]) for j in range(2 * pairs)]
    a, b = sum(t[0::2]) / pairs, sum(t[1::2]) / pairs
    even, odd = (b, a) if first_odd else (a, b)
    return {"even_ms": round(even, 4), "odd_ms": round(odd, 4)}


def streaming_leg(torch, lbm, p, store, ncell, steps, warmup, hbm):
    """The two in-place streaming maps on the same workload and storage: autotuned
    form, K steps (CUDA events), and the even and odd step times."""
    out = {"store": store}
    for name, mode in (("aa", 0), ("esoteric_twist", 1)):
        d = lbm.Domain(dict(p, streaming=mode), store=store)
        d.init_tgv(1.0, 1.25, 1.0)
        tune = d.autotune(pairs_per_trial=3)  # advances the state: re-init below
        d.init_tgv(1.0, 1.25, 1.0)
        ms, _ = time_steps(torch, d, steps, max(warmup, 3))
        par = parity_times(torch, d)
        d.close()
        del d
        torch.cuda.empty_cache()
        ach = BYTES_PER_CELL[store] * ncell / (ms / steps * 1e-3) / 1e9
        out[name] = {"value": round(ncell * steps / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                     "ms_per_step": round(ms / steps, 4), "achieved_gbs": round(ach, 1),
                     "frac": round(ach / hbm, 4), "steps": steps, "tune": tune, **par}
    return out


def batch_size_sweep(torch, lbm, inputs, steps, warmup, store, cells=40e6, max_domains=700):
    """Uniform batches of one size each (32^3 ... 128^3 TGV domains, about `cells` cells
    per batch, at most `max_domains` domains): autotuned persistent launches, K steps
    timed with CUDA events."""
    out = []
    for n in (32, 48, 64, 96, 128):
        count = min(max_domains, max(1, int(cells // n ** 3)))
        B = lbm.Batch([inputs.tgv_params(n) for _ in range(count)], store=store)
        ic = [[1.0] * count, [1.25] * count, [1.0] * count]
        B.init_tgv(*ic)
        tune = B.autotune(4)
        B.init_tgv(*ic)
        B.step(warmup)
        B.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(B.stream)
        B.step(steps)
        b.record(B.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        total = count * n ** 3
        out.append({"n": n, "domains": count, "cells": total, "ms_per_step": round(ms, 4),
                    "value": round(total / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                    "achieved_gbs": round(BYTES_PER_CELL[store] * total / (ms * 1e-3) / 1e9, 1),
                    "tune": tune})
        B.close()
        torch.cuda.empty_cache()
    return {"store": store, "batches": out}


def batch_leg(torch, lbm, inputs, steps, warmup, n_domains=64, store="f32", sround=0,
              streaming=0):
    """Independent TGV domains (sizes, M0, Re from SplitMix64(0); 64 by default): one
    persistent launch per step (CUDA graph, autotuned tiles) against one plain launch
    per domain per step."""
    doms = inputs.batch_domains()[:n_domains]
    pl = inputs.batch_params(doms)
    B = lbm.Batch([dict(q, stochastic_round=sround, streaming=streaming) for q, _ in pl],
                  store=store)
    ic = [[c["U0"] for _, c in pl], [c["M0"] for _, c in pl], [c["rho0"] for _, c in pl]]
    B.init_tgv(*ic)
    tune = B.autotune(4)
    cells = B.total_cells()
    out = {"domains": len(doms), "cells": cells, "store": store, "stochastic_round": sround,
           "streaming": "esoteric twist" if streaming else "AA", "tune": tune}
    for name, fn in (("persistent", B.step), ("sequential", B.step_sequential)):
        B.init_tgv(*ic)
        fn(warmup)
        B.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(B.stream)
        fn(steps)
        b.record(B.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        B.synchronize()
        out[name] = {"value": round(cells / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                     "ms_per_step": round(ms, 4),
                     "achieved_gbs": round(BYTES_PER_CELL[store] * cells / (ms * 1e-3) / 1e9, 1)}
    B.close()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2608_13437_gb300 import inputs, lbm

    world, rank, local = dist_setup()
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    n = args.n
    ncell = n ** 3
    p = dict(inputs.tgv_params(n), streaming=args.streaming)
    dom = lbm.Domain(p, store=args.store)
    dom.init_tgv(1.0, 1.25, 1.0)
    tune = dom.autotune(pairs_per_trial=3)   # advances the state: re-init below
    ev_init = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev_init[0].record(dom.stream)
    dom.init_tgv(1.0, 1.25, 1.0)            # FP32 initial equilibrium on the device
    ev_init[1].record(dom.stream)
    torch.cuda.synchronize()
    init_tgv_ms = ev_init[0].elapsed_time(ev_init[1])
    ms_total, clocks = time_steps(torch, dom, args.steps, args.warmup, dist,
                                  sampler_index=dev if rank == 0 else None)
    ms_max = reduce_max(ms_total, dist, "cuda")
    ms_step = ms_max / args.steps
    value = job_value(world, ncell, args.steps, ms_max)
    # two shorter windows on the evolved state: best and median of three, as context
    # for run-to-run spread (the value above is the K-step window alone)
    rep_steps = max(2, min(args.steps, 500) // 2 * 2)
    repeats = [round(value, 1)]
    for _ in range(2):
        ms_r, _ = time_steps(torch, dom, rep_steps, 2, dist)
        repeats.append(round(job_value(world, ncell, rep_steps, reduce_max(ms_r, dist, "cuda")), 1))
    hbm, peak_kind = peaks()
    bpc = BYTES_PER_CELL[args.store]
    achieved = bpc * ncell / (ms_total / args.steps * 1e-3) / 1e9
    traffic = traffic_per_launch(args.store, ncell, args.streaming)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bpc * ncell}

    # end to end through the C ABI: host fields in, K steps with the FP64 diagnostic
    # time series read back every 50 steps, host primitives out.
    fields = torch.from_numpy(inputs.tgv_fields(n, dtype=np.float32)).pin_memory()
    out = torch.empty((6, n, n, n), dtype=torch.float32).pin_memory()
    diag_every = 50
    # one untimed pass of the same calls on the same page-locked buffers (warm-up, as
    # for the steps): the GPU's first accesses to freshly pinned host pages are slower
    # than later ones, a set-up cost of the buffers rather than of a step
    dom.init_fields_device(fields, src_on_device=False)
    dom.step_diag(2)
    dom.moments_into(out, which=lbm.MOM_PRIM, on_device=False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t0 = time.perf_counter()
    ev[0].record(dom.stream)
    dom.init_fields_device(fields, src_on_device=False)
    ev[1].record(dom.stream)
    series = []
    done = 0
    while done < args.steps:
        k = min(diag_every, args.steps - done)
        # the first of these k steps also returns the diagnostics of the state it reads
        series.append(dom.step_diag(k))
        done += k
    ev[2].record(dom.stream)
    dom.moments_into(out, which=lbm.MOM_PRIM, on_device=False)
    ev[3].record(dom.stream)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, dist, "cuda")
    phases = {"init_tgv_ms": round(init_tgv_ms, 2),
              "init_from_host_ms": round(ev[0].elapsed_time(ev[1]), 2),
              "steps_with_diagnostics_ms": round(ev[1].elapsed_time(ev[2]), 2),
              "moments_to_host_ms": round(ev[2].elapsed_time(ev[3]), 2)}
    e2e = {"value": round(job_value(world, ncell, args.steps, e2e_s * 1e3), 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int(fields.numel() * 4 / args.steps),
           "d2h_bytes_per_step": int((out.numel() * 4 + len(series) * 15 * 8) / args.steps),
           "api": "lbm_init_fields(host) + lbm_step_diag every 50 steps (diagnostics "
                  "computed in the step, FP64 global sums) + lbm_moments(host)",
           "diagnostics": len(series), "phases_gpu_ms": phases,
           "ek_last": series[-1]["ek_mean"] if series else None}
    diag_cost = None
    if not args.no_variants and rank == 0:
        diag_cost = diag_costs(torch, dom, ms_step)
        # the same readback again, outside the end-to-end timing, and a plain copy of
        # the same bytes into the same pinned buffer (transfer rate of this host buffer)
        t1 = time.perf_counter()
        dom.moments_into(out, which=lbm.MOM_PRIM, on_device=False)
        e2e["moments_to_host_repeat_ms"] = round(1e3 * (time.perf_counter() - t1), 2)
        dev_prim = dom.moments_device(lbm.MOM_PRIM)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out.copy_(dev_prim, non_blocking=True)
        torch.cuda.synchronize()
        e2e["plain_d2h_copy_ms"] = round(1e3 * (time.perf_counter() - t1), 2)
        del dev_prim
    dom.close()
    del dom, fields, out
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants and rank == 0:
        ref_curves = long_run_curves("f32")
        for st, sr in (("f16", 0), ("bf16", 0), ("f16", 1), ("bf16", 1)):
            if st == args.store:
                continue
            d2 = lbm.Domain(dict(p, stochastic_round=sr), store=st)
            d2.init_tgv(1.0, 1.25, 1.0)
            tune2 = d2.autotune(pairs_per_trial=3)  # advances the state: re-init below
            d2.init_tgv(1.0, 1.25, 1.0)
            k2 = max(10, min(args.steps, 400))
            ms2, _ = time_steps(torch, d2, k2, max(args.warmup, 3))
            d2.close()
            del d2
            torch.cuda.empty_cache()
            ach = BYTES_PER_CELL[st] * ncell / (ms2 / k2 * 1e-3) / 1e9
            variants[st + ("_stochastic_rounding" if sr else "")] = {
                "value": round(ncell * k2 / (ms2 * 1e-3) / 1e6, 1), "unit": "MLUPS",
                "achieved_gbs": round(ach, 1), "frac": round(ach / hbm, 4),
                "steps": k2, "tune": tune2, "stated_err": stated_error(st, sround=sr),
                "stated_err_long_run": long_run_error(long_run_curves(st, sr), ref_curves)}
        variants[args.store] = {"stated_err": stated_error(args.store), "tune": tune}
        k3 = max(10, min(args.steps, 400))
        variants["streaming_" + args.store] = streaming_leg(
            torch, lbm, inputs.tgv_params(n), args.store, ncell, k3, args.warmup, hbm)
        if args.store != "f16":
            variants["streaming_f16"] = streaming_leg(
                torch, lbm, inputs.tgv_params(n), "f16", ncell, k3, args.warmup, hbm)
        variants["diagnostics"] = diag_cost
        kb = min(args.steps, 200)
        variants["batch64"] = batch_leg(torch, lbm, inputs, kb, args.warmup,
                                        streaming=args.streaming)
        variants["batch64_f16"] = batch_leg(torch, lbm, inputs, kb, args.warmup, store="f16",
                                            streaming=args.streaming)
        variants["batch64_f16_stochastic_rounding"] = batch_leg(
            torch, lbm, inputs, kb, args.warmup, store="f16", sround=1, streaming=args.streaming)

    cpu = args.cpu
    if cpu is not None and not args.no_variants:
        # the same oracle in this process after the GPU legs, for comparison only
        in_proc, secs_ip, thr_ip = time_oracle(n, CPU_WINDOW, 4, 1)
        cpu["in_gpu_process_after_gpu_legs"] = {
            "value": round(in_proc, 3), "unit": "MLUPS", "cores": thr_ip,
            "sample": f"{CPU_WINDOW}^3 window, 4 steps ({secs_ip:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": bench_config(n, args.store, world, args.streaming),
            "roofline": roofline,
            "repeats": {"MLUPS": repeats, "best": max(repeats),
                        "median": sorted(repeats)[1], "steps": [args.steps, rep_steps, rep_steps]},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--store", default="f32", choices=("f32", "f16", "bf16"))
    ap.add_argument("--streaming", type=int, default=1, choices=(0, 1),
                    help="in-place streaming map of the single-domain legs: 0 AA pattern, "
                         "1 esoteric twist (default; both are timed in the streaming legs)")
    ap.add_argument("--impl", default="gpu", choices=("gpu", "reference"))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-variants", action="store_true", help="skip the 16-bit storage legs")
    ap.add_argument("--only-batch", type=int, default=0, metavar="K",
                    help="run only the batched-mode leg on the first K seeded domains "
                         "(storage from --store)")
    ap.add_argument("--only-diag", action="store_true",
                    help="run only the diagnostics-cost leg (separate pass and in-step) on the "
                         "--n^3 TGV with storage --store")
    ap.add_argument("--only-batch-sizes", action="store_true",
                    help="run only uniform batches of 32^3 ... 128^3 domains (about 40 M cells "
                         "each, storage from --store)")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_baseline_only:  # the child process of cpu_baseline_subprocess
        print(json.dumps(cpu_baseline(args.n)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    from paper_2608_13437_gb300 import build
    build.build()
    world, rank, _ = dist_setup()
    args.cpu = None
    if (rank == 0 and world == 1 and not args.no_cpu and not args.only_batch and not args.only_diag
            and not args.only_batch_sizes):
        args.cpu = cpu_baseline_subprocess(args.n)
    if args.only_diag:
        import torch

        from paper_2608_13437_gb300 import inputs, lbm
        torch.cuda.set_device(0)
        dom = lbm.Domain(dict(inputs.tgv_params(args.n), streaming=args.streaming), store=args.store)
        dom.init_tgv(1.0, 1.25, 1.0)
        ms, _ = time_steps(torch, dom, 20, args.warmup)
        out = {"n": args.n, "store": args.store,
               "diagnostics": diag_costs(torch, dom, ms / 20)}
        dom.close()
        print(json.dumps(out), flush=True)
        return
    if args.only_batch_sizes:
        import torch

        from paper_2608_13437_gb300 import inputs, lbm
        torch.cuda.set_device(0)
        print(json.dumps(batch_size_sweep(torch, lbm, inputs, min(args.steps, 100), args.warmup,
                                          args.store)), flush=True)
        return
    if args.only_batch:
        import torch

        from paper_2608_13437_gb300 import inputs, lbm
        torch.cuda.set_device(0)
        print(json.dumps(batch_leg(torch, lbm, inputs, args.steps, args.warmup, args.only_batch,
                                   store=args.store, streaming=args.streaming)), flush=True)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
