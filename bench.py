#!/usr/bin/env python
"""Throughput of one-site TDVP-PS (site updates per second) on B300.

A step is one full TDVP-PS time step (Eq. ps_trotter: left-to-right half sweep, turning site,
right-to-left half sweep) of every trajectory held on the GPU.  One site update is one forward
site evolution with its gauge shift, environment update and backward bond evolution, so a step
of an N-site chain is 2N-1 site updates per trajectory.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference] [--precision fp64]

Default workload: the FMO-sized Frenkel-Holstein chain (7 electronic sites x 10 Debye modes with
10 levels = 77 sites), bond dimension 64, dt = 10 fs, product start (exciton on site 1),
adaptive Lanczos with tolerance 1e-12.  All inputs are synthetic and seeded.
With N > 1 (torchrun) every rank advances its own replica; there is no exchange.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDVP-PS site-updates/s & % tensor peak, mixed vs FP64 GPU at pop. err ≤1e-4"
UNIT = "site-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25      # B300 FP64 (no FP64 tensor path); measured DFMA ceiling ~0.95


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64"])
    ap.add_argument("--D", type=int, default=64)
    ap.add_argument("--dt", type=float, default=10.0)
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-prof", action="store_true", help="time without per-launch events")
    return ap.parse_args()


def workload(args):
    import workloads as wl
    p = wl.fmo_sized()
    return p, {"workload": f"{p.name}: {len(p.chain())} sites, D={args.D}, dt={args.dt} fs, product start",
               "model": "Frenkel-Holstein (synthetic FMO-sized, Debye bath)",
               "sites": len(p.chain()), "bond_dim": args.D, "dt_fs": args.dt,
               "krylov": f"adaptive Lanczos, tol {args.tol:g}", "precision": args.precision,
               "realisations_per_gpu": 1}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1)          # 256 MiB read+write through L2 (126 MB), on the current stream


def run_ours(args, rank, world):
    import torch
    import paper_1907_12044_b300 as pkg
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    p, cfg = workload(args)
    N = len(p.chain())
    stream = torch.cuda.current_stream()
    eng = pkg.Engine(n_realisations=1, stream=stream.cuda_stream)
    eng.build_mpo(0, p)
    eng.init_mps(0, args.D, p.exciton_site)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        eng.step(args.dt, 1, tol=args.tol)
    torch.cuda.synchronize()
    eng.reset_stats()
    if not args.no_prof:
        eng.set_profiling(True)
    times = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eng.step(args.dt, 1, tol=args.tol)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st = eng.stats()
    eng.set_profiling(False)
    ms_local = float(np.sum(times))
    ms = ms_local
    if world > 1:
        t = torch.tensor([ms_local], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    updates_per_step = (2 * N - 1) * 1
    value = updates_per_step * args.steps * world / (ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)",
           "data": "synthetic (seeded FMO-sized Frenkel-Holstein chain)",
           "config": dict(cfg, parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                          l2="flushed between timed steps (256 MiB write)"),
           "gpu_launches": int(st["kernel_launches"]), "clocks": clk.summary()}
    # roofline of the dominant kernel (the FP64 contraction GEMM)
    if not args.no_prof:
        gms = st["prof_ms"]["gemm"]
        gfl = st["prof_flops"]["gemm"]
        nl = st["prof_launches"]["gemm"]
        ach = gfl / (gms * 1e-3) / 1e12 if gms > 0 else None
        total_prof = sum(st["prof_ms"].values())
        out["roofline"] = {"kernel": "zgemm_kernel (FP64 complex contraction GEMMs)", "bound": "alu",
                           "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                           "frac": ach / FP64_NOMINAL_TFLOPS if ach else None, "traffic": None,
                           "peak_source": "B300 FP64 nominal 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json)",
                           "launches": nl, "avg_launch_us": 1e3 * gms / max(nl, 1),
                           "share_of_step": gms / max(total_prof, 1e-9)}
        out["kernel_time_ms"] = {k: round(v, 3) for k, v in st["prof_ms"].items()}
    out["krylov"] = {"mean_dim": st["krylov_dim_sum"] / max(st["krylov_solves"], 1),
                     "max_dim": st["krylov_dim_max"], "host_syncs": st["host_syncs"]}
    eng.close()
    return out, p


def run_e2e(args, p):
    """Whole job through the public API from host buffers: parameters and the initial state go
    host->device, every step's populations come back device->host."""
    import torch
    import paper_1907_12044_b300 as pkg
    N = len(p.chain())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng = pkg.Engine(n_realisations=1)
    eng.build_mpo(0, p)
    eng.init_mps(0, args.D, p.exciton_site)
    d, bd, w = eng.chain_info(0)
    for _ in range(args.steps):
        eng.step(args.dt, 1, tol=args.tol)
        pops, E, nrm = eng.observables(0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    f = p.flat()
    h2d = sum(np.asarray(v).nbytes for v in f.values()) + 8 * 2 + sum(
        16 * int(bd[i]) * int(d[i]) * int(bd[i + 1]) for i in range(N))
    eng.close()
    return {"value": (2 * N - 1) * args.steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 8 * (p.n_el + 2),
            "includes": "MPO build + initial state upload + steps + per-step observables readback"}


def oracle_rate(p, args, n_steps=1):
    """The CPU oracle as it stands on the same workload; returns (site-updates/s, threads, seconds)."""
    from oracle import TDVPState, tdvp_ps_step
    try:
        from threadpoolctl import threadpool_info
        threads = max([x.get("num_threads", 1) for x in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count()
    st = TDVPState.start(p, D=args.D)
    N = len(p.chain())
    t0 = time.perf_counter()
    for _ in range(n_steps):
        tdvp_ps_step(st, args.dt, tol=args.tol)
    dt = time.perf_counter() - t0
    return (2 * N - 1) * n_steps / dt, threads, dt


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        p, cfg = workload(args)
        vals = []
        for _ in range(args.steps):
            v, thr, secs = oracle_rate(p, args, 1)
            vals.append(secs)
        N = len(p.chain())
        value = (2 * N - 1) * args.steps / sum(vals)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * sum(vals) / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)", "data": "synthetic",
               "config": dict(cfg, parallelism="CPU oracle (numpy/scipy, OpenBLAS threads)"), "impl": "reference",
               "cpu_baseline": {"kind": "oracle", "cores": thr, "value": value, "unit": UNIT,
                                "sample": f"{args.steps} full TDVP-PS step(s) of the bench workload from the product start"},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out, p = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_e2e:
            out["e2e"] = run_e2e(args, p)
        if not args.no_cpu_baseline and world == 1:
            v, thr, secs = oracle_rate(p, args, 1)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                                   "sample": f"one full TDVP-PS step of the bench workload from the product start ({secs:.1f} s)"}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
