#!/usr/bin/env python
"""Throughput of one-site TDVP-PS (site updates per second) on B300.

A step is one full TDVP-PS time step (Eq. ps_trotter: left-to-right half sweep, turning site,
right-to-left half sweep) of every trajectory held on the GPU.  One site update is one forward
site evolution with its gauge shift, environment update and backward bond evolution, so a step
of an N-site chain is 2N-1 site updates per trajectory.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference] [--precision P]

Workload: the FMO-sized Frenkel-Holstein chain (7 electronic sites x 10 Debye modes with 10
levels = 77 sites), bond dimension 64, dt = 10 fs, product start (exciton on site 1).  All
inputs are synthetic and seeded.  Three GPU arms run the same W warm-up and K timed steps:
  - the timed arm (`value`): mixed-precision matvecs, Lanczos tolerance 1e-8, each step replayed
    as a CUDA graph, learned Krylov controller trained on the warm-up;
  - `fp64_arm`: the same in every respect except FP64 matvecs (isolates the precision);
  - `plain_fp64_arm`: the plain method (FP64, tolerance 1e-12, convergence tested at every k,
    launch by launch), the reference of the population error.
With N > 1 (torchrun) every rank advances its own replica (a single trajectory is sequential
along the chain) and the disorder realisations of the batched section are sharded by index.
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
TF32_OF_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor rate ratio

# arithmetic of the Lanczos matvecs (TDVP_PREC_* of include/tdvp.h); the tensor-core input
# format decides the peak a contraction is measured against
PREC = {"fp64": 0, "tf32": 1, "tf32x3": 2, "bf16": 3, "bf16x3": 4, "tf32_3m": 5, "bf16_3m": 6}
TENSOR_FMT = {"tf32": "tf32", "tf32x3": "tf32", "tf32_3m": "tf32", "bf16": "bf16", "bf16x3": "bf16",
              "bf16_3m": "bf16"}
DTYPE = {"fp64": "f64 (complex128)",
         "tf32": "tf32 tensor cores, 4M complex products, f32 accumulate; f64 Lanczos/QR",
         "tf32x3": "tf32x3 split tensor cores, 4M, f32 accumulate; f64 Lanczos/QR",
         "tf32_3m": "tf32 tensor cores, 3M (Gauss) complex products, f32 accumulate; f64 Lanczos/QR",
         "bf16": "bf16 tensor cores, 4M, f32 accumulate; f64 Lanczos/QR",
         "bf16x3": "bf16x3 split tensor cores, 4M, f32 accumulate; f64 Lanczos/QR",
         "bf16_3m": "bf16 tensor cores, 3M (Gauss), f32 accumulate; f64 Lanczos/QR"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=sorted(PREC),
                    help="arithmetic of the Lanczos matvecs on the timed arm")
    ap.add_argument("--workload", default="fmo", choices=["fmo", "large"],
                    help="fmo: 7 x 10 Debye modes with 10 levels (77 sites); large: 20 modes with 16 levels "
                         "(147 sites)")
    ap.add_argument("--D", type=int, default=64)
    ap.add_argument("--dt", type=float, default=10.0)
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="Lanczos tolerance of the timed arm and of the FP64 arm beside it: the TF32x3 "
                         "matvecs are accurate to ~1e-7 relative, so a tighter tolerance only adds "
                         "iterations below that noise")
    ap.add_argument("--plain-tol", type=float, default=1e-12, help="Lanczos tolerance of the plain FP64 arm")
    ap.add_argument("--rank-rtol", type=float, default=1e-6,
                    help="rank threshold of the gauge-shift QR, the same on every arm")
    ap.add_argument("--arms", default="mixed,adaptive,fp64,plain",
                    help="GPU arms to run (mixed = the timed arm, adaptive = the same without the learned "
                         "controller (the library's default test rule), fp64 = the timed arm with FP64 "
                         "matvecs, plain = FP64 at --plain-tol, every k tested, launch by launch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-prof", action="store_true", help="skip the per-kernel breakdown step")
    ap.add_argument("--no-learned", action="store_true", help="no learned Krylov controller")
    ap.add_argument("--no-graph", action="store_true", help="launch by launch instead of CUDA-graph steps")
    ap.add_argument("--no-pdl", action="store_true",
                    help="launch the step's kernels in plain stream order (no programmatic dependent launch)")
    ap.add_argument("--kernel-case", choices=["heff", "qr", "ozaki"], default=None,
                    help="time one hot operation at the bench's full-size shapes instead of steps (for "
                         "kernel captures): heff = one H_eff matvec at a bath-mode site of a random D-bond "
                         "state, qr = one gauge-shift QR of a rank-8 640 x 64 matrix")
    ap.add_argument("--batched", type=int, default=32,
                    help="also time R disorder realisations with ragged bond dims in the same launches "
                         "(0: skip); with N ranks each takes the realisations r = rank mod N")
    ap.add_argument("--batched-steps", type=int, default=None, help="timed steps of the batched section")
    ap.add_argument("--batched-dmax", type=int, default=128, help="largest ragged bond dimension")
    ap.add_argument("--long", type=int, default=0,
                    help="accuracy run instead of the bench line: this many steps of the timed arm and "
                         "of the plain FP64 arm from the same start, Eq. error and max |dP| every 100 steps")
    ap.add_argument("--lz-chunks", type=int, default=None, help="chunk cap per Lanczos vector (library option)")
    ap.add_argument("--fused", type=int, default=1, help="0: four Lanczos launches per iteration instead of one")
    ap.add_argument("--env-fp64", type=int, default=0,
                    help="1: environment updates in FP64 in the mixed precisions (matvecs on the tensor cores)")
    ap.add_argument("--batched-kmax", type=int, default=48, help="Krylov cap of the batched section")
    ap.add_argument("--batched-check", action="store_true",
                    help="re-run the first and last realisation alone and compare populations")
    ap.add_argument("--batched-compare", action="store_true",
                    help="also time the batched steps without the learned controller")
    ap.add_argument("--batched-prof", action="store_true",
                    help="per-kernel breakdown of one more batched step (launch by launch, CUDA events)")
    ap.add_argument("--long-precisions", default=None,
                    help="comma-separated precisions for the long run (default: --precision), each against "
                         "the same FP64 reference; an entry prec@tol sets that arm's Lanczos tolerance")
    ap.add_argument("--long-ref", default=None,
                    help="populations of an earlier FP64 reference run of the same workload (.npy, one row "
                         "per step) instead of running it again")
    ap.add_argument("--long-dir", default=None,
                    help="where the long run writes its population checkpoints (none if unset)")
    ap.add_argument("--out", default=None, help="also write the JSON line to this file")
    return ap.parse_args(argv)


def workload(args):
    import workloads as wl
    p = wl.fmo_sized() if args.workload == "fmo" else wl.fmo_large()
    return p, {"workload": f"{p.name}: {len(p.chain())} sites, D={args.D}, dt={args.dt} fs, product start",
               "sites": len(p.chain()), "bond_dim": args.D, "dt_fs": args.dt, "rank_rtol": args.rank_rtol}


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


def sig(x, n=4):
    """x rounded to n significant digits (keeps the JSON line short)."""
    if x is None or not np.isfinite(x) or x == 0:
        return x
    return float(f"{x:.{n}g}")


def train_controller(eng, seed=0, samples=None):
    """Train the learned Krylov controller on the solve log of the warm-up steps (GPU): 150 passes
    over a small log, fewer over a large one (at least 8, about 3e6 sample visits)."""
    from paper_1907_12044_b300.controller import init_weights
    eng.controller_set_weights(init_weights(seed))
    epochs = 150 if not samples else int(min(150, max(8, 3e6 / samples)))
    return eng.controller_train(epochs=epochs, batch=256, lr=3e-3)


ARMS = {
    # name: (precision, tolerance attribute, graph, learned, test every k)
    "mixed": (None, "tol", True, True, False),
    "adaptive": (None, "tol", True, False, False),
    "fp64": ("fp64", "tol", True, True, False),
    "plain": ("fp64", "plain_tol", False, False, True),
    "fp64ref": ("fp64", "plain_tol", True, False, False),
}


def arm_setup(args, name):
    prec, tol_attr, graph, learned, every = ARMS[name]
    prec = prec or args.precision
    graph = graph and not args.no_graph and args.warmup >= 1
    learned = learned and not args.no_learned
    return prec, getattr(args, tol_attr), graph, learned, every


def timed_run(args, p, name, world, dev, stream, flush):
    """W warm-up steps, then K timed steps (L2 flushed before each); returns timing and populations.

    With the learned controller the warm-up steps log their solves and the controller is trained
    on them.  A graph arm captures its step in the last warm-up step.  After the timed steps one
    more step runs launch by launch with per-launch CUDA events for the per-kernel breakdown."""
    import torch
    import paper_1907_12044_b300 as pkg
    prec, tol, graph, learned, every = arm_setup(args, name)
    P = PREC[prec]
    eng = pkg.Engine(n_realisations=1, stream=stream.cuda_stream)
    eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
    if args.lz_chunks:
        eng.set_option(pkg.OPT_LANCZOS_CHUNKS, args.lz_chunks)
    eng.set_option(pkg.OPT_FUSED_LANCZOS, args.fused)
    eng.set_option(pkg.OPT_ENV_FP64, args.env_fp64)
    eng.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1 if every else 0)
    eng.build_mpo(0, p)
    eng.init_mps(0, args.D, p.exciton_site)
    eng.autotune()          # QR launch shape per gauge-shift shape
    pops = [eng.observables(0)[0]]
    if learned:
        eng.controller_logging(1 << 20)
    # the launch-by-launch warm-up steps (at least one when the controller learns from them), then
    # the graph capture step
    for _ in range(max(1 if learned else 0, args.warmup - (1 if graph else 0))):
        eng.step(args.dt, 1, precision=P, tol=tol)
        pops.append(eng.observables(0)[0])
    ctl = None
    if learned:
        nlog = eng.stats()["krylov_solves"]
        eng.controller_logging(0)
        ctl = {"train_loss": [sig(x, 3) for x in train_controller(eng, samples=nlog)], "samples": int(nlog)}
    mode = pkg.KRYLOV_LEARNED if learned else pkg.KRYLOV_ADAPTIVE
    if graph:
        eng.set_option(pkg.OPT_GRAPH, 1)
        eng.step(args.dt, 1, precision=P, krylov_mode=mode, tol=tol)   # capture
        pops.append(eng.observables(0)[0])
    torch.cuda.synchronize()
    eng.reset_stats()
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
            eng.step(args.dt, 1, precision=P, krylov_mode=mode, tol=tol)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            pops.append(eng.observables(0)[0])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st = eng.stats()
    prof = None
    if not args.no_prof:
        # per-kernel CUDA-event breakdown of one more (untimed) step, launch by launch
        eng.set_option(pkg.OPT_GRAPH, 0)
        eng.reset_stats()
        eng.set_profiling(True)
        eng.step(args.dt, 1, precision=P, krylov_mode=mode, tol=tol)
        eng.set_profiling(False)
        prof = eng.stats()
    eng.close()
    ms = max_over_ranks(float(np.sum(times)), world)
    return {"ms": ms, "stats": st, "prof": prof, "pops": np.array(pops), "clocks": clk.summary(),
            "controller": ctl, "graph": graph, "prec": prec, "tol": tol, "learned": learned, "every": every}


def max_over_ranks(ms, world):
    """The slowest rank's time (every rank gets it): all-reduce MAX over the default process group,
    on the device for NCCL and on the host for gloo."""
    if world <= 1:
        return ms
    import torch
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def site_update_rate(n_sites, steps, world, ms):
    """Whole-job site updates per second: every rank advances its own trajectory (2N-1 site
    updates per step each, Eq. ps_trotter) and the job takes the slowest rank's time."""
    return (2 * n_sites - 1) * steps * world / (ms / 1e3)


def pop_error(dt, pops, ref):
    """Eq. error at the last compared time (trapezoid in time) and max |dP|, against `ref`."""
    n = min(len(pops), len(ref))
    t = dt * np.arange(n)
    dP = np.abs(np.asarray(pops[:n]) - np.asarray(ref[:n]))
    if n < 2:
        return 0.0, float(dP.max()) if dP.size else 0.0
    s = dP.sum(1)
    err = float(np.sum(0.5 * (s[1:] + s[:-1]) * np.diff(t)) / (dP.shape[1] * t[-1]))
    return err, float(dP.max())


# kernel and roof of each timed category
# The Lanczos orthogonalisation does 32 (j+1) n FP64 flops on 64 (j+1) n bytes per iteration, 0.5
# flop/B, above B300's FP64 ridge point (1.25 TFLOP/s / 6.5 TB/s = 0.19 flop/B): it is bound by the
# FP64 pipe, not by HBM, and is measured against the FP64 peak (its HBM fraction is given beside).
ROOF_KERNELS = {"qr": ("bqr_kernel/cqr_kernel (FP64 gauge-shift QR)", "alu"),
                "gemm": ("zgemm_kernel (FP64 complex GEMM)", "alu"),
                "tc_gemm": ("tc_cgemm_kernel (tcgen05)", "tensor"),
                "lanczos_vec": ("lz_iter / lz_* (FP64 Lanczos orthogonalisation)", "alu")}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# kernel as it is built now, on the bench's workload (three launches each, cold caches, launch by
# launch): (bytes, what was captured).  A kernel missing here has no capture of its current form,
# and its `traffic` is null.
TRAFFIC = {"lanczos_vec": (2.099e6, "lz_iter, mean of 3 launches at a 64x10x64 site"),
           "tc_gemm": (0.703e6, "tc_cgemm_kernel<TF32x3>, mean of 3 launches (H0 stages, one finished solve)")}


def peaks():
    return json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}


def tensor_peak(fmt):
    pk = peaks()
    bf16 = pk.get("bf16_tflops")
    src = "measured bf16 burst" if bf16 else "fallback 1800 TFLOP/s bf16"
    bf16 = bf16 or 1800.0
    if fmt == "tf32":
        return bf16 * TF32_OF_BF16, src + " x nominal tf32/bf16 1.1/2.25"
    return bf16, src


def roofline(prof, cat, prec):
    """Achieved vs peak for one category of the profiled step: algorithmic work / summed
    CUDA-event time of its launches.  Lanczos vectors: FP64 flops of the two Gram-Schmidt passes
    (16 n k (k+1) per solve) against the FP64 peak, and beside it HBM with Sec. 8(d)'s count of
    k^2/2 vectors of 16 n bytes per solve (`hbm_frac`; `hbm_frac_4pass` counts the four reads per
    iteration of the kernels as written)."""
    ms, nl = prof["prof_ms"][cat], prof["prof_launches"][cat]
    name, bound = ROOF_KERNELS[cat]
    base = {"kernel": name, "bound": bound, "launches": nl, "avg_launch_us": sig(1e3 * ms / max(nl, 1)),
            "traffic": TRAFFIC.get(cat, (None, None))[0]}
    if cat == "lanczos_vec":
        by = prof.get("prof_bytes", {}).get(cat, 0.0)          # library count, 4 passes
        by_alg = prof.get("lz_alg_bytes", 0.0)
        pk = peaks()
        hbm = pk.get("hbm_gbs", 6400.0)
        gbs = by_alg / (ms * 1e-3) / 1e9 if ms > 0 else None
        base.update(hbm_gbs=sig(gbs), hbm_frac=sig(gbs / hbm) if gbs else None,
                    hbm_frac_4pass=sig(by / (ms * 1e-3) / 1e9 / hbm) if ms else None,
                    bytes_per_launch=sig(by_alg / max(nl, 1)))
    fl = prof["prof_flops"][cat]
    ach = fl / (ms * 1e-3) / 1e12 if ms > 0 else None
    if bound == "tensor":
        peak, src = tensor_peak(TENSOR_FMT.get(prec, "tf32"))
    else:
        peak, src = FP64_NOMINAL_TFLOPS, "FP64 nominal (no FP64 entry measured)"
    return dict(base, achieved=sig(ach), peak=sig(peak), unit="TFLOP/s", frac=sig(ach / peak) if ach else None,
                flops_per_launch=sig(fl / max(nl, 1)), peak_source=src)


def lz_alg_bytes(st):
    """Sec. 8(d)'s algorithmic bytes of the Lanczos vectors of the profiled step: k(k+1)/2 reads of
    a 16 n-byte vector per solve, from the library's 4-pass count 16 n (2k(k+1) + 10k + 5) summed
    over solves, taking k at the mean Krylov dimension."""
    k = st["krylov_dim_sum"] / max(st["krylov_solves"], 1)
    by4 = st["prof_bytes"]["lanczos_vec"]
    return by4 * (0.5 * k * (k + 1)) / (2 * k * (k + 1) + 10 * k + 5) if k > 0 else 0.0


def arm_summary(args, run, N, world):
    st = run["stats"]
    out = {"value": sig(site_update_rate(N, args.steps, world, run["ms"])), "unit": UNIT,
           "ms_per_step": sig(run["ms"] / args.steps), "precision": run["prec"], "tol": run["tol"],
           "graph": run["graph"], "learned": run["learned"], "every_k": run["every"],
           "krylov_mean": sig(st["krylov_dim_sum"] / max(st["krylov_solves"], 1), 3),
           "tri_evals_per_step": sig(st["tri_evals"] / args.steps, 4),
           "launches_per_step": int(st["kernel_launches"] / max(args.steps, 1))}
    if run["prof"]:
        out["phase_ms"] = {k: sig(v, 3) for k, v in run["prof"]["prof_phase_ms"].items() if v > 0}
    return out


def run_ours(args, rank, world):
    import torch
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    p, cfg = workload(args)
    N = len(p.chain())
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    names = [a for a in args.arms.split(",") if a]
    runs = {a: timed_run(args, p, a, world, dev, stream, flush) for a in names}
    main = runs.get("mixed") or runs[names[0]]
    st = main["stats"]
    out = {"metric": METRIC, "value": sig(site_update_rate(N, args.steps, world, main["ms"]), 5), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sig(main["ms"] / args.steps, 5), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE[main["prec"]], "data": "synthetic (seeded FMO-sized FH chain)",
           "config": dict(cfg, precision=main["prec"], tol=main["tol"],
                          krylov="learned controller" if main["learned"] else "adaptive",
                          execution="CUDA-graph steps" if main["graph"] else "launch by launch",
                          parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                          l2="flushed between timed steps (256 MiB write)"),
           "gpu_launches": int(st["kernel_launches"]), "clocks": main["clocks"]}
    if "fp64" in runs and main is not runs["fp64"]:
        out["speedup_vs_fp64"] = sig(runs["fp64"]["ms"] / main["ms"])
    if "plain" in runs and main is not runs["plain"]:
        out["speedup_vs_plain_fp64"] = sig(runs["plain"]["ms"] / main["ms"])
        e, m = pop_error(args.dt, main["pops"], runs["plain"]["pops"])
        out["pop_error_vs_fp64"] = {"eq_error": sig(e, 3), "max_abs_dP": sig(m, 3),
                                    "steps": len(main["pops"]) - 1, "against": "plain_fp64_arm"}
    if "fp64" in runs and main is not runs["fp64"]:
        e, m = pop_error(args.dt, main["pops"], runs["fp64"]["pops"])
        out["pop_error_vs_fp64_arm"] = {"eq_error": sig(e, 3), "max_abs_dP": sig(m, 3)}
    if "adaptive" in runs and main is not runs["adaptive"]:
        ad, ms = runs["adaptive"], main
        out["controller_gain"] = {"wall": sig(ad["ms"] / ms["ms"]),
                                  "tri_evals": sig(ad["stats"]["tri_evals"] / max(ms["stats"]["tri_evals"], 1)),
                                  "against": "default rule (tests from the previous k - 2)"}
    out["arms"] = {("timed" if r is main else a): arm_summary(args, r, N, world) for a, r in runs.items()}
    if main["controller"]:
        out["learned_controller"] = main["controller"]
    if main["prof"]:
        pr = main["prof"]
        pr["lz_alg_bytes"] = lz_alg_bytes(pr)
        cat_ms = pr["prof_ms"]
        ranked = sorted((c for c in ROOF_KERNELS if cat_ms.get(c, 0) > 0), key=lambda c: -cat_ms[c])
        if ranked:
            out["roofline"] = roofline(pr, ranked[0], main["prec"])
            out["roofline"]["category"] = ranked[0]
            out["roofline_other"] = {c: {k: v for k, v in roofline(pr, c, main["prec"]).items()
                                         if k in ("achieved", "peak", "unit", "frac", "avg_launch_us", "bound",
                                                  "hbm_gbs", "hbm_frac")}
                                     for c in ranked[1:]}
        tot = sum(cat_ms.values())
        out["kernel_share"] = {c: sig(v / tot, 3) for c, v in cat_ms.items() if v > 0}
    return out, p


def shard(R, rank, world):
    """Realisation indices of one rank: r = rank, rank + world, ... (no exchange during the run)."""
    return list(range(rank, R, world))


def run_batched(args, R, rank=0, world=1):
    """R static-disorder realisations of the FMO-sized chain with bond dims drawn from
    {32,48,64,96,128}, sharded by index over the ranks; each rank advances its share in the same
    launches.  Returns this rank's share, its timing and its final populations."""
    import torch
    import workloads as wl
    import paper_1907_12044_b300 as pkg
    base = wl.fmo_sized()
    choices = tuple(c for c in (32, 48, 64, 96, 128) if c <= args.batched_dmax)
    Ds = wl.ragged_bond_dims(R, choices=choices)
    # this rank's realisations, placed in the engine in order of bond dimension: the gauge-shift
    # QR is launched per run of equal shapes, so equal D side by side share launches
    mine = sorted(shard(R, rank, world), key=lambda r: (Ds[r], r))
    steps = args.batched_steps or args.steps
    tol = args.tol
    P = PREC[args.precision]
    eng = pkg.Engine(n_realisations=len(mine), kmax=args.batched_kmax)
    eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
    eng.set_option(pkg.OPT_ENV_FP64, args.env_fp64)
    eng.set_option(pkg.OPT_FUSED_LANCZOS, args.fused)
    if args.lz_chunks:
        eng.set_option(pkg.OPT_LANCZOS_CHUNKS, args.lz_chunks)
    for q, r in enumerate(mine):
        p = wl.disorder_realisation(base, r)
        eng.build_mpo(q, p)
        eng.init_mps(q, Ds[r], p.exciton_site)
    eng.autotune()
    graph = not args.no_graph and args.warmup >= 1
    learned = not args.no_learned
    ctl_loss, nlog = None, 0
    if learned:
        eng.controller_logging(1 << 22)
    nsteps = 0
    for _ in range(max(1 if learned else 0, args.warmup - (1 if graph else 0))):
        eng.step(args.dt, 1, precision=P, tol=tol)
        nsteps += 1
    mode = pkg.KRYLOV_ADAPTIVE
    if learned:
        eng.controller_logging(0)
        nlog = eng.stats()["krylov_solves"]
        ctl_loss = train_controller(eng, samples=nlog)
        mode = pkg.KRYLOV_LEARNED
    if graph:
        eng.set_option(pkg.OPT_GRAPH, 1)
        eng.step(args.dt, 1, precision=P, krylov_mode=mode, tol=tol)   # capture
        nsteps += 1
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    eng.reset_stats()
    e0.record(stream)
    eng.step(args.dt, steps, precision=P, krylov_mode=mode, tol=tol)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    nsteps += steps
    st = eng.stats()
    pops = {r: eng.observables(q)[0].tolist() for q, r in enumerate(mine)}
    check = None
    if args.batched_check:
        # the first and the last realisation of this rank advanced alone from the same start for
        # the same steps, same precision and tolerance (plain adaptive Lanczos): the batched run
        # agrees with them within the mixed-precision bound
        worst = 0.0
        for q in sorted({0, len(mine) - 1}):
            r = mine[q]
            pr = wl.disorder_realisation(base, r)
            one = pkg.Engine(n_realisations=1, kmax=args.batched_kmax)
            one.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
            one.build_mpo(0, pr)
            one.init_mps(0, Ds[r], pr.exciton_site)
            one.step(args.dt, nsteps, precision=P, tol=tol)
            P1 = one.observables(0)[0]
            one.close()
            worst = max(worst, float(np.max(np.abs(P1 - np.asarray(pops[r]))) / max(np.max(np.abs(P1)), 1e-300)))
        check = {"realisations": [mine[0], mine[-1]], "bond_dims": [Ds[mine[0]], Ds[mine[-1]]], "steps": nsteps,
                 "max_rel_dP": sig(worst, 3)}
    cmp = None
    if args.batched_compare and learned:
        # the following steps without the controller (the library's default test rule), timed
        # the same way: the controller's wall-time gain on the batched sweep
        eng.step(args.dt, 1, precision=P, krylov_mode=pkg.KRYLOV_ADAPTIVE, tol=tol)   # capture
        torch.cuda.synchronize()
        eng.reset_stats()
        e0.record(stream)
        eng.step(args.dt, steps, precision=P, krylov_mode=pkg.KRYLOV_ADAPTIVE, tol=tol)
        e1.record(stream)
        e1.synchronize()
        ms_ad = e0.elapsed_time(e1)
        sa = eng.stats()
        cmp = {"adaptive_ms_per_step": sig(ms_ad / steps), "learned_ms_per_step": sig(ms / steps),
               "wall_gain": sig(ms_ad / ms), "tri_evals_per_solve_adaptive":
               sig(sa["tri_evals"] / max(sa["krylov_solves"], 1), 3),
               "krylov_mean_adaptive": sig(sa["krylov_dim_sum"] / max(sa["krylov_solves"], 1), 3)}
    prof = None
    if args.batched_prof:
        # per-kernel CUDA-event breakdown of one more (untimed) step, launch by launch
        eng.set_option(pkg.OPT_GRAPH, 0)
        eng.reset_stats()
        eng.set_profiling(True)
        eng.step(args.dt, 1, precision=P, krylov_mode=mode, tol=tol)
        eng.set_profiling(False)
        pr = eng.stats()
        pr["lz_alg_bytes"] = lz_alg_bytes(pr)
        cat_ms = pr["prof_ms"]
        ranked = sorted((c for c in ROOF_KERNELS if cat_ms.get(c, 0) > 0), key=lambda c: -cat_ms[c])
        prof = {"phase_ms": {k: sig(v, 3) for k, v in pr["prof_phase_ms"].items() if v > 0},
                "kernel_ms": {k: sig(v, 3) for k, v in cat_ms.items() if v > 0},
                "roofline": {c: {k: v for k, v in roofline(pr, c, args.precision).items()
                                 if k in ("achieved", "peak", "unit", "frac", "avg_launch_us", "bound", "launches",
                                          "hbm_frac")}
                             for c in ranked}}
    eng.close()
    ms_max = max_over_ranks(ms, world)
    N = len(base.chain())
    return {"realisations": R, "per_rank": len(mine), "bond_dims": f"ragged {list(choices)}",
            "precision": args.precision, "steps": steps,
            "value": sig((2 * N - 1) * R * steps / (ms_max / 1e3)), "unit": UNIT,
            "ms_per_step": sig(ms_max / steps), "gpu_launches": int(st["kernel_launches"]),
            "krylov": "learned controller" if learned else "adaptive",
            "controller": {"samples": int(nlog), "train_loss": [sig(x, 3) for x in ctl_loss]} if ctl_loss else None,
            "krylov_mean": sig(st["krylov_dim_sum"] / max(st["krylov_solves"], 1), 3),
            "tri_evals_per_solve": sig(st["tri_evals"] / max(st["krylov_solves"], 1), 3),
            "execution": "CUDA-graph steps" if graph else "launch by launch",
            "sharding": f"realisation r on rank r mod {world}" if world > 1 else "one GPU",
            "profile": prof, "controller_vs_default": cmp, "check_vs_single": check}, pops


def gather_pops(pops, rank, world):
    """Final populations of every realisation on rank 0, over a host (gloo) group: the only
    exchange of the sharded batched run, after the timed region."""
    if world <= 1:
        return pops
    import torch.distributed as dist
    grp = dist.new_group(backend="gloo")
    allp = [None] * world if rank == 0 else None
    dist.gather_object(pops, allp, dst=0, group=grp)
    if rank != 0:
        return None
    out = {}
    for d in allp:
        out.update(d)
    return out


def run_e2e(args, p):
    """The timed arm end to end through the public API on the host clock: build_mpo from host
    parameters, init_mps, autotune, the warm-up steps with their solve log, controller training,
    then the timed steps, each followed by a device->host read of populations, energy and norm.
    The value counts the site updates of every step (warm-up included) over that whole time."""
    import torch
    import paper_1907_12044_b300 as pkg
    N = len(p.chain())
    prec, tol, graph, learned, every = arm_setup(args, "mixed")
    P = PREC[prec]
    d = np.asarray(p.phys_dims())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng = pkg.Engine(n_realisations=1)
    eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
    eng.set_option(pkg.OPT_ENV_FP64, args.env_fp64)
    eng.build_mpo(0, p)
    eng.init_mps(0, args.D, p.exciton_site)
    eng.autotune()
    if learned:
        eng.controller_logging(1 << 20)
    nsteps = 0
    for _ in range(max(1 if learned else 0, args.warmup - (1 if graph else 0))):
        eng.step(args.dt, 1, precision=P, tol=tol)
        eng.observables(0)
        nsteps += 1
    mode = pkg.KRYLOV_ADAPTIVE
    if learned:
        eng.controller_logging(0)
        train_controller(eng)
        mode = pkg.KRYLOV_LEARNED
    if graph:
        eng.set_option(pkg.OPT_GRAPH, 1)
    for _ in range(args.steps + (1 if graph else 0)):
        eng.step(args.dt, 1, precision=P, krylov_mode=mode, tol=tol)
        pops, E, nrm = eng.observables(0)
        nsteps += 1
    dt = time.perf_counter() - t0
    f = p.flat()
    h2d = sum(np.asarray(v).nbytes for v in f.values())
    eng.close()
    return {"value": sig(site_update_rate(N, nsteps, 1, 1e3 * dt)), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / nsteps), "d2h_bytes_per_step": 8 * (p.n_el + 2),
            "steps": nsteps, "seconds": sig(dt),
            "includes": "create, build_mpo, init, autotune, warm-up, training, steps + observables"}


def oracle_threads():
    """BLAS threads the oracle runs with (threadpoolctl when present, else the environment's
    OPENBLAS_NUM_THREADS / OMP_NUM_THREADS, else the host's CPU count, OpenBLAS's default)."""
    try:
        from threadpoolctl import threadpool_info
        return max([x.get("num_threads", 1) for x in threadpool_info()] or [1])
    except Exception:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
            if os.environ.get(k, "").isdigit():
                return int(os.environ[k])
        return os.cpu_count()


def oracle_run(p, args, warmup, steps, budget_s=None):
    """The CPU oracle as it stands on the same workload and the same steps as the GPU arms: the
    product start, `warmup` untimed steps, then up to `steps` timed ones (fewer if `budget_s`
    runs out).  Same Lanczos tolerance and rank threshold as the timed arm.  Returns
    (site-updates/s, threads, timed steps, seconds)."""
    from oracle import TDVPState, tdvp_ps_step
    st = TDVPState.start(p, D=args.D)
    for _ in range(warmup):
        tdvp_ps_step(st, args.dt, tol=args.tol, rank_rtol=args.rank_rtol)
    N = len(p.chain())

    def timed():
        t0 = time.perf_counter()
        n = 0
        while n < steps:
            tdvp_ps_step(st, args.dt, tol=args.tol, rank_rtol=args.rank_rtol)
            n += 1
            if budget_s is not None and time.perf_counter() - t0 > budget_s:
                break
        return n, time.perf_counter() - t0

    n, dt = timed()
    return (2 * N - 1) * n / dt, oracle_threads(), n, dt


_ONE_THREAD_STEP = """
import pickle, sys, time
sys.path.insert(0, sys.argv[1])
from oracle import tdvp_ps_step
st, dt, tol, rtol = pickle.load(open(sys.argv[2], "rb"))
t0 = time.perf_counter()
tdvp_ps_step(st, dt, tol=tol, rank_rtol=rtol)
print(time.perf_counter() - t0)
"""


def cpu_baseline(p, args):
    """The oracle on the host cores: step W+1 of the trajectory with every BLAS thread, then step
    W+2 in a child process limited to one BLAS thread (OPENBLAS/OMP/MKL_NUM_THREADS=1), handed the
    state after step W+1."""
    import pickle
    import tempfile
    from oracle import TDVPState, tdvp_ps_step
    N = len(p.chain())
    st = TDVPState.start(p, D=args.D)
    for _ in range(args.warmup):
        tdvp_ps_step(st, args.dt, tol=args.tol, rank_rtol=args.rank_rtol)
    t0 = time.perf_counter()
    tdvp_ps_step(st, args.dt, tol=args.tol, rank_rtol=args.rank_rtol)
    t_all = time.perf_counter() - t0
    cores = oracle_threads()
    out = {"value": sig((2 * N - 1) / t_all), "unit": UNIT, "cores": cores, "kind": "oracle",
           "host_cpus": os.cpu_count()}
    t_one = None
    with tempfile.NamedTemporaryFile(suffix=".pkl", delete=False) as f:
        pickle.dump((st, args.dt, args.tol, args.rank_rtol), f)
        path = f.name
    try:
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", _ONE_THREAD_STEP, ROOT, path], env=env, capture_output=True,
                           text=True, timeout=600)
        if r.returncode == 0:
            t_one = float(r.stdout.strip().splitlines()[-1])
            out["value_1thread"] = sig((2 * N - 1) / t_one)
    finally:
        os.unlink(path)
    one = f", step {args.warmup + 2} at 1 thread ({t_one:.1f} s)" if t_one else ""
    out["sample"] = (f"step {args.warmup + 1} with {cores} BLAS threads ({t_all:.1f} s){one}, after "
                     f"{args.warmup} untimed steps, tol {args.tol:g}")
    return out


def run_reference(args, world):
    """The reference arm: the CPU oracle, as it stands, on the timed arm's workload, tolerance and
    rank threshold, timing steps W+1.. of the same trajectory (bounded to ~150 s)."""
    p, cfg = workload(args)
    value, thr, n, secs = oracle_run(p, args, args.warmup, args.steps, budget_s=150.0)
    out = {"metric": METRIC, "value": sig(value), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": sig(1e3 * secs / n), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128 numpy/scipy)",
           "data": "synthetic (seeded FMO-sized FH chain)",
           "config": dict(cfg, precision="complex128", tol=args.tol, krylov="adaptive",
                          parallelism="CPU oracle (numpy/scipy, OpenBLAS threads)"),
           "impl": "reference",
           "cpu_baseline": {"kind": "oracle", "cores": thr, "value": sig(value), "unit": UNIT,
                            "sample": f"steps {args.warmup + 1}..{args.warmup + n} of the trajectory "
                                      f"({n} of the {args.steps} asked, 150 s budget), {secs:.1f} s"},
           "e2e": {"value": sig(value), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return out


def run_long(args):
    """Accuracy of the timed arm over a long run: `--long` steps of the timed arm (for every
    precision of --long-precisions) and of the FP64 reference (FP64 matvecs at --plain-tol,
    CUDA-graph steps) from the same product start; Eq. error and max |dP| every 100 steps (no
    timing).  Populations are written to <--long-dir>/long_<arm>.npy every 100 steps, so a run cut
    short still leaves its prefix."""
    import torch
    import paper_1907_12044_b300 as pkg
    p, cfg = workload(args)
    torch.cuda.set_device(0)
    if args.long_dir:
        os.makedirs(args.long_dir, exist_ok=True)
    precs = (args.long_precisions or args.precision).split(",")

    def run_arm(name, prec, tol, graph, learned, every, env_fp64=0):
        eng = pkg.Engine(n_realisations=1)
        eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
        eng.set_option(pkg.OPT_ENV_FP64, env_fp64)
        eng.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1 if every else 0)
        eng.build_mpo(0, p)
        eng.init_mps(0, args.D, p.exciton_site)
        eng.autotune()
        pops = [eng.observables(0)[0]]
        if learned:
            eng.controller_logging(1 << 20)
        for _ in range(args.warmup):
            eng.step(args.dt, 1, precision=PREC[prec], tol=tol)
            pops.append(eng.observables(0)[0])
        mode = pkg.KRYLOV_ADAPTIVE
        if learned:
            eng.controller_logging(0)
            train_controller(eng, samples=eng.stats()["krylov_solves"])
            mode = pkg.KRYLOV_LEARNED
        if graph:
            eng.set_option(pkg.OPT_GRAPH, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        path = os.path.join(args.long_dir, f"long_{name}.npy") if args.long_dir else None
        while len(pops) <= args.long:
            eng.step(args.dt, 1, precision=PREC[prec], krylov_mode=mode, tol=tol)
            pops.append(eng.observables(0)[0])
            if path and len(pops) % 100 == 1:
                np.save(path, np.array(pops))
        if path:
            np.save(path, np.array(pops))
        st = eng.stats()
        eng.close()
        return np.array(pops), time.perf_counter() - t0, st

    if args.long_ref:
        refP = np.load(args.long_ref)
        if refP.shape[0] < args.long + 1:
            raise SystemExit(f"--long-ref holds {refP.shape[0] - 1} steps, fewer than --long {args.long}")
        ref = (refP[:args.long + 1], None, None)
    else:
        ref = run_arm("fp64ref", *arm_setup(args, "fp64ref"))
    out = {"long_run": args.long, "config": cfg, "tol": args.tol,
           "reference": f"fp64, tol {args.plain_tol:g}, CUDA-graph steps" + (" (stored run)" if args.long_ref else ""),
           "reference_seconds": sig(ref[1]) if ref[1] else None, "final_pops_fp64": [sig(x, 6) for x in ref[0][-1]],
           "arms": {}}
    for entry in precs:
        # entry: prec[@tol][+env64]
        body, plus, flag = entry.partition("+")
        prec, _, tol_s = body.partition("@")
        _, tol, graph, learned, every = arm_setup(args, "mixed")
        tol = float(tol_s) if tol_s else tol
        env64 = 1 if (flag == "env64" or args.env_fp64) else 0
        P, secs, st = run_arm("mixed" if len(precs) == 1 else entry.replace("@", "_").replace("+", "_"), prec, tol,
                              graph, learned, every, env64)
        rows = []
        for s in list(range(100, args.long + 1, 100)) or [args.long]:
            e, m = pop_error(args.dt, P[:s + 1], ref[0][:s + 1])
            rows.append({"step": s, "t_fs": s * args.dt, "eq_error": sig(e, 3), "max_abs_dP": sig(m, 3)})
        out["arms"][entry] = {"errors": rows, "seconds": sig(secs), "precision": prec, "tol": tol, "env_fp64": env64,
                             "krylov_mean": sig(st["krylov_dim_sum"] / max(st["krylov_solves"], 1), 3),
                             "final_pops": [sig(x, 6) for x in P[-1]]}
    if len(precs) == 1:
        out["precision"] = precs[0]
        out["errors"] = out["arms"][precs[0]]["errors"]
    return out


def run_kernel_case(args):
    """--steps calls of one hot operation after --warmup untimed ones; CUDA events per call."""
    import torch
    import workloads as wl
    import paper_1907_12044_b300 as pkg
    p, cfg = workload(args)
    eng = pkg.Engine(n_realisations=1)
    rng = np.random.default_rng(1907)
    if args.kernel_case == "heff":
        eng.build_mpo(0, p)
        eng.init_mps_tensors(0, wl.random_mps_tensors(p.phys_dims(), args.D, seed=21))
        d, bd, _ = eng.chain_info(0)
        site = max(i for i in range(len(d)) if d[i] == max(d) and i < len(d) // 2)
        shape = (int(bd[site]), int(d[site]), int(bd[site + 1]))
        x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        call = lambda: eng.apply_heff(0, site, x, precision=PREC[args.precision])
        what = f"H_eff matvec at site {site}, shape {shape}, precision {args.precision}"
    else:
        eng.build_mpo(0, p)
        eng.init_mps(0, args.D, p.exciton_site)
        C = (rng.normal(size=(640, 8)) + 1j * rng.normal(size=(640, 8))) @ rng.normal(size=(8, 64))
        call = lambda: eng.debug_qr(C)
        what = "gauge-shift QR of a rank-8 640 x 64 complex matrix"
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    eng.reset_stats()
    eng.set_profiling(True)
    for _ in range(args.steps):
        call()
    eng.set_profiling(False)
    st = eng.stats()
    eng.close()
    dev_ms = {k: v / args.steps for k, v in st["prof_ms"].items() if v > 0}
    print(json.dumps({"kernel_case": args.kernel_case, "what": what, "calls": args.steps,
                      "device_ms_per_call": dev_ms, "launches_per_call": st["kernel_launches"] / args.steps}))


def run_ozaki_case(args):
    """The FP64 complex GEMM emulated on the BF16 tensor cores (tdvp_zgemm_ozaki) against cuBLAS
    ZGEMM (torch.matmul on complex128, the FP64 library GEMM) on the same device operands: CUDA
    events per call over --steps calls after --warmup, FLOP rate at 8 m n k, and the largest
    difference from the ZGEMM result relative to its largest element."""
    import torch
    import paper_1907_12044_b300 as pkg
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev).manual_seed(1907)
    rows = []
    for (m, n, k) in ((640, 64, 64), (1024, 1024, 1024), (4096, 4096, 4096)):
        A = torch.randn(m, k, dtype=torch.complex128, device=dev, generator=gen)
        B = torch.randn(k, n, dtype=torch.complex128, device=dev, generator=gen)

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / args.steps
        Cref = torch.empty(m, n, dtype=torch.complex128, device=dev)
        ms_ref = timed(lambda: torch.matmul(A, B, out=Cref))
        row = {"m": m, "n": n, "k": k, "zgemm_ms": round(ms_ref, 4),
               "zgemm_tflops": round(8.0 * m * n * k / (ms_ref * 1e-3) / 1e12, 3), "ozaki": {}}
        for sl in (8, 6):
            wsb = pkg.zgemm_ozaki_workspace(m, n, k, sl)
            ws = torch.empty(wsb // 8 + 128, dtype=torch.float64, device=dev)
            wp = (ws.data_ptr() + 1023) // 1024 * 1024
            C = torch.empty(m, n, dtype=torch.complex128, device=dev)
            call = lambda: pkg.zgemm_ozaki(m, n, k, A.data_ptr(), B.data_ptr(), C.data_ptr(), sl, wp, wsb,
                                           stream.cuda_stream)
            ms = timed(call)
            pkg.zgemm_ozaki_status(wp, stream.cuda_stream)
            rel = float((C - Cref).abs().max() / Cref.abs().max())
            row["ozaki"][f"slices{sl}"] = {"ms": round(ms, 4), "tflops_fp64_equiv": round(8.0 * m * n * k / (ms * 1e-3) / 1e12, 3),
                                           "speedup_vs_zgemm": round(ms_ref / ms, 2), "max_rel_diff": float(f"{rel:.2e}")}
            del ws, C
        rows.append(row)
        del A, B, Cref
        torch.cuda.empty_cache()
    print(json.dumps({"kernel_case": "ozaki", "calls": args.steps, "warmup": args.warmup, "cases": rows}))


def _compact(x):
    """Nested dicts without their null entries (the top level keeps every key)."""
    if isinstance(x, dict):
        return {k: _compact(v) for k, v in x.items() if v is not None}
    if isinstance(x, list):
        return [_compact(v) for v in x]
    return x


# headline comparisons, written last so that they sit in the end of the line a log keeps
TAIL_KEYS = ("speedup_vs_fp64", "speedup_vs_plain_fp64", "pop_error_vs_fp64", "pop_error_vs_fp64_arm",
             "controller_gain")


def emit(out, args):
    out = {k: (_compact(v) if isinstance(v, (dict, list)) else v) for k, v in out.items()}
    out = {**{k: v for k, v in out.items() if k not in TAIL_KEYS},
           **{k: out[k] for k in TAIL_KEYS if k in out}}
    line = json.dumps(out, ensure_ascii=False)
    print(line, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


def main():
    args = parse()
    if args.no_pdl:
        import paper_1907_12044_b300 as pkg
        e = pkg.Engine()
        e.set_option(pkg.OPT_PDL, 0)     # process-wide
        e.close()
    if args.kernel_case == "ozaki":
        run_ozaki_case(args)
        return
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.long:
        emit(run_long(args), args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            emit(run_reference(args, world), args)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.arms:
        out, p = run_ours(args, rank, world)
    else:                                   # batched section only (profiling captures)
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        p, cfg = workload(args)
        out = {"metric": METRIC, "config": cfg, "arms": {}}
        args.no_e2e = True
    if args.batched > 0:
        b, pops = run_batched(args, args.batched, rank, world)
        allp = gather_pops(pops, rank, world)
        if rank == 0:
            b["gathered_realisations"] = len(allp)
            out["batched"] = b
    if rank == 0:
        if not args.no_e2e:
            out["e2e"] = run_e2e(args, p)
        if not args.no_cpu_baseline and world == 1:
            try:
                out["cpu_baseline"] = cpu_baseline(p, args)
            except Exception as e:          # the GPU line stands without it
                out["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        emit(out, args)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
