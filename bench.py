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
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32", "tf32x3"],
                    help="arithmetic of the Lanczos matvecs on the timed arm; FP64 is always timed beside it")
    ap.add_argument("--D", type=int, default=64)
    ap.add_argument("--dt", type=float, default=10.0)
    ap.add_argument("--tol", type=float, default=1e-12, help="Lanczos tolerance of the FP64 arm")
    ap.add_argument("--mixed-tol", type=float, default=1e-8,
                    help="Lanczos tolerance of the mixed-precision arms: the TF32x3 matvecs are accurate to "
                         "~1e-7 relative, so a tighter tolerance only adds iterations below that noise")
    ap.add_argument("--rank-rtol", type=float, default=1e-6,
                    help="rank threshold of the gauge-shift QR, the same on both arms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-prof", action="store_true", help="time without per-launch events")
    ap.add_argument("--no-learned", action="store_true", help="mixed arm without the learned Krylov controller")
    ap.add_argument("--only-timed-arm", action="store_true",
                    help="skip the FP64 reference arm (for profiling captures; no population error then)")
    ap.add_argument("--no-graph", action="store_true",
                    help="timed arm launch by launch instead of replaying each step as a CUDA graph "
                         "(the FP64 arm is always launch by launch: the plain method)")
    ap.add_argument("--no-pdl", action="store_true",
                    help="launch the step's kernels in plain stream order (no programmatic dependent launch)")
    ap.add_argument("--kernel-case", choices=["heff", "qr"], default=None,
                    help="time one hot operation at the bench's full-size shapes instead of steps (for "
                         "kernel captures): heff = one H_eff matvec at a bath-mode site of a random D-bond "
                         "state, qr = one gauge-shift QR of a rank-8 640 x 64 matrix")
    ap.add_argument("--batched", type=int, default=32,
                    help="also time R disorder realisations with ragged bond dims in the same launches (0: skip)")
    return ap.parse_args()


def workload(args):
    import workloads as wl
    p = wl.fmo_sized()
    return p, {"workload": f"{p.name}: {len(p.chain())} sites, D={args.D}, dt={args.dt} fs, product start",
               "model": "Frenkel-Holstein (synthetic FMO-sized, Debye bath)",
               "sites": len(p.chain()), "bond_dim": args.D, "dt_fs": args.dt,
               "krylov": f"adaptive Lanczos, tol {arm_tol(args, args.precision):g}", "precision": args.precision,
           "rank_rtol": args.rank_rtol,
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


PREC = {"fp64": 0, "tf32": 1, "tf32x3": 2}
TF32_OF_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor rate ratio


def arm_tol(args, precision):
    """Lanczos tolerance of an arm: --tol for FP64, --mixed-tol (else --tol) for TF32 / TF32x3."""
    return args.mixed_tol if (precision != "fp64" and args.mixed_tol is not None and args.mixed_tol > 0) else args.tol


def train_controller(eng, seed=0):
    """Train the learned Krylov controller on the solve log of the warm-up steps (GPU)."""
    from paper_1907_12044_b300.controller import init_weights
    eng.controller_set_weights(init_weights(seed))
    return eng.controller_train(epochs=150, batch=256, lr=3e-3)


def timed_run(args, p, precision, rank, world, dev, stream, flush, prof, learned=False):
    """W warm-up steps, then K timed steps (L2 flushed before each); returns timing and populations.

    The plain method tests Lanczos convergence at every k.  With ``learned`` the warm-up steps
    log their solves, the controller is trained on them and the timed steps use it.  A mixed arm
    replays each step as a CUDA graph (unless --no-graph): the last warm-up step captures it, and
    since per-launch events are not available inside a graph, one more step after the timed ones
    runs launch by launch with CUDA-event timing for the per-kernel breakdown."""
    import torch
    import paper_1907_12044_b300 as pkg
    graph = precision != "fp64" and not args.no_graph and args.warmup >= 1
    tol = arm_tol(args, precision)
    eng = pkg.Engine(n_realisations=1, stream=stream.cuda_stream)
    eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
    eng.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1)
    eng.build_mpo(0, p)
    eng.init_mps(0, args.D, p.exciton_site)
    eng.autotune()          # QR launch shape per gauge-shift shape (both arms)
    pops = [eng.observables(0)[0]]
    if learned:
        eng.controller_logging(1 << 20)
    for _ in range(args.warmup - (1 if graph else 0)):
        eng.step(args.dt, 1, precision=PREC[precision], tol=tol)
        pops.append(eng.observables(0)[0])
    ctl = None
    if learned:
        nlog = eng.stats()["krylov_solves"]
        eng.controller_logging(0)
        ctl = {"train_loss": train_controller(eng), "samples": int(nlog)}
    mode = pkg.KRYLOV_LEARNED if learned else pkg.KRYLOV_ADAPTIVE
    if graph:
        eng.set_option(pkg.OPT_GRAPH, 1)
        eng.step(args.dt, 1, precision=PREC[precision], krylov_mode=mode, tol=tol)   # capture
        pops.append(eng.observables(0)[0])
    torch.cuda.synchronize()
    eng.reset_stats()
    if prof and not graph:
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
            eng.step(args.dt, 1, precision=PREC[precision], krylov_mode=mode, tol=tol)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            pops.append(eng.observables(0)[0])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st = eng.stats()
    eng.set_profiling(False)
    if prof and graph:
        # per-kernel CUDA-event breakdown of one more (untimed) step, launch by launch
        eng.set_option(pkg.OPT_GRAPH, 0)
        eng.reset_stats()
        eng.set_profiling(True)
        eng.step(args.dt, 1, precision=PREC[precision], krylov_mode=mode, tol=tol)
        eng.set_profiling(False)
        ps = eng.stats()
        for k in ("prof_ms", "prof_flops", "prof_launches", "prof_bytes"):
            st[k] = {c: v * args.steps for c, v in ps[k].items()}
        st["prof_note"] = "per-kernel breakdown from one launch-by-launch step after the timed ones, x steps"
    eng.close()
    ms = max_over_ranks(float(np.sum(times)), world)
    return {"ms": ms, "stats": st, "pops": np.array(pops), "clocks": clk.summary(), "controller": ctl,
            "graph": graph}


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


# kernel and arithmetic of each timed category with algorithmic flop counts
ROOF_KERNELS = {"qr": ("bqr_kernel / cqr_kernel (FP64 gauge-shift QR, grid or cluster kernel autotuned per shape)",
                       "alu"),
                "gemm": ("zgemm_kernel (FP64 complex GEMM)", "alu"),
                "tc_gemm": ("tc_cgemm_kernel (tcgen05 kind::tf32)", "tensor"),
                "lanczos_vec": ("lz_start / lz_dots / lz_upd / lz_next / lz_combine (FP64 Lanczos vectors: "
                                "two Gram-Schmidt passes, next vector, combination)", "hbm")}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# kernel in its current form, on the bench's dominant shape; None where no such capture exists or
# the kernel has changed since (bqr_kernel: 0.89 MB per 640 x 64 rank-8 shift at commit 92e9268,
# profiles/bqr_rank8_640x64.md, before a change of its certain-drop margin)
TRAFFIC = {}


def roofline(args, st, cat):
    """Achieved vs peak for one timed category: algorithmic flops / summed CUDA-event time."""
    cat_ms = st["prof_ms"]
    total = sum(cat_ms.values())
    if cat not in ROOF_KERNELS:
        return {"kernel": cat, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "share_of_step": cat_ms[cat] / max(total, 1e-9),
                "note": "no algorithmic flop count for this category"}
    name, bound = ROOF_KERNELS[cat]
    ms, fl, nl = cat_ms[cat], st["prof_flops"][cat], st["prof_launches"][cat]
    if bound == "hbm":
        # algorithmic bytes (counted by the library per finished solve) / summed CUDA-event time
        by = st.get("prof_bytes", {}).get(cat, 0.0)
        ach = by / (ms * 1e-3) / 1e9 if ms > 0 and by > 0 else None
        pk = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        peak = pk.get("hbm_gbs", 6400.0)
        src = ("measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in pk
               else "fallback 6.4 TB/s (no MEASURED_PEAKS.json)")
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak if ach else None, "traffic": TRAFFIC.get(cat, (None, None))[0],
                "traffic_source": TRAFFIC.get(cat, (None, None))[1], "peak_source": src, "launches": nl,
                "algorithmic_bytes_per_launch": by / max(nl, 1),
                "avg_launch_us": 1e3 * ms / max(nl, 1), "share_of_step": ms / max(total, 1e-9),
                "note": "algorithmic bytes: 16 n (2 k (k+1) + 10 k + 5) per Lanczos solve of dimension k on "
                        "n complex elements (each iteration j reads V_0..V_j for the dot and the update of "
                        "both Gram-Schmidt passes); the vectors of a solve (<= 7 MB here) stay in L2, so "
                        "these launches are latency bound, far from the HBM roof"}
    ach = fl / (ms * 1e-3) / 1e12 if ms > 0 else None
    if bound == "tensor":
        pk = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {"bf16_tflops": 1800.0}
        peak = pk["bf16_tflops"] * TF32_OF_BF16
        src = "measured bf16 burst (MEASURED_PEAKS.json) x nominal tf32/bf16 ratio 1.1/2.25"
    else:
        peak, src = FP64_NOMINAL_TFLOPS, "B300 FP64 nominal 1.25 TFLOP/s (MEASURED_PEAKS.json has no FP64 entry)"
    return {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if ach else None, "traffic": TRAFFIC.get(cat, (None, None))[0],
            "traffic_source": TRAFFIC.get(cat, (None, None))[1], "peak_source": src, "launches": nl,
            "avg_launch_us": 1e3 * ms / max(nl, 1), "share_of_step": ms / max(total, 1e-9),
            "note": "algorithmic flops: 8 per complex multiply-add of the logical products "
                    "(QR: 2 n^2 m per n x m shift, two Gram-Schmidt passes)"}


def run_ours(args, rank, world):
    import torch
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    p, cfg = workload(args)
    N = len(p.chain())
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    prof = not args.no_prof
    run = None if args.precision == "fp64" else timed_run(args, p, args.precision, rank, world, dev, stream, flush, prof,
                                                          learned=not args.no_learned)
    ref = run if args.only_timed_arm and run is not None else timed_run(args, p, "fp64", rank, world, dev, stream,
                                                                        flush, prof)
    if run is None:
        run = ref
    value = site_update_rate(N, args.steps, world, run["ms"])
    fp64_value = site_update_rate(N, args.steps, world, ref["ms"])
    # population error of the timed arm against the FP64 arm on the same steps (Eq. error)
    t = args.dt * np.arange(len(run["pops"]))
    dP = np.abs(run["pops"] - ref["pops"])
    err = float(np.sum(0.5 * (dP.sum(1)[1:] + dP.sum(1)[:-1]) * np.diff(t)) / (p.n_el * t[-1])) if len(t) > 1 else 0.0
    st = run["stats"]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": run["ms"] / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64 (complex128)", "tf32": "tf32 tensor cores, f32 accumulate; f64 Lanczos/QR",
                     "tf32x3": "tf32x3 split tensor cores, f32 accumulate; f64 Lanczos/QR"}[args.precision],
           "data": "synthetic (seeded FMO-sized Frenkel-Holstein chain)",
           "config": dict(cfg, precision=args.precision,
                          execution=("each step replayed as one CUDA graph (a conditional while node per "
                                     "Lanczos exponential)") if run["graph"] else "launch by launch",
                          parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                          l2="flushed between timed steps (256 MiB write)"),
           "fp64_arm": {"value": fp64_value, "unit": UNIT, "ms_per_step": ref["ms"] / args.steps,
                        "krylov": f"adaptive, convergence tested at every k, tol {args.tol:g}",
                        "tri_evals_per_step": ref["stats"]["tri_evals"] / args.steps,
                        "kernel_time_ms": {k: round(v, 3) for k, v in ref["stats"]["prof_ms"].items()}},
           "learned_controller": run["controller"],
           "tri_evals_per_step": run["stats"]["tri_evals"] / args.steps,
           "speedup_vs_fp64": value / fp64_value,
           "pop_error_vs_fp64": {"eq_error_final": err, "max_abs_dP": float(dP.max()),
                                 "steps_compared": len(t) - 1},
           "gpu_launches": int(st["kernel_launches"]), "clocks": run["clocks"]}
    if prof:
        cat_ms = st["prof_ms"]
        top = max(cat_ms, key=cat_ms.get)
        out["roofline"] = roofline(args, st, top)
        if top != "tc_gemm" and args.precision != "fp64":
            out["roofline_tc_gemm"] = roofline(args, st, "tc_gemm")
        # the other large categories against their own roofs (QR: FP64 ALU, Lanczos vectors: HBM)
        out["roofline_other"] = {c: roofline(args, st, c) for c in ("qr", "lanczos_vec", "gemm")
                                 if c != top and cat_ms.get(c, 0) > 0}
        out["kernel_time_ms"] = {k: round(v, 3) for k, v in cat_ms.items()}
        out["dominant_category"] = top
    out["krylov"] = {"mean_dim": st["krylov_dim_sum"] / max(st["krylov_solves"], 1),
                     "max_dim": st["krylov_dim_max"], "host_syncs": st["host_syncs"]}
    return out, p


def run_batched(args, R):
    """R static-disorder realisations of the FMO-sized chain with bond dims drawn from
    {32,48,64,96,128}, advanced together; total site updates per second."""
    import torch
    import workloads as wl
    import paper_1907_12044_b300 as pkg
    base = wl.fmo_sized()
    Ds = wl.ragged_bond_dims(R)
    eng = pkg.Engine(n_realisations=R)
    eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
    for r in range(R):
        q = wl.disorder_realisation(base, r)
        eng.build_mpo(r, q)
        eng.init_mps(r, Ds[r], q.exciton_site)
    eng.autotune()
    eng.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1)
    graph = not args.no_graph and args.warmup >= 1
    if not args.no_learned:
        eng.controller_logging(1 << 22)
    for _ in range(args.warmup - (1 if graph else 0)):
        eng.step(args.dt, 1, precision=PREC[args.precision], tol=arm_tol(args, args.precision))
    mode = pkg.KRYLOV_ADAPTIVE
    if not args.no_learned:
        eng.controller_logging(0)
        train_controller(eng)
        mode = pkg.KRYLOV_LEARNED
    if graph:
        eng.set_option(pkg.OPT_GRAPH, 1)
        eng.step(args.dt, 1, precision=PREC[args.precision], krylov_mode=mode, tol=arm_tol(args, args.precision))   # capture
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    eng.reset_stats()
    e0.record(stream)
    eng.step(args.dt, args.steps, precision=PREC[args.precision], krylov_mode=mode, tol=arm_tol(args, args.precision))
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = eng.stats()
    eng.close()
    N = len(base.chain())
    return {"realisations": R, "bond_dims": "ragged from {32,48,64,96,128} (seed 12044)",
            "precision": args.precision, "value": (2 * N - 1) * R * args.steps / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms / args.steps, "gpu_launches": int(st["kernel_launches"]),
            "qr_blocks": "autotuned", "krylov": "learned controller" if not args.no_learned else "adaptive",
            "execution": "each step of all realisations replayed as one CUDA graph" if graph else "launch by launch"}


def run_e2e(args, p):
    """The timed arm's workload end to end through the public API, on the host clock: the same
    options, warm-up steps and controller training (untimed), then --steps steps, each followed
    by a device->host read of that step's populations, energy and norm.  The MPO parameters and
    the initial state go host->device once, before the warm-up; the state stays resident."""
    import torch
    import paper_1907_12044_b300 as pkg
    N = len(p.chain())
    t0 = time.perf_counter()
    eng = pkg.Engine(n_realisations=1)
    eng.set_option(pkg.OPT_RANK_RTOL, args.rank_rtol)
    eng.set_option(pkg.OPT_KRYLOV_CHECK_ALL, 1)
    eng.build_mpo(0, p)
    eng.init_mps(0, args.D, p.exciton_site)
    torch.cuda.synchronize()
    upload_s = time.perf_counter() - t0
    eng.autotune()
    learned = args.precision != "fp64" and not args.no_learned
    graph = args.precision != "fp64" and not args.no_graph and args.warmup >= 1
    if learned:
        eng.controller_logging(1 << 20)
    for _ in range(args.warmup - (1 if graph else 0)):
        eng.step(args.dt, 1, precision=PREC[args.precision], tol=arm_tol(args, args.precision))
    mode = pkg.KRYLOV_ADAPTIVE
    if learned:
        eng.controller_logging(0)
        train_controller(eng)
        mode = pkg.KRYLOV_LEARNED
    if graph:
        eng.set_option(pkg.OPT_GRAPH, 1)
        eng.step(args.dt, 1, precision=PREC[args.precision], krylov_mode=mode, tol=arm_tol(args, args.precision))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        eng.step(args.dt, 1, precision=PREC[args.precision], krylov_mode=mode, tol=arm_tol(args, args.precision))
        pops, E, nrm = eng.observables(0)
    dt = time.perf_counter() - t0
    d, bd, w = eng.chain_info(0)
    f = p.flat()
    h2d_once = sum(np.asarray(v).nbytes for v in f.values()) + sum(
        16 * int(bd[i]) * int(d[i]) * int(bd[i + 1]) for i in range(N))
    eng.close()
    return {"value": (2 * N - 1) * args.steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * (p.n_el + 2),
            "includes": "steps through Engine.step and a populations/energy/norm readback after each; "
                        "state resident on the device between steps",
            "h2d_bytes_once": h2d_once, "upload_and_build_s": upload_s}


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
        tdvp_ps_step(st, args.dt, tol=args.tol, rank_rtol=args.rank_rtol)
    dt = time.perf_counter() - t0
    return (2 * N - 1) * n_steps / dt, threads, dt


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


def main():
    args = parse()
    if args.no_pdl:
        import paper_1907_12044_b300 as pkg
        e = pkg.Engine()
        e.set_option(pkg.OPT_PDL, 0)     # process-wide
        e.close()
    if args.kernel_case:
        run_kernel_case(args)
        return
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
        if args.batched > 0:
            out["batched"] = run_batched(args, args.batched)
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
