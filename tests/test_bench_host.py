"""bench.py's host side on CPU: the JSON line assembled around a stand-in engine.

The stand-in replaces only the CUDA library (steps, statistics, populations) and the CUDA timing
calls; the bench's own arithmetic (rates, population error, rooflines, JSON assembly) runs as it
does on a GPU, so a change to the bench is checked here before it reaches a GPU.
"""
import json
import sys
import time
import types

import numpy as np

import bench

CATS = ["gemm", "wapply", "lanczos_vec", "tridiag", "qr", "other", "tc_gemm"]
PHASES = ["Deriv-Forward", "Deriv-Backward", "Krylov", "QR", "MatMul-QR", "Get Env", "other"]


class FakeEngine:
    def __init__(self, n_realisations=1, kmax=64, device=0, stream=None):
        self.t = 0
        self.prof = False
        self.precisions = []
        self._reset()

    def _reset(self):
        self.s = {"steps": 0, "site_updates": 0, "matvecs": 0, "krylov_solves": 0, "krylov_dim_sum": 0,
                  "krylov_dim_max": 0, "host_syncs": 0, "kernel_launches": 0, "not_converged": 0,
                  "tri_evals": 0, "prof_ms": dict.fromkeys(CATS, 0.0), "prof_launches": dict.fromkeys(CATS, 0),
                  "prof_flops": dict.fromkeys(CATS, 0.0), "prof_bytes": dict.fromkeys(CATS, 0.0),
                  "prof_phase_ms": dict.fromkeys(PHASES, 0.0), "prof_phase_launches": dict.fromkeys(PHASES, 0)}

    def set_option(self, *a):
        pass

    def build_mpo(self, r, p):
        self.n_el = p.n_el
        self.d = np.asarray(p.phys_dims(), np.int32)

    def chain_info(self, r=0):
        n = len(self.d)
        return self.d, np.ones(n + 1, np.int32), np.ones(n + 1, np.int32)

    def init_mps(self, r, D, site):
        self.inits = getattr(self, "inits", 0) + 1

    def autotune(self):
        pass

    def controller_logging(self, n):
        pass

    def controller_set_weights(self, w):
        pass

    def controller_train(self, epochs=20, batch=1024, lr=1e-3):
        return 0.5, 0.4

    def reset_stats(self):
        self._reset()

    def set_profiling(self, on=True):
        self.prof = on

    def step(self, dt, n_steps=1, precision=0, krylov_mode=0, tol=1e-12):
        self.t += n_steps
        self.precisions.append(precision)
        s = self.s
        s["steps"] += n_steps
        s["krylov_solves"] += 305 * n_steps
        s["krylov_dim_sum"] += 6 * 305 * n_steps
        s["krylov_dim_max"] = 9
        s["kernel_launches"] += 19000 * n_steps
        s["tri_evals"] += 400 * n_steps
        if self.prof:
            for i, c in enumerate(CATS):
                s["prof_ms"][c] += 10.0 * (i + 1)
                s["prof_launches"][c] += 100 * (i + 1)
            s["prof_flops"]["qr"] += 6.4e9
            s["prof_flops"]["tc_gemm"] += 3.7e11
            s["prof_flops"]["gemm"] += 1e10
            s["prof_bytes"]["lanczos_vec"] += 1.8e10
            s["prof_flops"]["lanczos_vec"] += 2e9
            for i, ph in enumerate(PHASES):
                s["prof_phase_ms"][ph] += 5.0 * (i + 1)
        time.sleep(0.002)

    def stats(self):
        return json.loads(json.dumps(self.s))

    def observables(self, r=0):
        P = np.full(self.n_el, 1.0 / self.n_el)
        P[0] += 1e-9 * self.t * (1 + (2 in self.precisions))
        return P, 1.0, 1.0

    def close(self):
        pass


class FakeEvent:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return max(1e-3, (other.t - self.t) * 1e3)


def _patch(monkeypatch):
    import torch
    import paper_1907_12044_b300 as pkg
    monkeypatch.setattr(pkg, "Engine", FakeEngine)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    real_zeros = torch.zeros
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: real_zeros(4, dtype=k.get("dtype")))


def test_bench_line_is_complete_with_a_stand_in_engine(monkeypatch):
    _patch(monkeypatch)
    args = bench.parse(["--batched", "0", "--no-e2e", "--no-cpu-baseline"])
    out, p = bench.run_ours(args, 0, 1)
    line = json.loads(json.dumps(out))
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "arms", "speedup_vs_fp64", "speedup_vs_plain_fp64",
              "pop_error_vs_fp64", "pop_error_vs_fp64_arm", "gpu_launches", "clocks", "roofline",
              "kernel_share"):
        assert k in line, k
    n = len(p.chain())
    assert line["value"] > 0 and line["arms"]["fp64"]["value"] > 0 and line["arms"]["plain"]["value"] > 0
    assert abs(line["value"] * line["ms_per_step"] / 1e3 - (2 * n - 1)) < 1e-3 * (2 * n - 1)
    assert line["config"]["workload"].startswith(p.name)
    assert line["pop_error_vs_fp64"]["max_abs_dP"] > 0
    # the arms differ only where they should: the FP64 arm keeps the timed arm's tolerance, graph
    # and controller; the plain arm is FP64 at the tight tolerance, launch by launch, every k
    t, f, pl = line["arms"]["timed"], line["arms"]["fp64"], line["arms"]["plain"]
    assert (t["tol"], t["graph"], t["learned"]) == (f["tol"], f["graph"], f["learned"]) == (1e-8, True, True)
    a = line["arms"]["adaptive"]
    assert (a["precision"], a["tol"], a["graph"], a["learned"]) == ("tf32x3", 1e-8, True, False)
    assert line["controller_gain"]["wall"] > 0
    assert t["precision"] == "tf32x3" and f["precision"] == "fp64"
    assert (pl["precision"], pl["tol"], pl["graph"], pl["learned"], pl["every_k"]) == ("fp64", 1e-12, False, False, True)
    assert set(t["phase_ms"]) == set(PHASES)
    # the stand-in's largest category is tc_gemm (tensor roof); the others keep their own roofs
    roof = line["roofline"]
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s" and 0 < roof["frac"] < 1
    other = line["roofline_other"]
    # the Lanczos orthogonalisation against the FP64 peak, its HBM rate beside it
    assert other["lanczos_vec"]["bound"] == "alu" and other["lanczos_vec"]["unit"] == "TFLOP/s"
    assert abs(other["lanczos_vec"]["achieved"] - 2e9 / 30e-3 / 1e12) < 1e-3 * 2e9 / 30e-3 / 1e12
    # Sec. 8(d)'s count: k(k+1)/2 vector reads per solve, from the library's 4-pass count at k = 6
    k = 6.0
    alg = 1.8e10 * (0.5 * k * (k + 1)) / (2 * k * (k + 1) + 10 * k + 5)
    assert abs(other["lanczos_vec"]["hbm_gbs"] - alg / 30e-3 / 1e9) < 1e-3 * alg / 30e-3 / 1e9
    assert other["qr"]["bound"] == "alu" and other["qr"]["frac"] > 0
    assert len(json.dumps(out)) < 4000


def test_headline_comparisons_close_the_line(monkeypatch, tmp_path, capsys):
    """A log that keeps only the end of the line still holds the mixed-vs-FP64 comparisons."""
    _patch(monkeypatch)
    args = bench.parse(["--batched", "0", "--no-e2e", "--no-cpu-baseline", "--out", str(tmp_path / "l.json")])
    out, _ = bench.run_ours(args, 0, 1)
    out["cpu_baseline"] = {"value": 1.0, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "x" * 300}
    bench.emit(out, args)
    line = capsys.readouterr().out.strip().splitlines()[-1]
    assert list(json.loads(line))[-len(bench.TAIL_KEYS):] == list(bench.TAIL_KEYS)
    for k in bench.TAIL_KEYS:
        assert f'"{k}"' in line[-1500:], k


def test_batched_and_e2e_sections_with_a_stand_in_engine(monkeypatch):
    _patch(monkeypatch)
    args = bench.parse(["--steps", "2"])
    b, pops = bench.run_batched(args, 3)
    b = json.loads(json.dumps(b))
    assert b["realisations"] == 3 and b["value"] > 0 and b["unit"] == bench.UNIT and sorted(pops) == [0, 1, 2]
    p, _ = bench.workload(args)
    e = json.loads(json.dumps(bench.run_e2e(args, p)))
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in e, k
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert e["steps"] == args.warmup + args.steps


def test_batched_compare_check_and_profile_sections_with_a_stand_in_engine(monkeypatch):
    _patch(monkeypatch)
    args = bench.parse(["--steps", "1", "--batched-compare", "--batched-check", "--batched-prof"])
    b, _ = bench.run_batched(args, 4)
    b = json.loads(json.dumps(b))
    cmp = b["controller_vs_default"]
    for k in ("adaptive_ms_per_step", "learned_ms_per_step", "wall_gain", "tri_evals_per_solve_adaptive",
              "krylov_mean_adaptive"):
        assert k in cmp and cmp[k] > 0, k
    chk = b["check_vs_single"]                  # smallest and largest D of this rank's realisations
    assert len(chk["realisations"]) == 2 and set(chk["realisations"]) <= set(range(4))
    assert chk["bond_dims"][0] <= chk["bond_dims"][1] and chk["max_rel_dP"] >= 0
    assert b["profile"]["phase_ms"] and b["profile"]["kernel_ms"]


def test_realisation_shards_cover_every_index_once():
    for R, world in ((256, 8), (32, 3), (5, 8), (1, 2)):
        got = sorted(r for rank in range(world) for r in bench.shard(R, rank, world))
        assert got == list(range(R))
        sizes = [len(bench.shard(R, rank, world)) for rank in range(world)]
        assert max(sizes) - min(sizes) <= 1


def test_long_accuracy_run_with_a_stand_in_engine(monkeypatch, tmp_path):
    _patch(monkeypatch)
    args = bench.parse(["--long", "250", "--warmup", "1", "--long-dir", str(tmp_path)])
    out = json.loads(json.dumps(bench.run_long(args)))
    assert [r["step"] for r in out["errors"]] == [100, 200]
    assert all(r["max_abs_dP"] > 0 for r in out["errors"])
    assert np.load(tmp_path / "long_mixed.npy").shape == (251, 7)
    assert np.load(tmp_path / "long_fp64ref.npy").shape == (251, 7)
    args = bench.parse(["--long", "120", "--warmup", "1", "--long-dir", str(tmp_path),
                        "--long-precisions", "tf32x3,bf16x3"])
    out = json.loads(json.dumps(bench.run_long(args)))
    assert sorted(out["arms"]) == ["bf16x3", "tf32x3"] and out["arms"]["bf16x3"]["errors"][0]["step"] == 100
    # a stored reference and a per-arm tolerance
    args = bench.parse(["--long", "100", "--warmup", "1", "--long-dir", str(tmp_path / "b"),
                        "--long-ref", str(tmp_path / "long_fp64ref.npy"), "--long-precisions", "tf32x3@1e-10"])
    out = json.loads(json.dumps(bench.run_long(args)))
    assert out["arms"]["tf32x3@1e-10"]["tol"] == 1e-10 and out["reference_seconds"] is None


def test_bench_population_error_equals_the_oracle_metric():
    """bench.pop_error (Eq. error at the last time, trapezoid in time) against the oracle's
    mean_cumulative_deviation on the same random populations, and max |dP|."""
    from oracle import mean_cumulative_deviation
    rng = np.random.default_rng(5)
    P, Pref = rng.random((41, 7)), rng.random((41, 7))
    e, m = bench.pop_error(10.0, P, Pref)
    t = 10.0 * np.arange(41)
    assert abs(e - mean_cumulative_deviation(t, P, Pref)) <= 1e-15 * max(1.0, e)
    assert m == np.abs(P - Pref).max()
