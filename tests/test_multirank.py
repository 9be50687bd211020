"""The multi-rank host logic of bench.py on CPU, with two gloo ranks (world size 2).

Under torchrun every rank advances its own trajectory (replicas: a single TDVP-PS trajectory is
sequential along the chain, Eq. ps_trotter) and there is no data-path collective; the only
exchange is the all-reduce MAX of the timed region, so that the whole-job rate is taken over
the slowest rank.  Disorder realisations are independent: each rank takes the realisations
r = rank mod N, and rank 0 gathers the final populations over a host (gloo) group after the
timed region.  The reference arm runs on rank 0 only; the other ranks exit without work.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world)
        q.put((rank, ms, bench.site_update_rate(77, 3, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _batched_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    for d in (ROOT, os.path.join(ROOT, "tests")):
        if d not in sys.path:
            sys.path.insert(0, d)
    import types
    import torch
    import torch.distributed as dist
    import bench
    import paper_1907_12044_b300 as pkg
    from test_bench_host import FakeEngine, FakeEvent
    pkg.Engine = FakeEngine
    torch.cuda.synchronize = lambda *a: None
    torch.cuda.current_stream = lambda *a: types.SimpleNamespace(cuda_stream=0)
    torch.cuda.Event = FakeEvent
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = bench.parse(["--steps", "1", "--warmup", "2"])
        b, pops = bench.run_batched(args, 5, rank, world)
        allp = bench.gather_pops(pops, rank, world)
        q.put((rank, sorted(pops), None if allp is None else sorted(allp), b["per_rank"], b["value"]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_realisations_and_gather_populations():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batched_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert res[0][1] == [0, 2, 4] and res[1][1] == [1, 3]       # r on rank r mod 2
    assert res[0][2] == [0, 1, 2, 3, 4] and res[1][2] is None   # every realisation gathered on rank 0
    assert (res[0][3], res[1][3]) == (3, 2)
    assert res[0][4] == res[1][4] > 0                           # whole-job rate over the slowest rank


def test_two_gloo_ranks_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r[1] for r in res] == [150.0, 150.0]
    # 77 sites: 153 site updates per step and trajectory, 3 steps, 2 trajectories in 0.15 s
    assert res[0][2] == pytest.approx(153 * 3 * 2 / 0.150)
    assert res[1][2] == res[0][2]


def test_single_rank_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.site_update_rate(77, 3, 1, 1000.0) == pytest.approx(459.0)


def test_reference_arm_exits_without_work_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
