"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups (no GPU).

bench.py runs one independent simulation per rank (replicas: a seed offset per rank, no
data-path collective); the job's time is the slowest rank's and its throughput counts the
units of every rank.  These tests run that host logic in two gloo ranks.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_16793_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        w = W.lwfa_3d_128x128x1024()
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_workload(w, rank).seed)
        scans = [None] * world
        dist.all_gather_object(scans, [v.seed for v in W.scan_2d(n=4, seed=W.SEED + 1000 * rank)])
        local_ms = 10.0 + 5.0 * rank                    # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, "cpu")
        rate = bench.job_rate(w.pushes_per_step * 3, world, ms / 1e3)
        out.put((rank, seeds, scans, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, seeds, scans, ms, rate = out.get(timeout=120)
        res[rank] = (seeds, scans, ms, rate)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2509_16793_gb300 import workloads as W
    w = W.lwfa_3d_128x128x1024()
    for rank in range(world):
        seeds, scans, ms, rate = res[rank]
        assert seeds == [w.seed, w.seed + 1]               # every rank its own plasma
        assert not set(scans[0]) & set(scans[1])           # scan instances differ per rank
        assert ms == 15.0                                  # the slowest rank's time
        assert rate == pytest.approx(2 * w.pushes_per_step * 3 / 0.015)


def test_oracle_baseline_on_several_host_cores():
    """The CPU baseline runs the oracle as it stands in spawned processes, one per core (each a
    seeded copy of the workload's window): the rate covers all their pushes over the wall time
    from the first start to the last end, and `cores` says how many ran."""
    import bench
    from paper_2509_16793_gb300 import workloads as W
    w = W.small_3d(nx=8, ny=8, nzeta=64, ppc=1)
    one = bench.oracle_sample(w, seconds=1e9, max_steps=1, procs=1)
    two = bench.oracle_sample(w, seconds=1e9, max_steps=1, procs=2)
    assert one["cores"] == 1 and two["cores"] == 2
    assert one["value"] > 0 and two["value"] > 0
    assert "2 process(es)" in two["sample"] and "2 s-step(s)" in two["sample"]
