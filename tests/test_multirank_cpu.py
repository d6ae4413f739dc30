"""The N > 1 path of bench.py on CPU: two gloo ranks, each running an independent replica (its own seed), the
job time taken as the maximum over ranks and the throughput aggregated over ranks.  No GPU and no data-path
collective: the emulated PEs of one problem live on one GPU, so ranks only meet in the timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W
        from paper_1702_00496_gb300 import at_delay
        spec, T = W.workload("1d_n16m")
        seed = bench.replica_seed(spec["seed"], rank)
        # this rank's delay stream: the first 64 draws of side 0
        draws = [at_delay(seed, n, 0, spec["L"]) for n in range(64)]
        t = 1.0 + 0.25 * rank  # a rank-dependent "time"
        tmax = bench.max_over_ranks(t, world)
        rate = bench.aggregate_rate(100.0, world, tmax)
        gathered = [None] * world
        dist.all_gather_object(gathered, (seed, draws, tmax, rate))
        if rank == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas_and_reduce_time_by_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (s0, d0, t0, r0), (s1, d1, t1, r1) = res
    assert s0 != s1                                   # distinct replicas
    assert d0 != d1                                   # distinct delay realizations
    assert t0 == t1 == 1.25                           # the slowest rank's time on every rank
    assert r0 == r1 == pytest.approx(2 * 100.0 / 1.25)
    assert set(np.unique(d0)) <= {0, 1, 2, 3}
