"""The multi-GPU mode's host logic with two gloo ranks on CPU.

The sweep shards by replicas: each rank runs its own sweeps with its own seeds (no
collective on the data path), the timed region ends at a barrier, the job's time is the
slowest rank's, and the value is the whole job's throughput (weak scaling).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    dist.barrier()
    total = bench.max_over_ranks(local_ms, world)
    out[rank] = (total, bench.replica_seed_base(rank), bench.whole_job_value(10.0, 5, world, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=120)
            assert pr.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0  # every rank reports the slowest rank's time
    assert res[0][1] != res[1][1]  # independent replicas: distinct seed streams
    assert res[0][2] == res[1][2] == pytest.approx(2 * 10.0 * 5 / 0.150)


def test_single_rank_needs_no_collective():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_value(3.0, 2, 1, 1000.0) == pytest.approx(6.0)
