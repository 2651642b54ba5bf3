"""The N > 1 host logic of the benchmark on CPU: two gloo ranks, each an
independent replica, reduce their times to the slowest rank's and report
whole-job throughput.  No GPU is used."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env()[:2] == (rank, world)
    ms = 100.0 + 50.0 * rank                # rank 1 is the slowest
    m = bench.reduce_max(ms, world, device="cpu")
    out[rank] = (m, bench.whole_job_mlups(1_000_000, 4, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_reduce_to_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        m, v = out[r]
        assert m == 150.0
        assert v == pytest.approx(2 * 4 * 1e6 / 0.150 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.whole_job_mlups(10, 2, 1, 1000.0) == pytest.approx(2e-5)
