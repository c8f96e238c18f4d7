"""The N > 1 path of bench.py on CPU: world size 2 over gloo, each rank an
independent replica; only a barrier and a max of the timings cross ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    bench.init_replicas(world, rank, "gloo")
    bench.barrier(world)
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow replica
    m = bench.max_over_ranks(ms, world)
    out[rank] = (m, bench.replica_value(1000, 100, world, m))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_max_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0
    # whole-job throughput: both replicas' particles over the slowest time
    assert abs(out[0][1] - 2 * 1000 * 100 / 0.015) < 1e-6
