"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas) agree on the
job time as the slowest rank's, and the whole-job value divides it by the
number of replicas."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")
    out.put((rank, got, bench.aggregate_time(got, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert [r[2] for r in res] == [7.5, 7.5]


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.25, None, "cpu") == 3.25
    assert bench.aggregate_time(12.0, 1) == 12.0
