"""The benchmark's multi-GPU path (independent replicas, one process per GPU), host side:
the whole-job figures over two gloo ranks on CPU are the slowest rank's time and the sum
of every rank's units, as the JSON line's value (units of all ranks / that time) needs."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r: 10 (r + 1) ms, units (r + 1, 100, 7 r)
    ms, counts = bench.job_totals(10.0 * (rank + 1), [rank + 1, 100, 7 * rank], dist, "cpu")
    dist.barrier()
    q.put((rank, ms, counts))
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in results] == [0, 1]
    for _, ms, counts in results:
        assert ms == 20.0                     # the slowest rank's time, on every rank
        assert counts == [3.0, 200.0, 7.0]    # every rank's units


def test_job_totals_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(5.0, [1, 2], None, "cpu") == (5.0, [1.0, 2.0])
