"""The multi-GPU form is replicas only (independent solves, no data-path collective): the bench's cross-rank logic
-- the slowest replica's time sets the job time, throughput = replicas x steps / that time -- on two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]
        m = bench.max_over_ranks(local_ms, dist, "cpu")
        e = bench.max_over_ranks([0.9, 0.7][rank], dist, "cpu")
        q.put((rank, m, e, bench.replica_throughput(world, 5, m)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, e, thr in res:
        assert m == 150.0 and e == 0.9
        assert abs(thr - 2 * 5 / 0.150) < 1e-9


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert abs(bench.replica_throughput(1, 5, 1000.0) - 5.0) < 1e-12
