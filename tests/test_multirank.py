"""The multi-rank parts of bench.py (replicas): the max-over-ranks timing
and the whole-job aggregate, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total_ms, evolve_s = bench.max_over_ranks([100.0 + 10 * rank, 2.0 - rank], dist, "cpu")
        out.put((rank, total_ms, evolve_s, bench.aggregate_value(6.0, world, evolve_s)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, evolve_s, value in res:
        assert total_ms == 110.0 and evolve_s == 2.0
        assert value == 6.0  # 2 ranks x 6 units / 2 s
