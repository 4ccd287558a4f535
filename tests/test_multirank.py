"""The multi-rank parts, run as two gloo ranks on the CPU: bench.py's
max-over-ranks timing and whole-job aggregate, and the sharding of batched
instances (partition, evaluation of each share, one reduction of the
per-instance results) with the oracle standing in for the GPU."""
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


def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2104_03293_gb300 import instances as I, shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = I.config2(count=24, n_lo=6, n_hi=11, p_lo=1, p_hi=5)
        ns = [it[0].n for it in items]
        ps = [len(it[1]) for it in items]
        seen = []

        def compute(idx):
            seen.extend(int(i) for i in idx)
            return np.array([oracle.expect(items[i][0], items[i][1], items[i][2]) for i in idx])

        table = shard.sharded_results(ns, ps, compute, dist)
        out.put((rank, sorted(seen), table.tolist()))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_gloo():
    """Two ranks split a 24-instance batch; every instance is evaluated on
    exactly one rank, the work per rank is balanced to within the largest
    instance, and the combined table equals a one-rank evaluation."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2104_03293_gb300 import build, instances as I, qs
    build.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    items = I.config2(count=24, n_lo=6, n_hi=11, p_lo=1, p_hi=5)
    ns = [it[0].n for it in items]
    ps = [len(it[1]) for it in items]
    rank_of, load = qs.batch_partition(ns, ps, world)
    work = np.array([max(p, 1) * 2.0 ** n for n, p in zip(ns, ps)])
    assert sorted(res[0][1] + res[1][1]) == list(range(24))
    for r in range(world):
        assert res[r][1] == sorted(np.flatnonzero(rank_of == r).tolist())
    assert abs(load[0] - load[1]) <= work.max() and abs(load.sum() - work.sum()) < 1e-6
    ref = np.array([oracle.expect(it[0], it[1], it[2]) for it in items])
    for r in range(world):
        assert np.allclose(np.array(res[r][2]), ref, rtol=1e-12, atol=1e-14)  # host threads may differ per process


def test_partition_rules():
    """Longest-first greedy: deterministic, every rank used when there are
    enough instances, one rank takes everything."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2104_03293_gb300 import build, qs
    build.build()
    ns, ps = [20, 16, 16, 16, 16, 18], [1, 4, 4, 4, 4, 0]
    r, load = qs.batch_partition(ns, ps, 2)
    # work 2^20, then five equal 2^18 (4 x 2^16 and 1 x 2^18): the first goes
    # to rank 0, four fill rank 1 up to 2^20, the tie sends the last to rank 0
    assert r.tolist() == [0, 1, 1, 1, 1, 0]
    assert load.tolist() == [2.0 ** 20 + 2.0 ** 18, 2.0 ** 20]
    r1, l1 = qs.batch_partition(ns, ps, 1)
    assert r1.tolist() == [0] * 6
    with pytest.raises(qs.QSError):
        qs.batch_partition([35], [1], 2)
