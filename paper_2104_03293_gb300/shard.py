"""Batched instances over several ranks (one GPU each).

Instances are independent problems, so a batch shards without any exchange
on the data path: every rank takes the partition of qs_batch_partition
(greedy longest-first on max(p, 1) 2^n, identical on every rank), evolves
its own share as one qs_batch on its GPU, and the per-instance results are
combined at the end with one sum-reduction of a (count x width) table in
which each row is written by exactly one rank (2 doubles per instance for
E and P_ground, or 2p for gradients).  The only collective is that final
reduction; with one rank nothing is exchanged.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from . import qs


def local_indices(ns: Sequence[int], ps: Sequence[int], rank: int, world: int) -> np.ndarray:
    """Indices of the instances that rank `rank` of `world` evolves."""
    rank_of, _ = qs.batch_partition(ns, ps, world)
    return np.flatnonzero(rank_of == rank)


def combine(count: int, width: int, idx: np.ndarray, rows: np.ndarray, dist=None, device="cpu") -> np.ndarray:
    """The (count x width) table whose rows idx are `rows` on this rank and
    whose other rows come from the ranks that own them (one all-reduce)."""
    table = np.zeros((count, width))
    if len(idx):
        table[np.asarray(idx)] = np.asarray(rows, dtype=np.float64).reshape(len(idx), width)
    if dist is None or dist.get_world_size() == 1:
        return table
    import torch
    t = torch.from_numpy(table).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def sharded_results(ns, ps, compute: Callable[[np.ndarray], np.ndarray], dist=None, device="cpu"):
    """Evaluate every instance on the rank the partition gives it and return
    the combined (count x width) result table on every rank.  `compute`
    receives this rank's instance indices and returns one row per index."""
    world = dist.get_world_size() if dist is not None else 1
    rank = dist.get_rank() if dist is not None else 0
    idx = local_indices(ns, ps, rank, world)
    rows = np.asarray(compute(idx), dtype=np.float64).reshape(len(idx), -1) if len(idx) else np.zeros((0, 0))
    width = rows.shape[1] if len(idx) else 0
    if dist is not None and world > 1:
        import torch
        w = torch.tensor([width], dtype=torch.int64, device=device)
        dist.all_reduce(w, op=dist.ReduceOp.MAX)
        width = int(w.item())
        if rows.shape[1] != width:
            rows = np.zeros((len(idx), width))
    return combine(len(ns), width, idx, rows, dist, device)


def batch_readout(items, dist=None, device="cpu", stream=None):
    """E and P_ground of every (instance, gamma, beta) item, each rank
    evolving its share on its own GPU as one batch.  Returns (E, P) arrays
    of len(items) on every rank."""
    ns = [it[0].n for it in items]
    ps = [len(it[1]) for it in items]

    def compute(idx):
        bt = qs.Batch([ns[i] for i in idx], stream=stream)
        try:
            for j, i in enumerate(idx):
                inst = items[i][0]
                bt.set_ising(j, inst.h, inst.edges, inst.J)
            bt.evolve([items[i][1] for i in idx], [items[i][2] for i in idx])
            E, P = bt.results()
        finally:
            bt.close()
        return np.stack([E, P], axis=1)

    table = sharded_results(ns, ps, compute, dist, device)
    return table[:, 0], table[:, 1]
