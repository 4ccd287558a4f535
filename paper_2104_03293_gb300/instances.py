"""Seeded synthetic Ising instances and angle sets.

This module draws random inputs and nothing else: it holds none of the
method's arithmetic (no cost evaluation, no state evolution, no angle map).
Both the CUDA path and the CPU oracle consume what it produces, so that the
two sides are always fed identical instances.

An instance is the problem Hamiltonian of Eq. (HC),
``H_C = sum_i h_i Z_i + sum_{i<j} J_ij Z_i Z_j``, stored as
``(n, h[n], edges[m, 2] with i < j, J[m])``.  The exact-cover instances of the
paper (Sec. III.A.3) are not available, so seeded graphs of the shapes named
for each workload stand in for them:

* 3-regular MaxCut: J_ij = +1 on the edges of a random 3-regular graph,
  h_i = 0 (configuration model with rejection of loops and multi-edges).
* Erdos-Renyi Ising: G(n, d/(n-1)) with mean degree d, integer h and J drawn
  uniformly from a symmetric range (optionally excluding J = 0).
* Factorised instances: the union of independent components on disjoint,
  contiguous qubit ranges (the state is then a tensor product).
* Exact-cover problem matrices with a planted solution (the problem class of
  the paper, whose own instances are not available); the mapping to H_C is
  part of the method and lives in the package, not here.

Seeds follow ``seed = 2104032930 + 1000 * config + index``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

SEED_BASE = 2104032930


def workload_seed(config: int, index: int = 0) -> int:
    """Seed of instance ``index`` of workload ``config``."""
    return SEED_BASE + 1000 * int(config) + int(index)


@dataclass
class Instance:
    """Ising problem ``H_C`` of Eq. (HC): fields ``h`` and weighted edges."""

    n: int
    h: np.ndarray                      # float64 [n]
    edges: np.ndarray                  # int32 [m, 2], i < j, no duplicates
    J: np.ndarray                      # float64 [m]
    name: str = ""
    components: List[range] = field(default_factory=list)

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])

    def copy(self) -> "Instance":
        return Instance(self.n, self.h.copy(), self.edges.copy(), self.J.copy(),
                        self.name, list(self.components))


def _canon(n, h, edge_list, J, name, components=None) -> Instance:
    if len(edge_list):
        e = np.asarray(edge_list, dtype=np.int64)
        e = np.sort(e, axis=1)
        order = np.lexsort((e[:, 1], e[:, 0]))
        e = e[order]
        Jv = np.asarray(J, dtype=np.float64)[order]
    else:
        e = np.zeros((0, 2), dtype=np.int64)
        Jv = np.zeros(0, dtype=np.float64)
    return Instance(int(n), np.asarray(h, dtype=np.float64).copy(),
                    np.ascontiguousarray(e, dtype=np.int32), np.ascontiguousarray(Jv),
                    name, list(components or [range(0, n)]))


def random_regular3(n: int, rng: np.random.Generator, max_tries: int = 10000):
    """Edges of a uniformly drawn simple 3-regular graph on n nodes (n even)."""
    if n % 2 or n < 4:
        raise ValueError("a 3-regular graph needs an even n >= 4")
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        p = np.sort(pairs, axis=1)
        if len({(int(a), int(b)) for a, b in p}) != len(p):
            continue
        return [(int(a), int(b)) for a, b in p]
    raise RuntimeError("configuration model failed to produce a simple graph")


def maxcut_regular3(n: int, seed: int) -> Instance:
    """MaxCut on a seeded random 3-regular graph: J_ij = +1, h_i = 0."""
    rng = np.random.default_rng(seed)
    edges = random_regular3(n, rng)
    return _canon(n, np.zeros(n), edges, np.ones(len(edges)), f"maxcut3r_n{n}_s{seed}")


def erdos_renyi_ising(n: int, seed: int, mean_degree: float = 4.0,
                      h_values: Sequence[int] = (-2, -1, 0, 1, 2),
                      j_values: Sequence[int] = (-2, -1, 1, 2)) -> Instance:
    """Integer Ising weights on G(n, mean_degree/(n-1))."""
    rng = np.random.default_rng(seed)
    prob = min(1.0, mean_degree / max(n - 1, 1))
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < prob
    edges = list(zip(iu[keep].tolist(), ju[keep].tolist()))
    h = rng.choice(np.asarray(h_values, dtype=np.float64), size=n)
    J = rng.choice(np.asarray(j_values, dtype=np.float64), size=len(edges))
    return _canon(n, h, edges, J, f"er{mean_degree:g}_n{n}_s{seed}")


def union(parts: Sequence[Instance], name: str = "") -> Instance:
    """Disjoint union: part k occupies the next contiguous block of qubits."""
    n = 0
    h, edges, J, comps = [], [], [], []
    for p in parts:
        h.append(p.h)
        edges.extend((int(a) + n, int(b) + n) for a, b in p.edges)
        J.append(p.J)
        comps.append(range(n, n + p.n))
        n += p.n
    return _canon(n, np.concatenate(h), edges, np.concatenate(J) if J else [],
                  name or "union_" + "_".join(p.name for p in parts), comps)


def exact_cover(n: int, f: int, seed: int, extra_density: float | None = None):
    """A random exact-cover problem matrix a in {0,1}^{n x f} (rows =
    variables, columns = the f elements to cover) with a planted solution:
    a random half of the variables (at least one) split the columns among
    them, one owner per column; every other variable covers each column with
    probability ``extra_density`` (default: the owners' mean density).
    Returns (a as int8 [n, f], planted x as int8 [n])."""
    rng = np.random.default_rng(seed)
    x = np.zeros(n, dtype=np.int8)
    owners = rng.choice(n, size=max(1, n // 2), replace=False)
    x[owners] = 1
    a = np.zeros((n, f), dtype=np.int8)
    a[rng.choice(owners, size=f), np.arange(f)] = 1
    q = 1.0 / owners.size if extra_density is None else float(extra_density)
    rest = np.flatnonzero(x == 0)
    a[rest] = (rng.random((rest.size, f)) < q).astype(np.int8)
    return a, x


def uniform_angles(p: int, seed: int, lo: float = 0.0, hi: float = np.pi):
    """QAOA angles gamma_k, beta_k ~ U[lo, hi) (float64 arrays of length p)."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(lo, hi, size=p)
    b = rng.uniform(lo, hi, size=p)
    return g, b


# ----------------------------------------------------------------------------
# Named workloads (shapes of the paper's workloads, synthetic stand-ins)
# ----------------------------------------------------------------------------

def config1(n: int = 12, p: int = 2):
    """Plain forward: 3-regular MaxCut, QAOA angles ~ U[0, pi)."""
    inst = maxcut_regular3(n, workload_seed(1, 0))
    g, b = uniform_angles(p, workload_seed(1, 1))
    return inst, g, b


def config2(count: int = 512, n_lo: int = 16, n_hi: int = 24, p_lo: int = 1, p_hi: int = 10):
    """Batched forwards: n ~ U{16..24}, p ~ U{1..10}, ER(4), h,J in U{-2..2}, J != 0."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(workload_seed(2, i))
        n = int(rng.integers(n_lo, n_hi + 1))
        p = int(rng.integers(p_lo, p_hi + 1))
        inst = erdos_renyi_ising(n, workload_seed(2, i) + 500_000)
        g, b = uniform_angles(p, workload_seed(2, i) + 700_000)
        out.append((inst, g, b))
    return out


def config3(n: int = 26, p: int = 10, kind: str = "maxcut"):
    """Adjoint gradient: 3-regular MaxCut (or the ER(4) integer Ising variant)."""
    if kind == "maxcut":
        inst = maxcut_regular3(n, workload_seed(3, 0))
    else:
        inst = erdos_renyi_ising(n, workload_seed(3, 0))
    g, b = uniform_angles(p, workload_seed(3, 1))
    return inst, g, b


def config4(count: int = 64, n_lo: int = 18, n_hi: int = 22, p_lo: int = 5, p_hi: int = 20):
    """Batched optimiser loop: n ~ U{18..22}, p ~ U{5..20}, tau cycles 0.5/0.75/1.0."""
    taus = (0.5, 0.75, 1.0)
    out = []
    for i in range(count):
        rng = np.random.default_rng(workload_seed(4, i))
        n = int(rng.integers(n_lo, n_hi + 1))
        p = int(rng.integers(p_lo, p_hi + 1))
        inst = erdos_renyi_ising(n, workload_seed(4, i) + 500_000)
        out.append((inst, p, taus[i % 3]))
    return out


def config5(n: int = 34, p: int = 20, tau: float = 0.75):
    """Largest single-GPU instance: ER(4), h, J in U{-1,0,1}, AQA p = 20 knots."""
    inst = erdos_renyi_ising(n, workload_seed(5, 0), h_values=(-1, 0, 1), j_values=(-1, 0, 1))
    s = np.arange(1, p + 1, dtype=np.float64) / (p + 1)
    return inst, s, tau
