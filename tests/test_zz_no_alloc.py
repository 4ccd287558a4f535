"""qs_enumerate_noalloc (static device scratch, no allocation) against the
allocating entry point qs_set_ising / qs_cost_info, through the C ABI, and
against the oracle's enumeration.

Both entry points run the same integer enumeration, so their results must
be identical.  The two no-alloc calls run back to back on different
instances, so a result left over in the shared scratch from the first call
would show in the second.  Beyond the single-state range (35 to 40 qubits,
which the no-alloc limit opens) the instances are disjoint unions of
components the oracle enumerates one by one: the minimum and maximum add,
the lowest argmin is the components' argmins side by side and the count is
the product.  Collected last: it must pass in a fresh process and after the
other GPU tests.
"""
import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2104_03293_gb300 import build, qs as _qs
    build.build()
    return _qs


def _half_integer(inst, seed):
    rng = np.random.default_rng(seed)
    J = inst.J + 0.5 * rng.integers(0, 2, size=inst.J.shape)
    return inst.h - 0.25 * rng.integers(0, 2, size=inst.h.shape), inst.edges, J


def _allocating(qs, n, h, edges, J):
    with qs.State(n) as s:
        s.set_ising(h, edges, J)
        return s.cost_info()


def test_noalloc_matches_cost_info_on_two_calls(qs):
    a = I.maxcut_regular3(20, seed=11)
    b_inst = I.erdos_renyi_ising(23, seed=12, mean_degree=5.0)
    cases = [(a.n, a.h, a.edges, a.J), (b_inst.n,) + _half_integer(b_inst, 13)]
    got = [qs.enumerate_noalloc(h, e, J) for _, h, e, J in cases]  # two calls in a row
    want = [_allocating(qs, n, h, e, J) for n, h, e, J in cases]
    assert got == want
    assert got[1][4] == 2  # quarter-integer fields: costs in units of 2^-2


def test_noalloc_small_and_repeated(qs):
    # n < 6 (fewer qubits than the 6 register bits of the enumeration) and a
    # repeat of the same call
    inst = I.erdos_renyi_ising(4, seed=5, mean_degree=3.0)
    first = qs.enumerate_noalloc(inst.h, inst.edges, inst.J)
    second = qs.enumerate_noalloc(inst.h, inst.edges, inst.J)
    assert first == second == _allocating(qs, inst.n, inst.h, inst.edges, inst.J)


def test_noalloc_rejects_sizes_beyond_the_limit(qs):
    with pytest.raises(qs.QSError, match="outside"):
        qs.enumerate_noalloc(np.zeros(41), np.zeros((0, 2)), np.zeros(0))
    edges = np.tile([0, 1], (4097, 1))  # one more coupling than the limit
    with pytest.raises(qs.QSError, match="n_edges"):
        qs.enumerate_noalloc(np.zeros(40), edges, np.ones(len(edges)))


def test_noalloc_matches_oracle_enumeration(qs):
    for inst in (I.erdos_renyi_ising(18, seed=31, h_values=(-1, 0, 1), j_values=(-1, 0, 1)),
                 I.maxcut_regular3(16, seed=32)):
        cmin, cmax, arg, cnt, shift = qs.enumerate_noalloc(inst.h, inst.edges, inst.J)
        rc = oracle.ground(inst)
        assert shift == 0 and (cmin, cmax, arg, cnt) == (int(rc[0]), int(rc[1]), rc[2], rc[3])


@pytest.mark.parametrize("sizes", [(18, 17), (20, 20)])
def test_noalloc_beyond_the_state_range_by_factorisation(qs, sizes):
    """35 and 40 qubits: disjoint unions of two ER(4) components."""
    parts = [I.erdos_renyi_ising(m, seed=40 + k, h_values=(-1, 0, 1), j_values=(-1, 0, 1))
             for k, m in enumerate(sizes)]
    U = I.union(parts)
    assert U.n == sum(sizes)
    cmin, cmax, arg, cnt, shift = qs.enumerate_noalloc(U.h, U.edges, U.J)
    g = [oracle.ground(p) for p in parts]
    assert shift == 0
    assert cmin == int(g[0][0] + g[1][0]) and cmax == int(g[0][1] + g[1][1])
    assert arg == g[0][2] + (g[1][2] << sizes[0])
    assert cnt == g[0][3] * g[1][3]
