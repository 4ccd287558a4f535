"""Seeded input generators: determinism and the structure each workload names."""
import json
import os

import numpy as np

from paper_2104_03293_gb300 import instances as I


def test_regular3_is_simple_and_cubic():
    for n, seed in [(12, 1), (26, 2), (34, 3)]:
        inst = I.maxcut_regular3(n, seed)
        deg = np.bincount(inst.edges.ravel(), minlength=n)
        assert np.all(deg == 3)
        assert np.all(inst.edges[:, 0] < inst.edges[:, 1])
        assert len({tuple(e) for e in inst.edges.tolist()}) == inst.m == 3 * n // 2
        assert np.all(inst.J == 1) and np.all(inst.h == 0)


def test_er_weights_and_determinism():
    a = I.erdos_renyi_ising(24, 5)
    b = I.erdos_renyi_ising(24, 5)
    assert np.array_equal(a.edges, b.edges) and np.array_equal(a.J, b.J) and np.array_equal(a.h, b.h)
    assert set(np.unique(a.J)) <= {-2, -1, 1, 2}
    assert set(np.unique(a.h)) <= {-2, -1, 0, 1, 2}
    big = I.erdos_renyi_ising(34, 7, h_values=(-1, 0, 1), j_values=(-1, 0, 1))
    assert 34 <= big.m <= 110  # mean degree 4 -> ~68 edges


def test_union_blocks_are_contiguous():
    u = I.union([I.maxcut_regular3(6, 1), I.erdos_renyi_ising(5, 2)])
    assert u.n == 11 and u.components == [range(0, 6), range(6, 11)]
    for a, b in u.edges:
        assert (a < 6) == (b < 6)


def test_workloads_shapes():
    c2 = I.config2(count=40)
    assert all(16 <= inst.n <= 24 and 1 <= len(g) <= 10 for inst, g, b in c2)
    c4 = I.config4(count=9)
    assert [t for _, _, t in c4[:3]] == [0.5, 0.75, 1.0]
    inst, s, tau = I.config5()
    assert inst.n == 34 and s.size == 20 and tau == 0.75


def test_golden_config1_matches_generator():
    path = os.path.join(os.path.dirname(__file__), "golden", "config1_maxcut3r_n12_p2.json")
    rec = json.load(open(path))
    inst, g, b = I.config1()
    assert rec["edges"] == inst.edges.tolist()
    assert np.array_equal(np.array(rec["gamma"]), g) and np.array_equal(np.array(rec["beta"]), b)
