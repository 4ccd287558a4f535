"""C ABI checks that need no GPU: the library builds, loads and exports every
function declared in include/qs.h; the host-only helpers (AQA angle maps,
chain rule, sweep planner) agree with the oracle's restatement or with the
schedule's closed-form sweep count; the shared-memory swizzle is
conflict-free for every register layout the kernels use."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2104_03293_gb300 import build, qs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return qs.lib()


def test_every_header_function_is_exported(lib):
    names = qs.header_functions()
    assert len(names) >= 25
    raw = ctypes.CDLL(build.LIB)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    assert set(names) == set(qs._SIGS), set(names) ^ set(qs._SIGS)


def test_version_and_error_text(lib):
    assert "sm_103a" in qs.version()
    h = ctypes.c_void_p()
    # argument validation happens before any CUDA call
    rc = lib.qs_create(ctypes.byref(h), 0, qs.QS_C64, None, None, 0)
    assert rc == qs.QS_EINVAL and b"n = 0" in lib.qs_last_error()
    rc = lib.qs_create(ctypes.byref(h), 35, qs.QS_C64, None, None, 0)
    assert rc == qs.QS_EINVAL
    rc = lib.qs_create(ctypes.byref(h), 31, qs.QS_C128, None, None, 0)
    assert rc == qs.QS_EINVAL
    rc = lib.qs_create(ctypes.byref(h), 10, 7, None, None, 0)
    assert rc == qs.QS_EINVAL
    rc = lib.qs_create(ctypes.byref(h), 10, qs.QS_C64, None, ctypes.c_void_p(0x1004), 1 << 20)
    assert rc == qs.QS_EINVAL and b"aligned" in lib.qs_last_error()
    assert lib.qs_destroy(None) == qs.QS_OK


@pytest.mark.parametrize("p", [1, 5, 20])
def test_aqa_angles_match_oracle(lib, p):
    s = np.arange(1, p + 1) / (p + 1)
    for tau in (0.5, 0.75, 1.0):
        g, b = qs.aqa_angles(tau, s)
        go, bo = oracle.aqa_angles(tau, s)
        assert np.array_equal(g, go) and np.array_equal(b, bo)
        if p > 1:
            s2 = np.arange(p) / (p - 1)
            g2, b2 = qs.aqa_angles_2nd(tau, s2)
            go2, bo2 = oracle.aqa_angles_second_order(tau, s2)
            assert np.allclose(g2, go2, rtol=0, atol=1e-15) and np.allclose(b2, bo2, rtol=0, atol=1e-15)
        rng = np.random.default_rng(p)
        dg, db = rng.normal(size=p), rng.normal(size=p)
        dt, ds = qs.aqa_chain(tau, s, dg, db)
        dto, dso = oracle.aqa_chain(tau, s, dg, db)
        assert abs(dt - dto) <= 1e-12 and np.allclose(ds, dso, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 7, 20])
def test_aqa_chain_2nd_matches_oracle(lib, p):
    """The library's chain rule for the second-order map against the
    oracle's term-by-term restatement (pinned by finite differences)."""
    rng = np.random.default_rng(100 + p)
    s = np.sort(rng.uniform(0, 1, size=p))
    for tau in (0.4, 0.8):
        dg, db = rng.normal(size=p), rng.normal(size=p)
        dt, ds = qs.aqa_chain_2nd(tau, s, dg, db)
        dto, dso = oracle.aqa_chain_second_order(tau, s, dg, db)
        assert abs(dt - dto) <= 1e-12 and np.allclose(ds, dso, rtol=0, atol=1e-12)
    with pytest.raises(qs.QSError):
        qs.aqa_chain_2nd(0.5, [], [], [])


def test_aqa_bad_arguments(lib):
    with pytest.raises(qs.QSError):
        qs.aqa_angles(float("nan"), [0.5])


@pytest.mark.parametrize("n", [1, 11, 12, 13, 16, 23, 24, 25, 30, 33, 34])
def test_zigzag_sweep_count(lib, n):
    """Shape A covers qubits 0..11, every further shape 11 more (2 carried low
    bits); states are stored with at least 13 qubits.  With S shapes the
    zig-zag order merges one sweep per layer boundary: p layers take
    (S - 1) p + 1 sweeps."""
    nphys = max(n, 13)
    S = 1 + (nphys - 12 + 10) // 11
    for p in (0, 1, 2, 3, 7, 20):
        s, w = qs.plan_sweeps(n, p)
        assert s == S
        assert w == (1 if p == 0 else (S - 1) * p + 1)


@pytest.mark.parametrize("dtype", [0, 1])
def test_planner_matches_host_mirror(lib, dtype):
    """The library's tile shapes are exactly those the index-math checks use."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from layout_mirror import CFG, PAGE_BIT, make_shapes
    key = ("c64" if dtype == 0 else "c128", False)
    KA, KB, R, cmin = CFG[key]
    for n in range(1, 35 if dtype == 0 else 31):
        got = qs.plan_shapes(n, dtype)
        want = make_shapes(max(n, 13), KA, KB, cmin, PAGE_BIT[key[0]])
        assert [(s["kind"], s["K"], s["c"]) for s in got] == [(s["kind"], s["K"], s["c"]) for s in want], n
        for g, w in zip(got, want):
            if w["kind"] == 1:
                assert (g["g0"], g["n1"], g["g1"]) == (w["g0"], w["n1"], w["g1"]), (n, g, w)


def test_grid_scan_rejects_an_empty_grid_before_any_device_call(lib):
    with pytest.raises(qs.QSError):
        qs.grid_scan(np.zeros(3), np.zeros((0, 2), dtype=np.int32), np.zeros(0), [], [0.1])
    with pytest.raises(qs.QSError):
        qs.grid_scan(np.zeros(3), np.zeros((0, 2), dtype=np.int32), np.zeros(0), [0.2], np.zeros(0))


def test_binding_checks_the_lengths_the_c_side_reads(lib):
    """The binding rejects arrays shorter than what the C entry points read
    (h of n entries, one J per edge, matching angle lists) before calling."""
    h, e, J = qs._ising_arrays(3, [0.5, 0, -1], [[0, 1], [1, 2]], [1.0, -1.0])
    assert h.shape == (3,) and e.shape == (2, 2) and e.dtype == np.int32 and J.shape == (2,)
    with pytest.raises(ValueError):
        qs._ising_arrays(4, [0.5, 0, -1], [[0, 1]], [1.0])
    with pytest.raises(ValueError):
        qs._ising_arrays(3, [0.5, 0, -1], [[0, 1], [1, 2]], [1.0])
    with pytest.raises(ValueError):
        qs.enumerate_noalloc([0.0, 1.0], [[0, 1]], [])
    with pytest.raises(ValueError):
        qs._angles([0.1, 0.2], [0.3])
    with pytest.raises(ValueError):
        qs._angles([[0.1]], [[0.3]])
    g, b = qs._angles(0.1, 0.3)  # a scalar is one layer
    assert g.shape == b.shape == (1,)
    with pytest.raises(ValueError):
        qs.State(4, dtype="c32")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qsds_layers_reproduce_the_product_formula(lib, seed):
    """qs_qsds_layers: applying its layers with the oracle's own gates (the
    phase exp(-i gamma H_C) with the fields, then each qubit's 2 x 2 matrix)
    gives the oracle's step-by-step Eq. (AQA4) state; every matrix is
    unitary; the layer count is nsteps + 1."""
    from paper_2104_03293_gb300 import instances as I
    inst = I.erdos_renyi_ising(7, 40 + seed)
    nsteps, tau = 6, 0.5
    s = (np.arange(nsteps) + 0.5) / nsteps
    A, B = 1.0 - s, s
    g, u = qs.qsds_layers(inst.n, tau, A, B, inst.h)
    assert g.shape == (nsteps + 1,) and u.shape == (nsteps + 1, inst.n, 2, 2)
    for m in u.reshape(-1, 2, 2):
        assert np.max(np.abs(m.conj().T @ m - np.eye(2))) <= 1e-14
    psi = oracle.evolve(inst, [0.0], [0.0])  # |+>^n
    for k in range(nsteps + 1):
        psi = oracle.evolve(inst, [g[k]], [0.0], psi=psi)
        for q in range(inst.n):
            oracle.gate_u(inst.n, psi, q, u[k, q])
    want = oracle.qsds_evolve(inst, tau, A, B)
    assert np.max(np.abs(psi - want)) <= 1e-12
    with pytest.raises(qs.QSError):
        qs.qsds_layers(0, tau, A, B, inst.h[:0])
