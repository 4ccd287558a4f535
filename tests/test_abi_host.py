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


def test_aqa_bad_arguments(lib):
    with pytest.raises(qs.QSError):
        qs.aqa_angles(float("nan"), [0.5])


@pytest.mark.parametrize("n", [1, 11, 12, 13, 16, 23, 24, 25, 30, 33, 34])
def test_zigzag_sweep_count(lib, n):
    """Shape A covers qubits 0..11, every further shape 11 more (2 carried low
    bits).  With S shapes the zig-zag order merges one sweep per layer
    boundary: p layers take (S - 1) p + 1 sweeps (S = 1: all layers share one
    tile, up to 8 layers per sweep)."""
    nphys = max(n, 12)
    S = 1 + (max(0, nphys - 12) + 10) // 11
    for p in (0, 1, 2, 3, 7, 20):
        s, w = qs.plan_sweeps(n, p)
        assert s == S
        if p == 0:
            assert w == 1
        elif S == 1:
            assert w == -(-p // 8)
        else:
            assert w == (S - 1) * p + 1


def _layouts(K, R):
    G = -(-K // R)
    out = []
    for g in range(G):
        lo = max(K - (g + 1) * R, 0)
        regs = list(range(lo, lo + R))
        thread = [b for b in range(K) if b not in regs]
        out.append((regs, thread))
    return out


@pytest.mark.parametrize("K,R,elem", [(12, 6, 8), (13, 6, 8), (12, 5, 8), (13, 5, 8), (11, 5, 16), (12, 5, 16)])
def test_swizzle_is_conflict_free(K, R, elem):
    """phys(e) = e ^ ((e >> S) & 31), S = max(R, 5): for every layout, slot and
    warp, the lanes of each shared-memory wavefront (16 lanes for 8-byte
    elements, 8 for 16-byte ones) hit distinct bank groups."""
    S = max(R, 5)
    phys = lambda e: e ^ ((e >> S) & 31)
    group = 128 // elem
    for regs, thread in _layouts(K, R):
        for m in range(1 << R):
            base_m = sum(((m >> i) & 1) << regs[i] for i in range(R))
            for t0 in range(0, 1 << (K - R), 32):
                addrs = []
                for lane in range(32):
                    t = t0 + lane
                    e = base_m | sum(((t >> i) & 1) << thread[i] for i in range(K - R))
                    addrs.append(phys(e))
                for w in range(0, 32, group):
                    banks = {a % group for a in addrs[w:w + group]}
                    assert len(banks) == group, (regs, m, t0)
