"""Host-side check of the sweep kernel's index arithmetic (no GPU).

The functions below restate, line for line, the address formulas of the
sweep kernel (tile_base, gofs, SlotMap, the register layouts) and the planner's
tile shapes.  For every qubit count and tile shape they must map
(tile, thread, slot) onto the 2^n amplitudes one-to-one and in bounds, and
the layout-0 slot offsets must agree with the tile-to-global map used by the
cost evaluation.  This is the check that keeps a wrong stride from ever
reaching the GPU as an out-of-bounds access.
"""
import numpy as np
import pytest

CFG = {("c64", False): (12, 13, 6, 2), ("c64", True): (12, 13, 5, 2),
       ("c128", False): (11, 12, 5, 2), ("c128", True): (11, 12, 4, 2)}


def make_shapes(nphys, KA, KB, R, cmin):
    shapes = [(KA, 0, 0, KA)]
    g = KA
    while g < nphys:
        nt = min(KB - cmin, nphys - g)
        shapes.append((KB, KB - nt, g, nt))
        g += nt
    return shapes


def gofs(e, c, g0):
    return (e & ((1 << c) - 1)) | ((e >> c) << g0)


def tile_base(t, c, g0, K):
    mid = g0 - c
    midm = (1 << mid) - 1 if mid > 0 else 0
    return ((t & midm) << c) | ((t >> mid) << (g0 + K - c))


def slot_off(m, K, R, c, g0):
    lo = K - R
    cs = c - lo if c > lo else 0
    sh = g0 if cs else g0 + lo - c
    if cs == 0:
        return m << sh
    return ((m & ((1 << cs) - 1)) << lo) | ((m >> cs) << sh)


def e_thread(tid, lo, R):
    return (tid & ((1 << lo) - 1)) | ((tid >> lo) << (lo + R))


def layouts(K, R):
    G = -(-K // R)
    return [max(K - (g + 1) * R, 0) for g in range(G)]


@pytest.mark.parametrize("key", list(CFG))
def test_every_sweep_is_a_bijection(key):
    KA, KB, R, cmin = CFG[key]
    nmax = 34 if key[0] == "c64" else 30
    for n in range(1, nmax + 1):
        nphys = max(n, 12)
        shapes = make_shapes(nphys, KA, KB, R, cmin)
        covered = 0
        for K, c, g0, nt in shapes:
            assert 0 <= c <= K and c <= g0 and g0 + nt <= nphys and K - c == nt
            assert K - R >= 5
            covered += nt
            ntiles = 1 << (nphys - K)
            NT, NS = 1 << (K - R), 1 << R
            offs = np.array([slot_off(m, K, R, c, g0) for m in range(NS)], dtype=np.int64)
            # layout 0 slot offsets == tile-to-global map of the register tile bits
            assert all(offs[m] == gofs(m << (K - R), c, g0) for m in range(NS))
            thr = np.array([gofs(t, c, g0) for t in range(NT)], dtype=np.int64)
            in_tile = (thr[:, None] + offs[None, :]).ravel()
            if nphys <= 22:
                tiles = np.array([tile_base(t, c, g0, K) for t in range(ntiles)], dtype=np.int64)
                allidx = (tiles[:, None] + in_tile[None, :]).ravel()
                assert allidx.min() == 0 and allidx.max() == (1 << nphys) - 1
                assert np.unique(allidx).size == 1 << nphys
            else:
                # in-tile offsets and tile bases occupy disjoint bits
                tmask = 0
                for t in range(ntiles.bit_length()):
                    tmask |= tile_base(1 << t, c, g0, K) if (1 << t) < ntiles else 0
                imask = int(np.bitwise_or.reduce(in_tile))
                assert tmask & imask == 0 and (tmask | imask) == (1 << nphys) - 1
                assert np.unique(in_tile).size == 1 << K
            # every layout: thread part and slot part are disjoint tile bits
            for lo in layouts(K, R):
                regs = sum(1 << (lo + b) for b in range(R))
                tparts = {e_thread(t, lo, R) for t in range(NT)}
                assert all(tp & regs == 0 and tp < (1 << K) for tp in tparts) and len(tparts) == NT
        assert covered == nphys
