"""Host-side check of the sweep kernel's index arithmetic (no GPU).

tests/layout_mirror.py restates the tile shapes, the register layouts and
the address formulas of the CUDA sweep.  For every qubit count and shape they
must map (tile, thread, slot) onto the 2^n amplitudes one-to-one and in
bounds; layout 0's slot offsets (the coalesced stores) must agree with the
tile-to-global map (the TMA box and the cost evaluation); the layouts must
rotate every target exactly once; and the shared-memory swizzle must be
conflict-free in every layout.  This keeps a wrong stride from ever reaching
the GPU as an out-of-bounds access.
"""
import numpy as np
import pytest

from layout_mirror import (CFG, FAR_BIT_C64, MIN_PHYS, PAGE_BIT, PAIR_K, e_slot, e_thread, make_layout, make_shapes, pair_adj_layout, pair_layout, pair_runs_layout,
                           land, land_fwd, pair_phys, pair_unit, phys, rank_of, slot_off0, tile_base, tile_to_global)


@pytest.mark.parametrize("key", list(CFG))
def test_every_sweep_is_a_bijection(key):
    KA, KB, R, cmin = CFG[key]
    nmax = 34 if key[0] == "c64" else 30
    for n in range(1, nmax + 1):
        nphys = max(n, MIN_PHYS)
        page = PAGE_BIT[key[0]]
        shapes = make_shapes(nphys, KA, KB, cmin, page)
        assert sum(s["nt"] for s in shapes) == nphys
        # every qubit is a target of exactly one shape
        gbit = lambda tb, sh: tile_to_global(1 << tb, sh).bit_length() - 1
        owned = []
        for sh in shapes:
            owned += [gbit(tb, sh) for tb in range(sh["K"] - 1 if sh["kind"] == 0 else sh["K"])
                      if sh["kind"] == 0 or tb >= sh["c"]]
        assert sorted(owned) == list(range(nphys))
        if nphys >= 33 and key[0] == "c64":
            # the largest states spread the far bits: shape A takes the top
            # four qubits (2 KB runs), the strided shapes at most four each
            assert shapes[0]["c"] == 8 and owned[8:12] == list(range(nphys - 4, nphys))
            # the kernel takes the run-structured tile base as tile << 9
            assert all(tile_base(t, shapes[0]) == t << 9 for t in (1, 2, 3, 5, (1 << (nphys - 13)) - 1))
            assert max(sum(1 for tb in range(sh["c"], sh["K"]) if gbit(tb, sh) >= FAR_BIT_C64)
                       for sh in shapes[1:]) <= 4
        for sh in shapes:
            K, c, g0, nt = sh["K"], sh["c"], sh["g0"], sh["nt"]
            assert K - R >= 5 and K <= nphys
            if sh["kind"] == 1:
                assert 0 <= c <= K and c <= g0 and K - c == nt and 0 <= sh["n1"] <= nt
                assert sh["g1"] + nt - sh["n1"] <= nphys and (sh["n1"] == 0 or sh["g0"] + sh["n1"] <= sh["g1"])
            lays = make_layout(K, R, sh["kind"])
            ntiles = 1 << (nphys - K)
            NT, NS = 1 << (K - R), 1 << R
            offs = np.array([slot_off0(m, sh, R, lays[0]) for m in range(NS)], dtype=np.int64)
            assert all(offs[m] == tile_to_global(e_slot(m, lays[0]), sh) for m in range(NS))
            thr = np.array([tile_to_global(e_thread(t, lays[0]), sh) for t in range(NT)], dtype=np.int64)
            in_tile = (thr[:, None] + offs[None, :]).ravel()
            assert np.unique(in_tile).size == 1 << K
            if nphys <= 21:
                tiles = np.array([tile_base(t, sh) for t in range(ntiles)], dtype=np.int64)
                allidx = (tiles[:, None] + in_tile[None, :]).ravel()
                assert allidx.min() == 0 and allidx.max() == (1 << nphys) - 1
                assert np.unique(allidx).size == 1 << nphys
            else:
                tmask = 0
                for b in range(nphys - K):
                    tmask |= tile_base(1 << b, sh)
                imask = int(np.bitwise_or.reduce(in_tile))
                assert tmask & imask == 0 and (tmask | imask) == (1 << nphys) - 1
            # every target rotated exactly once per round, carried bits never
            targets = set(range(K - 1)) if sh["kind"] == 0 else set(range(c, K))
            rotated = []
            for lay in lays:
                lo, hi = lay["rot"]
                rotated += [b for b in lay["regs"] if lo <= rank_of(K, sh["kind"], b) < hi and b in targets]
            assert sorted(rotated) == sorted(targets)
            for lay in lays:
                tp = {e_thread(t, lay) for t in range(NT)}
                regs = sum(1 << b for b in lay["regs"])
                assert len(tp) == NT and all(x & regs == 0 and x < (1 << K) for x in tp)


@pytest.mark.parametrize("key", list(CFG))
def test_swizzle_is_conflict_free(key):
    """For every layout, slot and warp the lanes of each shared-memory
    wavefront (16 lanes for 8-byte elements, 8 for 16-byte ones) hit distinct
    bank groups; dense layout-0 accesses (TMA landing buffer) too."""
    KA, KB, R, _ = CFG[key]
    group = 16 if key[0] == "c64" else 8
    for K, kind in ((KA, 0), (KB, 1)):
        lays = make_layout(K, R, kind)
        for li, lay in enumerate(lays):
            for m in range(1 << R):
                for t0 in range(0, 1 << (K - R), 32):
                    for sw in (True, False) if li == 0 else (True,):
                        addrs = [(phys if sw else (lambda e, r: e))(e_thread(t0 + l, lay) | e_slot(m, lay), R)
                                 for l in range(32)]
                        for w in range(0, 32, group):
                            assert len({a % group for a in addrs[w:w + group]}) == group, (key, kind, li, m)



@pytest.mark.parametrize("C", [2, 3])
def test_pair_layouts(C):
    """Packed-pair layouts: (thread, pair, half) covers the tile once in both
    layouts; every target [C, 13) is rotated exactly once per round (the pack
    bit in layout 0); the 16-byte transposes are conflict-free per
    quarter-warp; the layout-0 store offsets reduce to one shift when the
    first target run ends below tile bit 8."""
    L = pair_layout(C)
    P = L["P"]
    assert L["tbits"][0][:C] == list(range(C))  # stores: whole 32-byte runs
    for g in range(2):
        regs, tb = L["regs"][g], L["tbits"][g]
        assert sorted(regs + tb + [P]) == list(range(PAIR_K))
        es = [sum(((j >> b) & 1) << regs[b] for b in range(5)) for j in range(32)]
        et = [sum(((t >> i) & 1) << tb[i] for i in range(7)) for t in range(128)]
        allv = {a | s | (h << P) for a in et for s in es for h in range(2)}
        assert len(allv) == 1 << PAIR_K
        for j in range(32):
            for w0 in range(0, 128, 32):
                for q in range(0, 32, 8):
                    banks = {pair_phys(pair_unit(et[w0 + q + l] | es[j], P)) % 8 for l in range(8)}
                    assert len(banks) == 8, (C, g, j, w0, q)
    rotated = [P] + [L["regs"][g][b] for g in range(2) for b in range(5) if (L["rotmask"][g] >> b) & 1]
    assert sorted(rotated) == list(range(C, PAIR_K))
    assert len({pair_phys(u) for u in range(1 << (PAIR_K - 1))}) == 1 << (PAIR_K - 1)
    for n in (24, 25, 28, 30, 32, 33, 34):
        for sh in make_shapes(n, 13, 13, 2, PAGE_BIT["c64"])[1:]:
            if sh["c"] != C:
                continue
            assert sh["K"] == PAIR_K
            if sh["c"] + sh["n1"] <= 8:
                shift = sh["g1"] + 8 - sh["c"] - sh["n1"]
                assert all(tile_to_global(j << 8, sh) == j << shift for j in range(32))


def test_pair_runs_layouts():
    """Run-structured shape A, forward packed pairs: (thread, pair, half)
    covers the tile once in both layouts; the targets [0, 12) are rotated
    once per round (pack bit and registers of layout 0, registers of layout
    1, the shuffle bit on lane bit 0 of layout 1), the batch bit 12 never;
    the 16-byte transposes are conflict-free per quarter-warp; the landing
    reads into layout 0 are 512 contiguous bytes per warp; the store offsets
    of layout 0's slots are (j & 3) << 6 plus (j >> 2) << g0."""
    L = pair_runs_layout()
    P = L["P"]
    for g in range(2):
        regs, tb = L["regs"][g], L["tbits"][g]
        assert sorted(regs + tb + [P]) == list(range(PAIR_K))
        es = [sum(((j >> b) & 1) << regs[b] for b in range(5)) for j in range(32)]
        et = [sum(((t >> i) & 1) << tb[i] for i in range(7)) for t in range(128)]
        assert len({a | s | (h << P) for a in et for s in es for h in range(2)}) == 1 << PAIR_K
        for j in range(32):
            for w0 in range(0, 128, 32):
                for q in range(0, 32, 8):
                    banks = {pair_phys(pair_unit(et[w0 + q + l] | es[j], P)) % 8 for l in range(8)}
                    assert len(banks) == 8, (g, j, w0, q)
                if g == 0:
                    units = sorted((et[w0 + l] | es[j]) >> 1 for l in range(32))
                    assert units == list(range(units[0], units[0] + 32))
    assert L["tbits"][1][0] == L["shuf"]
    rotated = [P] + L["regs"][0] + L["regs"][1] + [L["shuf"]]
    assert sorted(rotated) == list(range(12))
    for n in (33, 34):
        sh = make_shapes(n, 13, 13, 2, PAGE_BIT["c64"])[0]
        assert sh["c"] == 8 and sh["n1"] == 4 and sh["g0"] == n - 4
        for j in range(32):
            e = sum(((j >> b) & 1) << L["regs"][0][b] for b in range(5))
            assert tile_to_global(e, sh) == ((j & 3) << 6) + ((j >> 2) << sh["g0"])


@pytest.mark.parametrize("C", [1, 2, 3])
def test_pair_adjoint_layouts(C):
    """Adjoint packed-pair layouts (256 threads, 16 pairs per array): each of
    the three layouts covers the tile once, every target is rotated once per
    round, the 16-byte transposes are conflict-free per quarter-warp, and the
    two layouts a tile is stored from (0 after an even number of rounds, 2
    after an odd one) put adjacent amplitudes on the lowest lanes."""
    L = pair_adj_layout(C)
    P = L["P"]
    for g in range(3):
        regs, tb = L["regs"][g], L["tbits"][g]
        assert sorted(regs + tb + [P]) == list(range(PAIR_K))
        es = [sum(((j >> b) & 1) << regs[b] for b in range(4)) for j in range(16)]
        et = [sum(((t >> i) & 1) << tb[i] for i in range(8)) for t in range(256)]
        assert len({a | s | (h << P) for a in et for s in es for h in range(2)}) == 1 << PAIR_K
        for j in range(16):
            for w0 in range(0, 256, 32):
                for q in range(0, 32, 8):
                    banks = {pair_phys(pair_unit(et[w0 + q + l] | es[j], P)) % 8 for l in range(8)}
                    assert len(banks) == 8, (C, g, j, w0, q)
    rotated = [P] + [L["regs"][g][b] for g in range(3) for b in range(4) if (L["rotmask"][g] >> b) & 1]
    if C == 1:  # run-structured shape A: targets [0, 12), batch bit 12
        assert sorted(rotated) == list(range(PAIR_K - 1))
        # layout-0 lanes on tile bits 1..5: each store instruction covers 32
        # adjacent pairs; the 16-byte landing reads are conflict-free
        assert L["tbits"][0][:5] == [1, 2, 3, 4, 5]
        assert L["tbits"][2][:4] == [1, 2, 3, 4]
        return
    assert sorted(rotated) == list(range(C, PAIR_K))
    for g in (0, 2):  # lanes on the carried bits: whole 32-byte runs per store
        assert L["tbits"][g][:C] == list(range(C))


@pytest.mark.parametrize("C", [2, 3])
@pytest.mark.parametrize("adjoint", [False, True])
def test_pair_landing_reads_conflict_free(C, adjoint):
    """The 8-byte reads of a landed tile into the layouts it is read into
    (layout 0; the forward also layout 1, for an odd number of rounds) hit 16
    distinct bank pairs per half-warp, and the landing map keeps every
    16-byte copy whole, the tile a bijection and the copies of a
    quarter-warp on distinct 16-byte bank groups."""
    L = pair_adj_layout(C) if adjoint else pair_layout(C)
    lf = land if adjoint else land_fwd
    P = L["P"]
    assert P >= 2
    assert sorted(lf(e, P) for e in range(1 << PAIR_K)) == list(range(1 << PAIR_K))
    assert all(lf(e + 1, P) == lf(e, P) + 1 for e in range(0, 1 << PAIR_K, 2))
    for q0 in range(0, 1 << (PAIR_K - 1), 8):  # cp.async copies: element 2 q per thread
        assert len({(lf(2 * q, P) >> 1) % 8 for q in range(q0, q0 + 8)}) == 8
    for g in ((0,) if adjoint else (0, 1)):
        regs, tb = L["regs"][g], L["tbits"][g]
        nr, ntb = len(regs), len(tb)
        et = [sum(((t >> i) & 1) << tb[i] for i in range(ntb)) for t in range(1 << ntb)]
        for j in range(1 << nr):
            es = sum(((j >> b) & 1) << regs[b] for b in range(nr))
            for h in range(2):
                for w0 in range(0, 1 << ntb, 16):
                    slots = {lf(et[w0 + l] | es | (h << P), P) % 16 for l in range(16)}
                    assert len(slots) == 16, (C, adjoint, g, j, h, w0)


def test_gray_slot_walk_visits_every_slot_with_its_cost():
    """The packed-pair phase and readout walk a thread's 64 slots in four
    Gray-code chains of 16 (slot bits 4 and 5 fixed per chain), adding or
    subtracting one doubled slot term per step: every slot is visited once
    and its running value equals base - sum of 2 fb[b] over its set bits."""
    import random
    rng = random.Random(3)
    for _ in range(20):
        fb = [rng.randint(-9, 9) for _ in range(6)]
        base = rng.randint(-50, 50)
        f2 = [2 * x for x in fb]
        seen = {}
        for ch in range(4):
            run = base - (f2[4] if ch & 1 else 0) - (f2[5] if ch & 2 else 0)
            for i in range(16):
                gc = i ^ (i >> 1)
                if i > 0:
                    bb = (i & -i).bit_length() - 1
                    run += -f2[bb] if (gc >> bb) & 1 else f2[bb]
                m = (ch << 4) | gc
                seen[m] = run
        assert sorted(seen) == list(range(64))
        for m, v in seen.items():
            assert v == base - sum(f2[b] for b in range(6) if (m >> b) & 1)
