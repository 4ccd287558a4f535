"""Tensor-map tile loads of the strided packed-pair forward sweep, checked on
the host (no GPU): for strided complex64 shapes (c = 2, 3 carried bits, the
two target runs anywhere above them) the library's tensor-map view
(qs_pair_tile_map) covers every global index bit once, its boxes hold
exactly the tile's bits in the landing order, the coordinates of a tile and
its two box copies address exactly the tile's amplitudes at their landing
positions, the box limits of the copy engine hold (at most 256 elements per
dimension, 2^32 per tensor dimension, five dimensions), and the first read
from the landing buffer into the layout is free of shared-memory bank
conflicts (16 distinct 8-byte bank pairs per half-warp)."""
import random

import pytest

from layout_mirror import gofs, pair_layout, tile_base
from paper_2104_03293_gb300 import build, qs

PAIR_K = 13


@pytest.fixture(scope="module")
def lib():
    build.build()
    return qs.lib()


def _shapes():
    """Plan shapes of the forward sweeps plus random strided shapes."""
    out = []
    for n in range(20, 35):
        for k in range(8):
            try:
                sh = qs.plan_shapes(n)[k]
            except IndexError:
                break
            if sh["kind"] == 1 and sh["c"] in (2, 3):
                out.append((n, sh["c"], sh["g0"], sh["n1"], sh["g1"]))
    rng = random.Random(7)
    while len(out) < 160:
        n = rng.randint(20, 34)
        c = rng.choice((2, 3))
        nt = PAIR_K - c
        n1 = rng.randint(0, nt)
        n2 = nt - n1
        # runs [g0, g0 + n1), [g1, g1 + n2) above c, disjoint, either order
        free = n - c - nt
        gaps = sorted(rng.randint(0, free) for _ in range(2))
        if rng.random() < 0.5:
            g0 = c + gaps[0]
            g1 = g0 + n1 + (gaps[1] - gaps[0])
        else:
            g1 = c + gaps[0]
            g0 = g1 + n2 + (gaps[1] - gaps[0])
        if n1 == 0:
            g0 = g1
        out.append((n, c, g0, n1, g1))
    return out


@pytest.mark.parametrize("g", [0, 1])
def test_pair_tile_maps(lib, g):
    fits = 0
    for n, c, g0, n1, g1 in _shapes():
        m = qs.pair_tile_map(n, c, g0, n1, g1, g)
        if m is None:
            continue
        fits += 1
        sh = dict(K=PAIR_K, c=c, g0=g0, n1=n1, g1=g1, kind=1)
        tglob = [gofs(1 << tb, sh).bit_length() - 1 for tb in range(PAIR_K)]
        r, st, wd, bx, land = m["rank"], m["start"], m["width"], m["box"], m["landing"]
        assert 1 <= r <= 5 and st[0] == 0
        # every global bit in exactly one dimension
        cover = sorted(b for d in range(r) for b in range(st[d], st[d] + wd[d]))
        assert cover == list(range(n)), (n, c, g0, n1, g1)
        # box bits, in dimension order, are the tile bits in landing order
        boxbits = [b for d in range(r) for b in range(st[d], st[d] + bx[d])]
        assert sorted(land) == list(range(PAIR_K)) and land[c] == PAIR_K - 1
        by_pos = sorted(range(PAIR_K), key=lambda tb: land[tb])
        assert boxbits == [tglob[tb] for tb in by_pos[:PAIR_K - 1]]
        assert m["kbit"] == tglob[c]
        # copy-engine limits: 256 elements per box dimension (dimension 0 in
        # floats), 2^32 per tensor dimension
        assert (1 << (bx[0] + 1)) <= 256 and all((1 << bx[d]) <= 256 for d in range(1, r))
        assert (1 << (wd[0] + 1)) <= 1 << 32 and all(wd[d] <= 32 for d in range(1, r))
        # a tile's two box copies address exactly its amplitudes, each at its
        # landing position
        rng = random.Random(n * 131 + g0)
        for t in (0, (1 << (n - PAIR_K)) - 1, rng.randrange(1 << (n - PAIR_K))):
            base = tile_base(t, sh)
            want = {base | gofs(e, sh): sum(((e >> tb) & 1) << land[tb] for tb in range(PAIR_K))
                    for e in range(1 << PAIR_K)}
            got = {}
            for k in range(2):
                bk = base | (k << m["kbit"])
                coord = [(bk >> st[d]) & ((1 << wd[d]) - 1) for d in range(r)]
                assert coord[0] * 8 % 16 == 0  # innermost coordinate x element size: 16-byte aligned
                for i in range(1 << (PAIR_K - 1)):
                    gi, rem = 0, i
                    for d in range(r):
                        idx = coord[d] + (rem & ((1 << bx[d]) - 1))
                        rem >>= bx[d]
                        assert idx < 1 << wd[d]
                        gi |= idx << st[d]
                    got[gi] = i | (k << (PAIR_K - 1))
            assert got == want, (n, c, g0, n1, g1, t)
        # first read into layout g: half-warps hit 16 distinct bank pairs
        L = pair_layout(c)
        regs, tb = L["regs"][g], L["tbits"][g]
        for j in range(32):
            for half in range(2):
                es = sum(((j >> b) & 1) << regs[b] for b in range(5)) | (half << c)
                for h0 in range(0, 128, 16):
                    pairs = set()
                    for l in range(16):
                        e = es | sum((((h0 + l) >> i) & 1) << tb[i] for i in range(7))
                        pairs.add(sum(((e >> q) & 1) << land[q] for q in range(PAIR_K)) % 16)
                    assert len(pairs) == 16, (c, g, j, h0)
    assert fits >= 60


def test_plan_shapes_fit_a_box(lib):
    """Every strided c = 2, 3 shape of the plans for 20-34 qubits fits the
    tensor-map view for both first-read layouts."""
    for n in range(20, 35):
        for sh in qs.plan_shapes(n):
            if sh["kind"] == 1 and sh["c"] in (2, 3):
                for g in (0, 1):
                    assert qs.pair_tile_map(n, sh["c"], sh["g0"], sh["n1"], sh["g1"], g) is not None, (n, sh, g)
