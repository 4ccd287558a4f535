"""Python restatement of the tile shapes, register layouts and index maps of
the CUDA sweep (qs_layout.h, make_shapes, the kernel's address formulas), for
host-side checks of the index arithmetic."""

CFG = {("c64", False): (13, 13, 6, 2), ("c64", True): (13, 13, 5, 2),
       ("c128", False): (12, 12, 5, 2), ("c128", True): (12, 12, 4, 2)}
MIN_PHYS = 13


def ranked_bit(K, kind, i):
    if kind == 0:
        return K - 2 - i if i < K - 1 else K - 1
    return K - 1 - i


def rank_of(K, kind, b):
    if kind == 0:
        return K - 1 if b == K - 1 else K - 2 - b
    return K - 1 - b


def make_layout(K, R, kind):
    ntg = K - 1 if kind == 0 else K
    G = -(-ntg // R)
    out = []
    for g in range(G):
        if g * R + R <= ntg:
            regs = sorted(ranked_bit(K, kind, i) for i in range(g * R, g * R + R))
        else:
            regs = list(range(R))
        tbits = [b for b in range(K) if b not in regs]
        out.append({"regs": regs, "tbits": tbits, "rot": (g * R, min((g + 1) * R, ntg))})
    return out


PAGE_BIT = {"c64": 18, "c128": 17}


FAR_BIT_C64 = 22


def make_shapes(nphys, KA, KB, cmin, page_bit=18):
    a = dict(K=KA, c=0, g0=0, nt=KA - 1, kind=0, n1=0, g1=0)
    lo, hi, split = KA - 1, nphys, page_bit
    if KA == 13 and KB == 13 and nphys >= 33:
        f = 4
        a.update(c=KA - 1 - f, g0=nphys - f, n1=f, g1=KA - 1 - f)
        lo, hi, split = a["c"], nphys - f, FAR_BIT_C64
    shapes = [a]
    per = KB - cmin
    rest = hi - lo
    if rest <= 0:
        return shapes
    S = -(-rest // per)
    below = max(0, min(split, hi) - lo)
    high = rest - below
    nt = [min(per, rest - k * per) for k in range(S)]
    nh = [0] * S
    for _ in range(high):
        best = min((k for k in range(S) if nh[k] < nt[k]), key=lambda k: (nh[k], k))
        nh[best] += 1
    lo_next, hi_next = lo, lo + below
    for k in range(S):
        n1 = nt[k] - nh[k]
        g0 = lo_next
        lo_next += n1
        g1 = hi_next if nh[k] else g0 + n1
        hi_next += nh[k]
        if n1 == 0:
            g0 = g1
        if g0 + n1 == g1:
            n1, g1 = 0, g0
        shapes.append(dict(K=KB, c=KB - nt[k], g0=g0, nt=nt[k], kind=1, n1=n1, g1=g1))
    return shapes


def contiguous(sh):
    return sh["kind"] == 0 and sh["c"] == 0 and sh["n1"] == 0


def gofs(e, sh):
    c, g0, n1, g1 = sh["c"], sh["g0"], sh["n1"], sh["g1"]
    return (e & ((1 << c) - 1)) | (((e >> c) & ((1 << n1) - 1)) << g0) | ((e >> (c + n1)) << g1)


def tile_base(t, sh):
    """Non-tile global bits, ascending, take the bits of the tile index t."""
    K, c, g0, n1, g1 = sh["K"], sh["c"], sh["g0"], sh["n1"], sh["g1"]
    if contiguous(sh):
        return t << K
    runs = sorted((g, l) for g, l in ((g0, n1), (g1, K - c - n1)) if l > 0)
    out, pos, bit = 0, c, 0
    for g, l in runs + [(200, 0)]:
        for q in range(pos, g):
            if (t >> bit) == 0:
                return out
            out |= ((t >> bit) & 1) << q
            bit += 1
        pos = g + l
    return out


def tile_to_global(e, sh):
    return e if contiguous(sh) else gofs(e, sh)


def slot_off0(m, sh, R, lay0):
    """Global offset of register slot m in layout 0 (the kernel's for_slots)."""
    K = sh["K"]
    if sh["kind"] == 0:
        if contiguous(sh):
            return sum(((m >> b) & 1) << lay0["regs"][b] for b in range(R))
        lo = K - 1 - R  # registers: tile bits [lo, K - 1); below c in place, the rest on run 1
        cl = sh["c"] - lo
        assert cl >= 0 and sh["n1"] >= K - 1 - sh["c"]
        return ((m & ((1 << cl) - 1)) << lo) | ((m >> cl) << sh["g0"])
    lo = K - R
    if sh["c"] + sh["n1"] <= lo:
        return m << (sh["g1"] + lo - sh["c"] - sh["n1"])
    return gofs(m << lo, sh)


def e_thread(t, lay):
    return sum(((t >> j) & 1) << b for j, b in enumerate(lay["tbits"]))


def e_slot(m, lay):
    return sum(((m >> j) & 1) << b for j, b in enumerate(lay["regs"]))


def phys(e, R):
    return e ^ ((e >> R) & 31)


# Packed-pair layouts (qs_pair.h): strided complex64 tiles with c = 2 or 3.
PAIR_K = 13


def pair_layout(C):
    regs0 = [8, 9, 10, 11, 12]
    if C == 2:
        return dict(P=2, regs=[regs0, [3, 4, 5, 6, 7]], tbits=[[0, 1, 3, 4, 5, 6, 7], [0, 1, 9, 8, 10, 11, 12]],
                    rotmask=[0x1f, 0x1f])
    return dict(P=3, regs=[regs0, [4, 5, 6, 7, 12]], tbits=[[0, 1, 2, 4, 5, 6, 7], [0, 1, 2, 8, 9, 10, 11]],
                rotmask=[0x1f, 0x0f])


def pair_unit(e, P):
    return (e & ((1 << P) - 1)) | ((e >> (P + 1)) << P)


def pair_phys(u):
    return u ^ ((u >> 3) & 7) ^ ((u >> 6) & 7) ^ ((u >> 9) & 7)


def pair_adj_layout(C):
    if C == 1:  # run-structured shape A: pack bit = tile bit 0
        return dict(P=0, regs=[[8, 9, 10, 11], [1, 2, 3, 4], [5, 6, 7, 12]],
                    tbits=[[1, 2, 3, 4, 5, 6, 7, 12], [5, 6, 7, 8, 9, 10, 11, 12], [1, 2, 3, 4, 8, 9, 10, 11]],
                    rotmask=[0xf, 0xf, 0x7])
    if C == 2:
        return dict(P=2, regs=[[9, 10, 11, 12], [3, 4, 5, 6], [7, 8, 11, 12]],
                    tbits=[[0, 1, 3, 4, 5, 6, 7, 8], [0, 1, 9, 7, 8, 10, 11, 12], [0, 1, 3, 4, 5, 6, 9, 10]],
                    rotmask=[0xf, 0xf, 0x3])
    return dict(P=3, regs=[[9, 10, 11, 12], [4, 5, 6, 7], [8, 10, 11, 12]],
                tbits=[[0, 1, 2, 4, 5, 6, 7, 8], [0, 1, 2, 8, 9, 10, 11, 12], [0, 1, 2, 4, 5, 6, 7, 9]],
                rotmask=[0xf, 0xf, 0x1])


def pair_runs_layout():
    """Forward layouts of the run-structured shape A (pack bit = tile bit 0;
    tile bit 11 on lane bit 0 of layout 1, rotated by shuffles)."""
    return dict(P=0, regs=[[6, 7, 8, 9, 10], [1, 2, 3, 4, 5]],
                tbits=[[1, 2, 3, 4, 5, 11, 12], [11, 6, 7, 8, 9, 10, 12]], shuf=11)


def land(e, P):
    """Landing-buffer position of tile element e (packed-pair adjoint)."""
    return e if P == 0 else e ^ (((e >> 4) & 1) << P)


def land_fwd(e, P):
    """Landing-buffer position of tile element e (packed-pair forward: read
    into layout 0 or layout 1)."""
    f = ((e >> 4) ^ (e >> 8)) & 1
    return e ^ (f << 2) ^ (((e >> 9) & 1) << 3) if P == 2 else e ^ (f << P)
