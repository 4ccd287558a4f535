// Register layouts of the packed-pair sweep: strided complex64 tiles (kind 1,
// K = 13 tile bits, c = 2 or 3 carried low bits), forward rotations and phase.
//
// A thread holds 64 amplitudes as 32 pairs.  The two amplitudes of a pair
// differ in the pack bit P = c (the lowest target bit) and are stored split
// by component, X = (re_a, re_b) and Y = (im_a, im_b), so one packed f32x2
// FMA updates both: a butterfly on any other register bit costs four f32x2
// FMAs per four amplitudes instead of eight scalar FMAs.  The rotation of the
// pack bit itself mixes the two halves of a pair and is done with scalar FMAs.
//
// Layout g puts the pack bit and the five tile bits regs[g][0..4] into the
// registers (pair index j: bit b <-> regs[g][b]) and the seven tbits[g] into
// the thread index (tbits[g][0..4] are the lane bits).  Layout 0 holds the
// five top tile bits, so its stores are coalesced over the carried bits;
// layout 1 holds the remaining targets.  Both layouts hold the pack bit, which
// layout 0 rotates.  The shared-memory transposes move 16-byte pairs (X, Y);
// the pair unit u is the tile index with the pack bit removed, placed at
// phys(u) = u ^ fold3(u), where fold3 XORs the 3-bit groups of u above the
// lowest into it.  The lane order puts on lanes 0..2 three thread bits whose
// u positions differ mod 3, so every quarter-warp of 16-byte accesses hits
// eight distinct bank groups (checked on the host by the test-suite).
#pragma once

#ifdef __CUDACC__
#define QS_PHD __host__ __device__
#else
#define QS_PHD
#endif

namespace qs {

constexpr int kPairK = 13;

struct PairLayout {
    int C, P;
    int regs[2][5];   // tile bit of pair-index bit b (ascending)
    int tbits[2][7];  // tile bit of thread-index bit t (lane order)
    int rotmask[2];   // bit b: regs[g][b] is a target rotated in layout g
};

QS_PHD constexpr bool pair_c_ok(int c) { return c == 2 || c == 3; }

QS_PHD constexpr PairLayout pair_layout(int C) {
    PairLayout t{};
    t.C = C;
    t.P = C;
    for (int b = 0; b < 5; ++b) t.regs[0][b] = 8 + b;  // top five tile bits
    if (C == 2) {
        const int r1[5] = {3, 4, 5, 6, 7};
        const int t0[7] = {0, 1, 3, 4, 5, 6, 7};
        const int t1[7] = {0, 1, 9, 8, 10, 11, 12};
        for (int b = 0; b < 5; ++b) t.regs[1][b] = r1[b];
        for (int i = 0; i < 7; ++i) {
            t.tbits[0][i] = t0[i];
            t.tbits[1][i] = t1[i];
        }
        t.rotmask[0] = 0x1f;
        t.rotmask[1] = 0x1f;
    } else {
        // C = 3: targets 3..12; layout 1 rotates 4..7 and holds bit 12 idle
        const int r1[5] = {4, 5, 6, 7, 12};
        const int t0[7] = {0, 1, 2, 4, 5, 6, 7};
        const int t1[7] = {0, 1, 2, 8, 9, 10, 11};
        for (int b = 0; b < 5; ++b) t.regs[1][b] = r1[b];
        for (int i = 0; i < 7; ++i) {
            t.tbits[0][i] = t0[i];
            t.tbits[1][i] = t1[i];
        }
        t.rotmask[0] = 0x1f;
        t.rotmask[1] = 0x0f;
    }
    return t;
}

// Adjoint layouts (two arrays, 32 amplitudes = 16 pairs per array and
// thread, 256 threads): the pack bit plus four register bits per layout and
// three layouts.  Layout 0 holds the four top target bits, so its stores
// are coalesced over the low tile bits.  C = 2, 3: strided tiles with C
// carried bits; C = 1: the run-structured shape A.
struct PairAdjLayout {
    int C, P;
    int regs[3][4];   // tile bit of pair-index bit b (ascending)
    int tbits[3][8];  // tile bit of thread-index bit t (lane order)
    int rotmask[3];   // bit b: regs[g][b] is rotated in layout g
};

QS_PHD constexpr PairAdjLayout pair_adj_layout(int C) {
    PairAdjLayout t{};
    t.C = C;
    t.P = C;
    if (C == 1) {
        // run-structured shape A (targets tile bits [0, 12), batch bit 12):
        // the pack bit is tile bit 0, so a pair is two adjacent amplitudes
        t.P = 0;
        const int r[3][4] = {{8, 9, 10, 11}, {1, 2, 3, 4}, {5, 6, 7, 12}};
        const int tt[3][8] = {{1, 2, 3, 4, 5, 6, 7, 12}, {5, 6, 7, 8, 9, 10, 11, 12}, {1, 2, 3, 4, 8, 9, 10, 11}};
        for (int g = 0; g < 3; ++g) {
            for (int b = 0; b < 4; ++b) t.regs[g][b] = r[g][b];
            for (int i = 0; i < 8; ++i) t.tbits[g][i] = tt[g][i];
        }
        t.rotmask[0] = 0xf;
        t.rotmask[1] = 0xf;
        t.rotmask[2] = 0x7;  // bits 5, 6, 7; bit 12 is the batch bit
        return t;
    }
    const int r0[4] = {9, 10, 11, 12};
    const int r1c2[4] = {3, 4, 5, 6}, r2c2[4] = {7, 8, 11, 12};
    const int t0c2[8] = {0, 1, 3, 4, 5, 6, 7, 8}, t1c2[8] = {0, 1, 9, 7, 8, 10, 11, 12}, t2c2[8] = {0, 1, 3, 4, 5, 6, 9, 10};
    const int r1c3[4] = {4, 5, 6, 7}, r2c3[4] = {8, 10, 11, 12};
    const int t0c3[8] = {0, 1, 2, 4, 5, 6, 7, 8}, t1c3[8] = {0, 1, 2, 8, 9, 10, 11, 12}, t2c3[8] = {0, 1, 2, 4, 5, 6, 7, 9};
    for (int b = 0; b < 4; ++b) {
        t.regs[0][b] = r0[b];
        t.regs[1][b] = C == 2 ? r1c2[b] : r1c3[b];
        t.regs[2][b] = C == 2 ? r2c2[b] : r2c3[b];
    }
    for (int i = 0; i < 8; ++i) {
        t.tbits[0][i] = C == 2 ? t0c2[i] : t0c3[i];
        t.tbits[1][i] = C == 2 ? t1c2[i] : t1c3[i];
        t.tbits[2][i] = C == 2 ? t2c2[i] : t2c3[i];
    }
    t.rotmask[0] = 0xf;
    t.rotmask[1] = 0xf;
    t.rotmask[2] = C == 2 ? 0x3 : 0x1;  // C = 2: bits 7, 8; C = 3: bit 8
    return t;
}

// Forward layouts of the run-structured shape A (kind 0 with runs: tile bits
// [0, 8) one 2 KB run, [8, 12) the top four qubits, 12 the batch bit; targets
// [0, 12)).  The pack bit is tile bit 0 (a pair is two adjacent amplitudes,
// one 16-byte unit).  Layout 0 holds five run bits in the registers and puts
// run bits 1..5 on the lanes, so its stores are 512 contiguous bytes per warp;
// layout 1 holds run bits 1..5 and has tile bit 11 on lane bit 0, rotated by
// lane shuffles (two layouts of five bits plus the pack bit hold eleven of the
// twelve targets).
struct PairRunsLayout {
    int regs[2][5];
    int tbits[2][7];
    int shuf;  // tile bit on lane bit 0 of layout 1, rotated by shuffles
};

QS_PHD constexpr PairRunsLayout pair_runs_layout() {
    PairRunsLayout t{};
    const int r0[5] = {6, 7, 8, 9, 10}, t0[7] = {1, 2, 3, 4, 5, 11, 12};
    const int r1[5] = {1, 2, 3, 4, 5}, t1[7] = {11, 6, 7, 8, 9, 10, 12};
    for (int b = 0; b < 5; ++b) {
        t.regs[0][b] = r0[b];
        t.regs[1][b] = r1[b];
    }
    for (int i = 0; i < 7; ++i) {
        t.tbits[0][i] = t0[i];
        t.tbits[1][i] = t1[i];
    }
    t.shuf = 11;
    return t;
}

// Landing order of a strided tile loaded by tensor-map copies (the TMA
// variant of the packed-pair forward sweep), for a tile first read into
// layout g.  pos[tb] is the shared-memory position bit (in 8-byte
// amplitudes) of tile bit tb; the pack bit sits on position 12, so the tile
// arrives as two box copies of 2^12 amplitudes, one per value of the pack
// bit.  A box lays its dimensions out in the order of their position bits,
// and each dimension is a run of consecutive global bits, so the host
// derives the tensor map from this table and the tile's shape.  Positions
// 0-3 hold the four lane bits of a half-warp of layout g (tile bits 0, 1
// and, for C = 2, 3, 4 in layout 0 or 8, 9 in layout 1; for C = 3, bit 2
// and 4 or 8), so the 8-byte reads into layout g hit 16 distinct bank pairs
// without a swizzle (checked on the host by the test-suite).  The copies are
// unswizzled: a swizzle span above the 32- or 64-byte box rows would space
// the rows out to the span.
struct PairTmaPos {
    int pos[13];
};

QS_PHD constexpr PairTmaPos pair_tma_pos(int C, int g) {
    PairTmaPos t{};
    // landing order: the carried bits, then the half-warp's other lane
    // bits with the run they start, then the remaining tile bits in order
    int order[12] = {};
    int k = 0;
    for (int b = 0; b < C; ++b) order[k++] = b;
    const int first = C == 2 ? (g == 0 ? 3 : 8) : (g == 0 ? 4 : 8);
    for (int b = first; b < 13; ++b) order[k++] = b;
    for (int b = C + 1; b < first; ++b) order[k++] = b;
    for (int q = 0; q < 12; ++q) t.pos[order[q]] = q;
    t.pos[C] = 12;  // the pack bit: which box copy
    return t;
}

// Landing position of tile element e (a bit permutation: linear over XOR).
QS_PHD constexpr unsigned pair_tma_land(int C, int g, unsigned e) {
    unsigned p = 0;
    for (int b = 0; b < 13; ++b) p |= ((e >> b) & 1u) << pair_tma_pos(C, g).pos[b];
    return p;
}

// Pair unit of tile element e: e with the pack bit P removed.
QS_PHD constexpr unsigned pair_unit(unsigned e, int P) {
    return (e & ((1u << P) - 1u)) | ((e >> (P + 1)) << P);
}

// Shared-memory position (in 16-byte pairs) of pair unit u; linear in u.
QS_PHD constexpr unsigned pair_phys(unsigned u) {
    return u ^ ((u >> 3) & 7u) ^ ((u >> 6) & 7u) ^ ((u >> 9) & 7u);
}

}  // namespace qs
