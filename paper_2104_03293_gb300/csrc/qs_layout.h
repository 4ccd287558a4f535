// Register layouts of a tile, shared by the host planner (cost programs) and
// the sweep kernel (constexpr), so both sides agree on which tile bits a
// thread holds in registers.
//
// A tile has K bits.  Two kinds:
//   kind 0 ("contiguous"): the tile is 2^K consecutive amplitudes; its targets
//          are tile bits [0, K-1); bit K-1 only pairs two such target blocks
//          in one CTA (it is never rotated by this shape).
//   kind 1 ("strided"): tile bits [0, c) are the c lowest index bits, carried
//          so that every tile row is contiguous in HBM; tile bits [c, K) are
//          the targets, global bits g0 .. g0 + K - c - 1 (c chosen per shape).
// Registers: a thread holds 2^R amplitudes.  Tile bits are ranked (kind 0:
// K-2, K-3, ..., 0, K-1; kind 1: K-1, ..., 0); layout g puts the ranked bits
// [g R, (g + 1) R) into the register slot index (a last, partial group holds
// tile bits [0, R) instead) and the remaining K - R tile bits, in ascending
// order, into the thread index (the lowest five are the lane).  Layout g
// rotates the targets among ranked bits [g R, (g + 1) R).
#pragma once

#ifdef __CUDACC__
#define QS_HD __host__ __device__
#else
#define QS_HD
#endif

namespace qs {

constexpr int kMaxLay = 3;

struct LayoutTab {
    int K, R, kind, G;
    int regs[kMaxLay][8];    // tile bit of register slot bit b (ascending)
    int tbits[kMaxLay][16];  // tile bit of thread-index bit j (ascending)
    int rot_lo[kMaxLay];     // ranked positions [rot_lo, rot_hi) rotated in layout g
    int rot_hi[kMaxLay];
};

QS_HD constexpr int ranked_bit(int K, int kind, int i) {
    return kind == 0 ? (i < K - 1 ? K - 2 - i : K - 1) : K - 1 - i;
}

QS_HD constexpr LayoutTab make_layout(int K, int R, int kind) {
    LayoutTab t{};
    t.K = K;
    t.R = R;
    t.kind = kind;
    const int ntg = kind == 0 ? K - 1 : K;  // bits that can be targets
    t.G = (ntg + R - 1) / R;
    for (int g = 0; g < t.G; ++g) {
        bool inreg[32] = {};
        if (g * R + R <= ntg) {
            for (int i = g * R; i < g * R + R; ++i) inreg[ranked_bit(K, kind, i)] = true;
        } else {
            // partial last group: its targets are the lowest tile bits; hold
            // tile bits [0, R) so that the lanes stay on contiguous bits
            for (int b = 0; b < R; ++b) inreg[b] = true;
        }
        int nr = 0, nt = 0;
        for (int b = 0; b < K; ++b) {
            if (inreg[b]) t.regs[g][nr++] = b;
            else t.tbits[g][nt++] = b;
        }
        t.rot_lo[g] = g * R;
        t.rot_hi[g] = (g + 1) * R < ntg ? (g + 1) * R : ntg;
    }
    return t;
}

// Ranked position of tile bit b (inverse of ranked_bit).
QS_HD constexpr int rank_of(int K, int kind, int b) {
    return kind == 0 ? (b == K - 1 ? K - 1 : K - 2 - b) : K - 1 - b;
}

}  // namespace qs
