// Host-side planning declarations (no CUDA dependencies).
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {

struct IsingInt {
    int n = 0, shift = 0;
    std::vector<int32_t> h, ei, ej, J;  // weights scaled by 2^shift
    int64_t bound = 0;                   // sum |h| + sum |J| (scaled)
};

// 0 = ok, 1 = QS_EINVAL, 5 = QS_ENOTINT; err receives the reason.
int validate_ising(int n, const double* hfield, int n_edges, const int32_t* edges, const double* J, IsingInt& out,
                   std::string& err);

// A tile shape (see qs_layout.h).  Tile bits [0, c) are global bits [0, c),
// tile bits [c, c + n1) global [g0, g0 + n1), the rest global [g1, ...).
//   kind 0: targets are tile bits [0, K - 1).  Contiguous (c = n1 = g1 = 0),
//           or runs of 2^c amplitudes whose tile bits [c, K - 1) sit on the
//           top global bits (g0) and whose batch bit K - 1 is global bit c.
//   kind 1: c carried low bits (not targets) + nt = K - c targets in the two
//           runs [g0, g0 + n1) and [g1, g1 + nt - n1) (n1 may be 0).
struct Shape {
    int K, c, g0, nt, kind, n1, g1;
    int64_t ntiles;
};

// Global bit of tile bit tb of a shape.
inline int shape_bit(const Shape& s, int tb) {
    if (tb < s.c) return tb;
    if (tb < s.c + s.n1) return s.g0 + (tb - s.c);
    return s.g1 + (tb - s.c - s.n1);
}

// Sweep-kernel kind of a shape: 0 contiguous, 1 strided, 2 kind-0 runs.
inline int kernel_kind(const Shape& s) { return s.kind == 0 && (s.c != 0 || s.n1 != 0) ? 2 : s.kind; }

// Complex64 index bit from which amplitudes lie 32 MB or more apart: a
// strided tile with many target bits at or above it streams far slower at
// 32-byte runs (measured), so the largest states spread those bits over all
// shapes, including a run-structured shape A.
constexpr int kFarBitC64 = 22;

struct PlanSweep {
    int shape = 0;
    int nr = 0;
    int flags = 0;
    SweepRound r[kMaxRounds];
};

// Index bit at which a new 2 MB page starts (complex64: 8-byte amplitudes).
inline int page_bit_for(int dtype) { return dtype == 0 ? 18 : 17; }
// Shape-plan choice (set by the autotuner or the caller): runs_a = 1 makes
// shape A run-structured (complex64, K = 13), 0 contiguous, -1 the default
// rule (run-structured from 33 qubits); split = index bit from which the
// strided shapes' qubits are dealt out evenly, -1 = default (bit 22 with a
// run-structured A, else the 2 MB page bit); cmin = carried bits of the
// strided shapes (each holds 13 - cmin targets in rows of 2^cmin amplitudes);
// order = 1 reverses the strided shapes (which of them the zig-zag merges).
struct ShapeRule {
    int runs_a = -1;
    int split = -1;
    int cmin = -1;  // carried low bits of the strided shapes (2 or 3; -1 = the kernel default, 2)
    int order = 0;  // 1: the strided shapes in reverse order (the zig-zag merges the last shape's sweeps)
};
inline bool same_shapes(const ShapeRule& a, const ShapeRule& b) {
    return a.runs_a == b.runs_a && a.split == b.split && a.cmin == b.cmin && a.order == b.order;
}
std::vector<Shape> make_shapes(int nphys, const KernelCfg& cfg, int page_bit, ShapeRule rule = ShapeRule{});

// Tensor-map view of a strided packed-pair tile (complex64, K = 13, c = 2 or
// 3) in the landing order pair_tma_pos(c, g) of a tile first read into
// layout g: dimension d covers global index
// bits [start[d], start[d] + width[d]), of which the box holds the lowest
// box[d]; dimension 0 starts at bit 0 (the carried run).  Every global bit
// belongs to one dimension: bits that are neither box bits nor the pack bit
// (global bit kbit) are the tile index, set by the copy's coordinates.
// False when the shape does not fit five dimensions in that order.
struct PairTmaDims {
    int rank = 0, kbit = 0;
    int start[5] = {}, width[5] = {}, box[5] = {};
};
bool pair_tma_dims(const Shape& s, int nphys, int g, PairTmaDims& d);
void shape_regq(const Shape& s, int R, int g, int* regq);
int num_layouts(const Shape& s, int R);
std::vector<PlanSweep> plan_forward(int S, int p, bool gen);
std::vector<PlanSweep> plan_reverse(const std::vector<PlanSweep>& fwd, const std::vector<Shape>& shapes, int p);
int count_sweeps(int nphys, int dtype, int p);

// Tile programs: Eq. (HC) split by where each term's qubits sit relative to a
// tile of a shape.  With O the qubits outside the tile (the tile index), T a
// layout's thread-index qubits and R its register-slot qubits, and spins s
// of the stored index z, the cost is
//   C = Kf + Kc + sum_{t in T} (h_t + D_t) s_t + TT + sum_{b in R} (h_b + D_b + hRT_b) s_b + Q[slot]
// with Kf = sum_{O} h s, Kc = sum_{O-O} J s s and D_q = sum_{o in O} J_qo s_o
// (per tile, from the tile's base index), TT = sum_{T-T} J s s and hRT_b =
// sum_{t in T} J_bt s_t (per thread and layout) and Q the couplings among
// the slot qubits.  A stored array in the flipped frame (every bit inverted)
// negates every field: Kf, h_t, h_b change sign, nothing else.
//
// Tile program (layout-independent):
//   [0] nterms  [1] K  [2..4) 0  [4..20) H[16]: field of the qubit on tile bit tb
//   [20 ...) nterms int4 terms: (0, i, 0, h_i) -> Kf;  (1, i, j, J) -> Kc;
//   (2 | tb << 8, o, 0, J) -> D[tb]   (i, j, o outside the tile)
std::vector<int32_t> build_tile_prog(const Shape& s, const std::vector<int32_t>& h, const std::vector<int32_t>& ei,
                                     const std::vector<int32_t>& ej, const std::vector<int32_t>& J);
// Layout program of one register layout of a kernel: Q[2^R], then for each
// thread index t < 2^NTB eight ints (TT, hRT[0..R), 0...).  slot_tb[b] is the
// tile bit of register-slot bit b, thr_tb[j] that of thread-index bit j.
std::vector<int32_t> build_layout_prog(const Shape& s, const std::vector<int32_t>& ei, const std::vector<int32_t>& ej,
                                       const std::vector<int32_t>& J, const int* slot_tb, int R, const int* thr_tb,
                                       int NTB);

}  // namespace qs
