// Host-side planning: Ising validation and integer scaling, cost programs,
// tile shapes and the zig-zag sweep schedule.  No CUDA calls here, so the
// planner can be exercised on a machine without a GPU.
#include <cmath>
#include <cstring>
#include <vector>

#include "qs_layout.h"
#include "qs_pair.h"
#include "qs_plan.h"

namespace qs {

// Eq. (HC) restricted to one register layout.  For z = zt + (slot m placed on
// the register qubits), with zt's register bits clear and spins s = 1 - 2 b:
//   C(z) = C_out(zt) + sum_b fb_b(zt) s_b(m) + Q[m]
// where C_out holds the terms without register qubits, fb_b the field on
// register qubit b from h and the couplings to non-register qubits, and Q the
// couplings among register qubits.
std::vector<int32_t> build_cost_prog(int n, const std::vector<int32_t>& h, const std::vector<int32_t>& ei,
                                     const std::vector<int32_t>& ej, const std::vector<int32_t>& J,
                                     const int* regq, int R) {
    std::vector<int> slot(n, -1);
    for (int b = 0; b < R; ++b)
        if (regq[b] >= 0 && regq[b] < n) slot[regq[b]] = b;
    std::vector<int32_t> out(12, 0);
    out[0] = R;
    for (int b = 0; b < 6; ++b) out[5 + b] = (b < R) ? regq[b] : -1;
    int64_t const0 = 0;
    int nf = 0, ne = 0;
    for (int i = 0; i < n; ++i) {
        if (slot[i] >= 0 || (i < (int)h.size() ? h[i] : 0) == 0) continue;
        out.push_back(i);
        out.push_back(h[i]);
        const0 += h[i];
        ++nf;
    }
    const int m = (int)ei.size();
    for (int e = 0; e < m; ++e) {
        if (slot[ei[e]] >= 0 || slot[ej[e]] >= 0 || J[e] == 0) continue;
        out.push_back(ei[e] | (ej[e] << 8));
        out.push_back(J[e]);
        const0 += J[e];
        ++ne;
    }
    for (int b = 0; b < R; ++b) {
        const int q = regq[b];
        if (q < 0 || q >= n) {
            out.push_back(0);
            out.push_back(0);
            continue;
        }
        int64_t fb0 = h[q];
        std::vector<int32_t> lst;
        for (int e = 0; e < m; ++e) {
            int other = -1;
            if (ei[e] == q && slot[ej[e]] < 0) other = ej[e];
            else if (ej[e] == q && slot[ei[e]] < 0) other = ei[e];
            if (other < 0 || J[e] == 0) continue;
            fb0 += J[e];
            lst.push_back(other);
            lst.push_back(J[e]);
        }
        out.push_back((int32_t)fb0);
        out.push_back((int32_t)(lst.size() / 2));
        out.insert(out.end(), lst.begin(), lst.end());
    }
    const int qoff = (int)out.size();
    for (int mm = 0; mm < (1 << R); ++mm) {
        int64_t q = 0;
        for (int e = 0; e < m; ++e) {
            const int a = slot[ei[e]], b = slot[ej[e]];
            if (a < 0 || b < 0) continue;
            const int sa = ((mm >> a) & 1) ? -1 : 1, sb = ((mm >> b) & 1) ? -1 : 1;
            q += (int64_t)J[e] * sa * sb;
        }
        out.push_back((int32_t)q);
    }
    out[1] = nf;
    out[2] = ne;
    out[3] = (int32_t)const0;
    out[4] = qoff;
    return out;
}

int validate_ising(int n, const double* hfield, int n_edges, const int32_t* edges, const double* J,
                   IsingInt& out, std::string& err) {
    if (n < 1 || n > 40) { err = "n out of range"; return 1; }
    if (n_edges < 0 || n_edges > 4096) { err = "n_edges out of range [0, 4096]"; return 1; }
    if (!hfield && n > 0) { err = "hfield is NULL"; return 1; }
    if (n_edges > 0 && (!edges || !J)) { err = "edges or J is NULL"; return 1; }
    std::vector<char> seen;
    if (n <= 40) seen.assign((size_t)n * n, 0);
    for (int e = 0; e < n_edges; ++e) {
        const int i = edges[2 * e], j = edges[2 * e + 1];
        if (i < 0 || j < 0 || i >= n || j >= n) { err = "edge index out of range"; return 1; }
        if (i >= j) { err = "edges must satisfy i < j"; return 1; }
        if (seen[(size_t)i * n + j]) { err = "duplicate edge"; return 1; }
        seen[(size_t)i * n + j] = 1;
        if (!std::isfinite(J[e])) { err = "non-finite coupling"; return 1; }
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(hfield[i])) { err = "non-finite field"; return 1; }
    // smallest s in 0..3 with every weight * 2^s an integer
    int shift = -1;
    for (int s = 0; s <= 3 && shift < 0; ++s) {
        const double sc = std::ldexp(1.0, s);
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) ok = std::nearbyint(hfield[i] * sc) == hfield[i] * sc;
        for (int e = 0; e < n_edges && ok; ++e) ok = std::nearbyint(J[e] * sc) == J[e] * sc;
        if (ok) shift = s;
    }
    if (shift < 0) { err = "weights are not integer multiples of 2^-s for s <= 3"; return 5; }
    const double sc = std::ldexp(1.0, shift);
    out.n = n;
    out.shift = shift;
    out.h.assign(n, 0);
    out.ei.clear(); out.ej.clear(); out.J.clear();
    double bound = 0;
    for (int i = 0; i < n; ++i) {
        const double v = hfield[i] * sc;
        bound += std::fabs(v);
        if (std::fabs(v) > (double)(1 << 24)) { err = "field too large"; return 5; }
        out.h[i] = (int32_t)v;
    }
    for (int e = 0; e < n_edges; ++e) {
        const double v = J[e] * sc;
        bound += std::fabs(v);
        if (std::fabs(v) > (double)(1 << 24)) { err = "coupling too large"; return 5; }
        out.ei.push_back(edges[2 * e]);
        out.ej.push_back(edges[2 * e + 1]);
        out.J.push_back((int32_t)v);
    }
    if (bound > (double)(1 << 24)) { err = "cost range exceeds 2^24 units"; return 5; }
    out.bound = (int64_t)bound;
    return 0;
}

// Shape A: contiguous tiles of 2^K_A amplitudes rotating qubits [0, K_A - 1)
// (two 2^(K_A - 1) blocks per tile).  Then strided shapes of K_B tile bits,
// each rotating the next K_B - c_min qubits (fewer for the last one, which
// then carries more low bits so that every tile keeps K_B bits).
//
// The strided shapes split the remaining qubits [K_A - 1, n).  A tile's rows
// sit 2^(lowest target bit) apart, so a target run above the page bit
// (2 MB pages: 2^18 complex64 amplitudes) makes every row of the tile land in
// a different page: a tile with t such targets touches 2^t pages at once.  The
// qubits between K_A - 1 and the page bit are therefore dealt out evenly, one
// low run per strided shape, and each shape fills up with a high run.
std::vector<Shape> make_shapes(int nphys, const KernelCfg& cfg, int page_bit, ShapeRule rule) {
    std::vector<Shape> v;
    Shape a;
    a.K = cfg.K_A; a.c = 0; a.g0 = 0; a.nt = cfg.K_A - 1; a.kind = 0; a.n1 = 0; a.g1 = 0;
    a.ntiles = (int64_t)1 << (nphys - cfg.K_A);
    // strided shapes cover qubits [lo, hi); bits from `split` up are dealt out
    int lo = cfg.K_A - 1, hi = nphys, split = rule.split >= 0 ? rule.split : page_bit;
    const bool runs_ok = cfg.K_A == 13 && cfg.K_B == 13 && nphys >= 2 * cfg.K_A - 2;
    if (runs_ok && (rule.runs_a == 1 || (rule.runs_a < 0 && nphys >= 33))) {
        // complex64, largest states: shape A = runs of 2^8 amplitudes (2 KB)
        // with targets [0, 8) and the top four qubits, batch bit 8; the far
        // bits left go evenly to the strided shapes
        const int f = cfg.K_A - 1 - kRunBits;
        a.c = kRunBits;
        a.g0 = nphys - f;
        a.n1 = f;
        a.g1 = a.c;
        lo = a.c;
        hi = nphys - f;
        split = rule.split >= 0 ? rule.split : kFarBitC64;
        // the sweep kernel relies on this structure (tile index = bits
        // [kRunBits + 1, nphys - f), i.e. base = tile << (kRunBits + 1))
        if (a.g0 + a.n1 != nphys || a.g1 != kRunBits || a.c + a.n1 + 1 != cfg.K_A) return {};
    }
    v.push_back(a);
    const int per = cfg.K_B - (rule.cmin >= 0 ? rule.cmin : cfg.c_min);  // targets per strided shape
    const int rest = hi - lo;
    if (rest <= 0) return v;
    const int S = (rest + per - 1) / per;                  // strided shapes
    const int below = std::max(0, std::min(split, hi) - lo);  // qubits below the split bit
    const int high = rest - below;
    // water-filling: deal the high qubits one at a time to the shape holding
    // the fewest, so that the largest far footprint is as small as possible
    std::vector<int> nt(S), nh(S, 0);
    for (int k = 0; k < S; ++k) nt[k] = std::min(per, rest - k * per);
    for (int i = 0; i < high; ++i) {
        int best = -1;
        for (int k = 0; k < S; ++k)
            if (nh[k] < nt[k] && (best < 0 || nh[k] < nh[best])) best = k;
        nh[best]++;
    }
    int lo_next = lo, hi_next = lo + below;
    for (int k = 0; k < S; ++k) {
        Shape s;
        s.K = cfg.K_B;
        s.kind = 1;
        s.nt = nt[k];
        s.c = cfg.K_B - nt[k];
        s.n1 = nt[k] - nh[k];
        s.g0 = lo_next;
        lo_next += s.n1;
        s.g1 = nh[k] ? hi_next : s.g0 + s.n1;
        hi_next += nh[k];
        if (s.n1 == 0) s.g0 = s.g1;  // empty first run
        s.ntiles = (int64_t)1 << (nphys - cfg.K_B);
        v.push_back(s);
    }
    // shapes whose low run ends where their high run starts are one run
    for (auto& s : v)
        if (s.kind == 1 && s.g0 + s.n1 == s.g1) { s.n1 = 0; s.g1 = s.g0; }
    if (rule.order == 1 && v.size() > 2) std::reverse(v.begin() + 1, v.end());
    return v;
}

bool pair_tma_dims(const Shape& s, int nphys, int g, PairTmaDims& d) {
    if (s.kind != 1 || s.K != kPairK || !pair_c_ok(s.c) || (g != 0 && g != 1)) return false;
    const PairTmaPos tp = pair_tma_pos(s.c, g);
    int at[kPairK];  // tile bit on each landing position
    for (int tb = 0; tb < kPairK; ++tb) at[tp.pos[tb]] = tb;
    // positions 0..11 in order: a new dimension wherever the global bit of
    // the next position does not follow the previous one, or the box of the
    // current one is full (256 elements; dimension 0 counts floats)
    d = PairTmaDims{};
    int prev = -2;
    for (int q = 0; q + 1 < kPairK; ++q) {
        const int g = shape_bit(s, at[q]);
        if (d.rank > 0 && g == prev + 1 && d.box[d.rank - 1] < (d.rank == 1 ? 7 : 8)) {
            d.box[d.rank - 1]++;
        } else {
            if (d.rank == 5) return false;
            d.start[d.rank] = g;
            d.box[d.rank] = 1;
            d.rank++;
        }
        prev = g;
    }
    d.kbit = shape_bit(s, at[kPairK - 1]);
    if (d.start[0] != 0) return false;
    // each dimension reaches up to the next dimension's first bit
    for (int i = 0; i < d.rank; ++i) {
        int hi = nphys;
        for (int j = 0; j < d.rank; ++j)
            if (d.start[j] > d.start[i]) hi = std::min(hi, d.start[j]);
        d.width[i] = hi - d.start[i];
        // box limits: 256 elements (dimension 0 counts floats, two per amplitude)
        if (d.box[i] > d.width[i] || d.box[i] + (i == 0 ? 1 : 0) > 8 || d.width[i] + (i == 0 ? 1 : 0) > 32)
            return false;
    }
    return true;
}

void shape_regq(const Shape& s, int R, int g, int* regq) {
    const LayoutTab L = make_layout(s.K, R, s.kind);
    for (int b = 0; b < 6; ++b) {
        if (b >= R || g >= L.G) { regq[b] = -1; continue; }
        regq[b] = shape_bit(s, L.regs[g][b]);
    }
}

int num_layouts(const Shape& s, int R) { return make_layout(s.K, R, s.kind).G; }

// Zig-zag schedule: layer k visits the shapes in order 0..S-1 (k even) or
// S-1..0 (k odd).  The x-rotations of one layer commute, so the order inside a
// layer is free; with it the last sweep of layer k and the first sweep of
// layer k+1 share a shape and merge into one sweep, with the (diagonal) phase
// of layer k+1 applied between the two rounds.
std::vector<PlanSweep> plan_forward(int S, int p, bool gen) {
    std::vector<PlanSweep> v;
    for (int k = 0; k < p; ++k) {
        for (int i = 0; i < S; ++i) {
            const int s = (k % 2 == 0) ? i : (S - 1 - i);
            const bool ph = (i == 0);
            if (ph && !v.empty() && v.back().shape == s && v.back().nr < kMaxRounds) {
                v.back().r[v.back().nr++] = SweepRound{k, 1, 0, 0};
            } else {
                PlanSweep w;
                w.shape = s;
                w.nr = 1;
                w.r[0] = SweepRound{k, ph ? 1 : 0, 0, 0};
                w.flags = T_STORE;
                v.push_back(w);
            }
        }
    }
    if (v.empty()) {
        PlanSweep w;
        w.shape = 0;
        w.nr = 0;
        w.flags = T_STORE;
        v.push_back(w);
    }
    if (gen) v.front().flags |= T_GEN;
    v.back().flags |= T_READOUT;
    return v;
}

// The adjoint schedule: the forward sweeps in reverse order, each with its
// rounds reversed; a round undoes the layer's rotations, then its phase.
std::vector<PlanSweep> plan_reverse(const std::vector<PlanSweep>& fwd, const std::vector<Shape>& shapes, int p) {
    std::vector<PlanSweep> v;
    std::vector<int> cnt(p > 0 ? p : 1, 0);
    for (int i = (int)fwd.size() - 1; i >= 0; --i) {
        const PlanSweep& f = fwd[i];
        PlanSweep w;
        w.shape = f.shape;
        w.nr = f.nr;
        w.flags = T_ADJOINT | T_STORE;
        for (int r = 0; r < f.nr; ++r) {
            const SweepRound& fr = f.r[f.nr - 1 - r];
            w.r[r] = SweepRound{fr.layer, 0, fr.phase_pre, cnt[fr.layer]};
            cnt[fr.layer] += shapes[f.shape].nt;
        }
        v.push_back(w);
    }
    if (!v.empty()) v.back().flags &= ~T_STORE;  // undoes the |+> generation: nothing to keep
    return v;
}

std::vector<int32_t> build_tile_prog(const Shape& s, const std::vector<int32_t>& h, const std::vector<int32_t>& ei,
                                     const std::vector<int32_t>& ej, const std::vector<int32_t>& J) {
    const int n = (int)h.size();
    std::vector<int> tb_of(n, -1);
    for (int tb = 0; tb < s.K; ++tb) {
        const int q = shape_bit(s, tb);
        if (q >= 0 && q < n) tb_of[q] = tb;
    }
    std::vector<int32_t> out(kTileProgHead, 0);
    out[1] = s.K;
    for (int tb = 0; tb < s.K && tb < 16; ++tb) {
        const int q = shape_bit(s, tb);
        out[4 + tb] = (q >= 0 && q < n) ? h[q] : 0;
    }
    int nt = 0;
    auto term = [&](int a, int b, int c, int d) {
        out.push_back(a); out.push_back(b); out.push_back(c); out.push_back(d);
        ++nt;
    };
    for (int i = 0; i < n; ++i)
        if (tb_of[i] < 0 && h[i] != 0) term(0, i, 0, h[i]);
    for (size_t e = 0; e < ei.size(); ++e) {
        if (J[e] == 0) continue;
        const int i = ei[e], j = ej[e], ti = tb_of[i], tj = tb_of[j];
        if (ti < 0 && tj < 0) term(1, i, j, J[e]);
        else if (ti >= 0 && tj < 0) term(2 | (ti << 8), j, 0, J[e]);
        else if (ti < 0 && tj >= 0) term(2 | (tj << 8), i, 0, J[e]);
    }
    out[0] = nt;
    return out;
}

std::vector<int32_t> build_layout_prog(const Shape& s, const std::vector<int32_t>& ei, const std::vector<int32_t>& ej,
                                       const std::vector<int32_t>& J, const int* slot_tb, int R, const int* thr_tb,
                                       int NTB) {
    // qubit -> (slot bit) or (thread bit), tile qubits only
    std::vector<int> slot_q(R), thr_q(NTB);
    for (int b = 0; b < R; ++b) slot_q[b] = shape_bit(s, slot_tb[b]);
    for (int j = 0; j < NTB; ++j) thr_q[j] = shape_bit(s, thr_tb[j]);
    auto find = [](const std::vector<int>& v, int q) {
        for (size_t k = 0; k < v.size(); ++k)
            if (v[k] == q) return (int)k;
        return -1;
    };
    const size_t NS = (size_t)1 << R, NT = (size_t)1 << NTB;
    std::vector<int32_t> out(NS + 8 * NT, 0);
    for (size_t e = 0; e < ei.size(); ++e) {
        if (J[e] == 0) continue;
        const int sa = find(slot_q, ei[e]), sb = find(slot_q, ej[e]);
        const int ta = find(thr_q, ei[e]), tb = find(thr_q, ej[e]);
        auto spin = [](size_t idx, int bit) { return ((idx >> bit) & 1) ? -1 : 1; };
        if (sa >= 0 && sb >= 0) {
            for (size_t m = 0; m < NS; ++m) out[m] += J[e] * spin(m, sa) * spin(m, sb);
        } else if (ta >= 0 && tb >= 0) {
            for (size_t t = 0; t < NT; ++t) out[NS + 8 * t] += J[e] * spin(t, ta) * spin(t, tb);
        } else if (sa >= 0 && tb >= 0) {
            for (size_t t = 0; t < NT; ++t) out[NS + 8 * t + 1 + sa] += J[e] * spin(t, tb);
        } else if (sb >= 0 && ta >= 0) {
            for (size_t t = 0; t < NT; ++t) out[NS + 8 * t + 1 + sb] += J[e] * spin(t, ta);
        }
    }
    return out;
}

int count_sweeps(int nphys, int dtype, int p) {
    const KernelCfg cfg = kernel_cfg(dtype, false);
    const auto sh = make_shapes(nphys, cfg, page_bit_for(dtype));
    return (int)plan_forward((int)sh.size(), p, true).size();
}

// Tile bits and register bits per configuration.  complex64: 2^13-amplitude
// tiles (64 KB); complex128: 2^12 (64 KB).  The adjoint holds psi and lambda,
// so it keeps half as many amplitudes per thread on the same tiles.
KernelCfg kernel_cfg(int dtype, bool adjoint) {
    if (dtype == 0) return adjoint ? KernelCfg{13, 13, 5, 2} : KernelCfg{13, 13, 6, 2};
    return adjoint ? KernelCfg{12, 12, 4, 2} : KernelCfg{12, 12, 5, 2};
}

}  // namespace qs
