#pragma once
// Tiled HBM sweep kernel: one read + one write of the state (or of psi and
// lambda) per launch, with the x-rotations of the tile's target bits
// (Eq. twocomponentupdates applied to e^{-i beta X}, Sec. III.B.1), the
// diagonal phase e^{-i gamma H_C} (Eq. HC, computed from the bit pattern, no
// 2^n diagonal), the readout (<H_C>, ground probability, norm) and the adjoint
// accumulations fused in.
//
// Persistent CTAs (two per SM for the forward sweep, one for the adjoint) walk
// over tiles of 2^K amplitudes:
//   * a tile lands in the CTA's shared-memory tile buffer: one bulk copy
//     (cp.async.bulk, TMA) for a contiguous tile, one per 2 KB run (warp 0)
//     for a run-structured one (kind 2), per-thread 16-byte cp.async copies
//     for a strided one (runs of 2^c amplitudes); all
//     complete on an mbarrier, with bounded waits.  The load of the next tile
//     is issued as soon as the current one has been read for the last time,
//     so it overlaps the tile's remaining work and the other CTA.
//   * each thread holds 2^R amplitudes per array in registers.  A layout
//     (qs_layout.h) assigns R tile bits to the register slot index; the
//     rotations of those bits are register butterflies.  Changing layout is a
//     transpose through a swizzled shared-memory tile.
//   * a round rotates every target once: the layouts in turn, then the next
//     round walks them back, so two rounds share the layout at their boundary
//     (the zig-zag inside a tile, matching the zig-zag of the sweep schedule).
//   * the butterfly is the tangent form a' = a + w (-i b), |w| <= 1; the
//     scalar per rotation is folded into the layer's phase table.
//   * results leave from registers in layout 0 with coalesced stores.
#include <type_traits>

#include <cuda.h>
#include <cuda_runtime.h>

#include "qs_internal.h"
#include "qs_layout.h"

namespace qs {

template <class Real> struct C2T;
template <> struct C2T<float> { using T = float2; };
template <> struct C2T<double> { using T = double2; };

template <class Real> __device__ __forceinline__ Real fma_(Real a, Real b, Real c) { return fma(a, b, c); }


// Compile-time loop: f(std::integral_constant<int, I>) for I in [Begin, End).
template <int I, int End, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < End) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, End>(f);
    }
}

// Shared-memory swizzle: phys(e) = e ^ ((e >> R) & 31).  It is linear
// (phys(a ^ b) = phys(a) ^ phys(b)), so a thread's base and its compile-time
// slot offsets combine with one XOR, and it makes every layout's accesses
// conflict-free for the configurations in kernel_cfg (checked on the host by
// the test-suite, tests/test_index_math.py).
template <int R> struct Swz {
    static constexpr int S = R;
    __host__ __device__ static constexpr uint32_t phys(uint32_t e) { return e ^ ((e >> S) & 31u); }
};

// ---------------------------------------------------------------------------
// mbarrier / TMA primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier, giving up after ~2 s of device time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && globaltimer() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Contiguous copy global -> shared, completion on the barrier.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Index maps
// ---------------------------------------------------------------------------
// Tile map: tile bits [0, c) are global bits [0, c); tile bits [c, c + n1)
// are global [g0, g0 + n1); tile bits [c + n1, K) are global [g1, ...).  The
// two runs may lie in either order above c.  The non-tile global bits, in
// ascending order, take the tile index.  A contiguous tile is c = 0, n1 = 0,
// g1 = 0; other kind-0 tiles are runs of 2^c amplitudes whose higher tile bits
// lie on distant global bits.
struct TMap {
    int c, g0, n1, g1, K;
    __device__ __forceinline__ uint64_t gofs(uint32_t e) const {
        const uint32_t cm = (1u << c) - 1u, m1 = (1u << n1) - 1u;
        return (uint64_t)(e & cm) | ((uint64_t)((e >> c) & m1) << g0) | ((uint64_t)(e >> (c + n1)) << g1);
    }
    // global bit of tile bit tb
    __device__ __forceinline__ int gbit(int tb) const {
        return tb < c ? tb : (tb < c + n1 ? g0 + tb - c : g1 + tb - c - n1);
    }
    // tile bit holding global bit q, or -1 when q lies outside the tile
    __device__ __forceinline__ int tile_bit(int q) const {
        if (q < c) return q;
        if (q >= g0 && q < g0 + n1) return c + q - g0;
        if (q >= g1 && q < g1 + K - c - n1) return c + n1 + q - g1;
        return -1;
    }
    __device__ __forceinline__ uint64_t base(int64_t t) const {
        // occupied runs above c in ascending global order: [s1, s1 + l1), [s2, s2 + l2)
        int s1 = g0, l1 = n1, s2 = g1, l2 = K - c - n1;
        if (l1 == 0) { s1 = s2; l1 = l2; l2 = 0; }
        if (l2 > 0 && s2 < s1) { const int ts = s1, tl = l1; s1 = s2; l1 = l2; s2 = ts; l2 = tl; }
        const int la = s1 - c;                        // gap [c, s1)
        const uint64_t u = (uint64_t)t;
        const uint64_t ma = la > 0 ? (1ull << la) - 1ull : 0ull;
        if (l2 == 0) return ((u & ma) << c) | ((u >> la) << (s1 + l1));
        const int lb = s2 - (s1 + l1);                // gap [s1 + l1, s2)
        const uint64_t mb = lb > 0 ? (1ull << lb) - 1ull : 0ull;
        return ((u & ma) << c) | (((u >> la) & mb) << (s1 + l1)) | ((u >> (la + lb)) << (s2 + l2));
    }
};

// ---------------------------------------------------------------------------
// Per-tile cost tables (see build_tile_prog / build_layout_prog).
// ---------------------------------------------------------------------------
struct TileTab {
    int kf, kc, pad0, pad1;
    int D[16];  // couplings of the qubit on tile bit tb to the qubits outside the tile
    int H[16];  // field of the qubit on tile bit tb
};

// Warp 0: the table of the tile whose base index (tile bits clear) is zb.
// The caller orders it before the table's readers with a block barrier.
__device__ __forceinline__ void tile_tab_fill(TileTab* tt, const int32_t* __restrict__ tp, uint64_t zb,
                                              uint32_t lane) {
    if (lane < 16) {
        tt->D[lane] = 0;
        tt->H[lane] = __ldg(tp + 4 + lane);
    }
    __syncwarp();
    const int nterms = __ldg(tp);
    const int4* terms = reinterpret_cast<const int4*>(tp + kTileProgHead);
    int kf = 0, kc = 0;
    for (int k = (int)lane; k < nterms; k += 32) {
        const int4 t = __ldg(terms + k);
        const int si = 1 - 2 * (int)((zb >> t.y) & 1ull);
        const int kind = t.x & 255;
        if (kind == 0) kf += t.w * si;
        else if (kind == 1) kc += t.w * si * (1 - 2 * (int)((zb >> t.z) & 1ull));
        else atomicAdd(&tt->D[t.x >> 8], t.w * si);
    }
    kf = __reduce_add_sync(0xffffffffu, kf);
    kc = __reduce_add_sync(0xffffffffu, kc);
    if (lane == 0) {
        tt->kf = kf;
        tt->kc = kc;
    }
}

// ---------------------------------------------------------------------------
// Cost program evaluation (see build_cost_prog).
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ int eval_cost(const int32_t* __restrict__ cp, uint64_t z, int (&fb)[R], const int32_t*& q) {
    const int nf = __ldg(cp + 1), ne = __ldg(cp + 2), const0 = __ldg(cp + 3), qoff = __ldg(cp + 4);
    const int32_t* t = cp + 12;
    int acc = 0;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) acc += __ldg(t + 2 * k + 1) * (int)((z >> __ldg(t + 2 * k)) & 1ull);
    t += 2 * nf;
#pragma unroll 4
    for (int k = 0; k < ne; ++k) {
        const int ij = __ldg(t + 2 * k), J = __ldg(t + 2 * k + 1);
        acc += J * (int)(((z >> (ij & 255)) ^ (z >> (ij >> 8))) & 1ull);
    }
    t += 2 * ne;
#pragma unroll
    for (int b = 0; b < R; ++b) {
        const int fb0 = __ldg(t), cnt = __ldg(t + 1);
        t += 2;
        int a2 = 0;
        for (int k = 0; k < cnt; ++k) a2 += __ldg(t + 2 * k + 1) * (int)((z >> __ldg(t + 2 * k)) & 1ull);
        t += 2 * cnt;
        fb[b] = fb0 - 2 * a2;
    }
    q = cp + qoff;
    return const0 - 2 * acc;
}

// idx(m) = C(slot m) - cost_lo from two partial-sum tables over the low /
// high halves of the register bits plus the intra-register coupling table Q.
template <int R>
struct SlotCost {
    static constexpr int R1 = R / 2, R2 = R - R1;
    int plo[1 << R1], phi[1 << R2];
    const int32_t* q;
    __device__ __forceinline__ void init(const int32_t* __restrict__ cp, uint64_t zt, int flip, int cost_lo) {
        int fb[R];
        const int cout = eval_cost<R>(cp, zt, fb, q);
        if (flip) {
#pragma unroll
            for (int b = 0; b < R; ++b) fb[b] = -fb[b];
        }
        int base = cout - cost_lo;
#pragma unroll
        for (int b = 0; b < R1; ++b) base += fb[b];
        plo[0] = base;
#pragma unroll
        for (int b = 0; b < R1; ++b)
#pragma unroll
            for (int k = 0; k < (1 << b); ++k) plo[k | (1 << b)] = plo[k] - 2 * fb[b];
        int hb = 0;
#pragma unroll
        for (int b = 0; b < R2; ++b) hb += fb[R1 + b];
        phi[0] = hb;
#pragma unroll
        for (int b = 0; b < R2; ++b)
#pragma unroll
            for (int k = 0; k < (1 << b); ++k) phi[k | (1 << b)] = phi[k] - 2 * fb[R1 + b];
    }
    // From the tile table: Map::slot(b) / Map::thr(j) are the tile bits of
    // register-slot bit b and thread-index bit j of the layout; lp is the
    // layout program; frame = 1 when the stored array is bit-flipped.
    template <class Map, int NTB>
    __device__ __forceinline__ void init_tile(const TileTab& tt, const int32_t* __restrict__ lp, uint32_t tid,
                                              int frame, int cost_lo) {
        const int sg = frame ? -1 : 1;
        const int4* tr = reinterpret_cast<const int4*>(lp + (1 << R)) + 2 * tid;
        const int4 a = __ldg(tr), b = __ldg(tr + 1);
        const int hrt[6] = {a.y, a.z, a.w, b.x, b.y, b.z};
        int cout = sg * tt.kf + tt.kc + a.x;
        static_for<0, NTB>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr int tb = Map::thr(j);
            const int v = sg * tt.H[tb] + tt.D[tb];
            cout += ((tid >> j) & 1u) ? -v : v;
        });
        int fb[R];
        static_for<0, R>([&](auto bc) {
            constexpr int bb = decltype(bc)::value;
            constexpr int tb = Map::slot(bb);
            fb[bb] = sg * tt.H[tb] + tt.D[tb] + hrt[bb];
        });
        q = lp;
        int base = cout - cost_lo;
#pragma unroll
        for (int b2 = 0; b2 < R1; ++b2) base += fb[b2];
        plo[0] = base;
#pragma unroll
        for (int b2 = 0; b2 < R1; ++b2)
#pragma unroll
            for (int k = 0; k < (1 << b2); ++k) plo[k | (1 << b2)] = plo[k] - 2 * fb[b2];
        int hb = 0;
#pragma unroll
        for (int b2 = 0; b2 < R2; ++b2) hb += fb[R1 + b2];
        phi[0] = hb;
#pragma unroll
        for (int b2 = 0; b2 < R2; ++b2)
#pragma unroll
            for (int k = 0; k < (1 << b2); ++k) phi[k | (1 << b2)] = phi[k] - 2 * fb[R1 + b2];
    }
    __device__ __forceinline__ int idx(int m) const { return plo[m & ((1 << R1) - 1)] + phi[m >> R1] + __ldg(q + m); }
    // without the intra-register couplings Q[m] (the caller adds them)
    __device__ __forceinline__ int idx_noq(int m) const { return plo[m & ((1 << R1) - 1)] + phi[m >> R1]; }
    // table index, kept inside [0, top] so that no cost can address memory
    // outside the phase table (one unsigned minimum: a negative index wraps
    // to a large one and is clamped to top)
    __device__ __forceinline__ static int clamp_tab(int ix, int top) { return (int)min((unsigned)ix, (unsigned)top); }
    __device__ __forceinline__ int tidx(int m, int top) const { return clamp_tab(idx(m), top); }
};

// Phase of a thread's 64 amplitudes held as 32 packed pairs (X[j] = the real
// parts, Y[j] = the imaginary parts of slots 2j and 2j + 1; slot bit 0 is the
// pack bit, slot bits 1..5 are the pair-index bits), layout Map (slot(b),
// thr(t) as in SlotCost::init_tile), layout program lp, intra-register
// couplings q (compile-time indexed; kernel parameters).  The cost of slot m
// is base - sum over the set bits b of m of f2[b], plus q[m]: base = the
// cost with every slot spin up (the tile constant, this thread's terms and
// every slot bit's term fb, less cost_lo) and f2[b] = 2 fb[b].  The slots
// are walked in four Gray-code chains (slot bits 4, 5 fixed per chain), one
// add per slot, which keeps eight values live instead of two 8-entry
// partial-sum tables.
template <class Map, int NTB>
__device__ __forceinline__ void pair_phase(float2 (&X)[32], float2 (&Y)[32], const int32_t* __restrict__ lp,
                                           const TileTab& tt, uint32_t tid, int frame, int cost_lo,
                                           const float2* __restrict__ tab, int top, const int32_t (&q)[64]) {
    const int sg = frame ? -1 : 1;
    const int4* tr = reinterpret_cast<const int4*>(lp + 64) + 2 * tid;
    const int4 ta = __ldg(tr), tb4 = __ldg(tr + 1);
    const int hrt[6] = {ta.y, ta.z, ta.w, tb4.x, tb4.y, tb4.z};
    int base = sg * tt.kf + tt.kc + ta.x - cost_lo;
    static_for<0, NTB>([&](auto jc) {
        constexpr int t = decltype(jc)::value;
        constexpr int tb = Map::thr(t);
        const int v = sg * tt.H[tb] + tt.D[tb];
        base += ((tid >> t) & 1u) ? -v : v;
    });
    int f2[6];
    static_for<0, 6>([&](auto bc) {
        constexpr int bb = decltype(bc)::value;
        constexpr int tb = Map::slot(bb);
        const int fb = sg * tt.H[tb] + tt.D[tb] + hrt[bb];
        base += fb;
        f2[bb] = 2 * fb;
    });
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        int run = base - ((ch & 1) ? f2[4] : 0) - ((ch & 2) ? f2[5] : 0);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int gc = i ^ (i >> 1);
            if (i > 0) {
                const int bb = __ffs(i) - 1;  // the bit that flips at step i
                run += ((gc >> bb) & 1) ? -f2[bb] : f2[bb];
            }
            const int m = (ch << 4) | gc, j = m >> 1;
            const float2 f = tab[SlotCost<6>::clamp_tab(run + q[m], top)];
            if (m & 1) {
                const float br = X[j].y, bi = Y[j].y;
                X[j].y = fmaf(br, f.x, -bi * f.y);
                Y[j].y = fmaf(br, f.y, bi * f.x);
            } else {
                const float ar = X[j].x, ai = Y[j].x;
                X[j].x = fmaf(ar, f.x, -ai * f.y);
                Y[j].x = fmaf(ar, f.y, ai * f.x);
            }
        }
    }
}

// Readout of a thread's 64 amplitudes held as 32 packed pairs (layout Map,
// as pair_phase): with the slot costs walked as in pair_phase, accumulates
// E += |psi|^2 C, P += |psi|^2 on the minimal cost (table index gidx) and
// N += |psi|^2, in float.
template <class Map, int NTB>
__device__ __forceinline__ void pair_readout(const float2 (&X)[32], const float2 (&Y)[32],
                                             const int32_t* __restrict__ lp, const TileTab& tt, uint32_t tid,
                                             int frame, int cost_lo, int gidx, const int32_t (&q)[64], float& E,
                                             float& P, float& N) {
    const int sg = frame ? -1 : 1;
    const int4* tr = reinterpret_cast<const int4*>(lp + 64) + 2 * tid;
    const int4 ta = __ldg(tr), tb4 = __ldg(tr + 1);
    const int hrt[6] = {ta.y, ta.z, ta.w, tb4.x, tb4.y, tb4.z};
    int base = sg * tt.kf + tt.kc + ta.x - cost_lo;
    static_for<0, NTB>([&](auto jc) {
        constexpr int t = decltype(jc)::value;
        constexpr int tb = Map::thr(t);
        const int v = sg * tt.H[tb] + tt.D[tb];
        base += ((tid >> t) & 1u) ? -v : v;
    });
    int f2[6];
    static_for<0, 6>([&](auto bc) {
        constexpr int bb = decltype(bc)::value;
        constexpr int tb = Map::slot(bb);
        const int fb = sg * tt.H[tb] + tt.D[tb] + hrt[bb];
        base += fb;
        f2[bb] = 2 * fb;
    });
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        int run = base - ((ch & 1) ? f2[4] : 0) - ((ch & 2) ? f2[5] : 0);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int gc = i ^ (i >> 1);
            if (i > 0) {
                const int bb = __ffs(i) - 1;
                run += ((gc >> bb) & 1) ? -f2[bb] : f2[bb];
            }
            const int m = (ch << 4) | gc, j = m >> 1;
            const int ix = run + q[m];
            const float re = (m & 1) ? X[j].y : X[j].x, im = (m & 1) ? Y[j].y : Y[j].x;
            const float w2 = fmaf(re, re, im * im);
            E = fmaf(w2, (float)(ix + cost_lo), E);
            N += w2;
            if (ix == gidx) P += w2;
        }
    }
}

// Warp-level sum, lane 0 stores into red[warp * nslots + slot].
__device__ __forceinline__ void warp_sum_to(double v, double* red, int slot, int nslots) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) * nslots + slot] = v;
}

// ---------------------------------------------------------------------------
// Spin expectations <Z_q> = sum_z |psi_z|^2 s_q(z), s_q = 1 - 2 bit_q (the
// per-qubit magnetisations recorded during AQA, Sec. III.B.2, Fig. 6).
// ---------------------------------------------------------------------------
// This thread's share, by tile bit: zv[tb] = sum_m w[m] s_tb over its 2^R
// amplitudes (w = |psi|^2 in slot m; Map::slot(b) / Map::thr(j) are the tile
// bits of slot bit b and thread-index bit j), zv[K] = sum_m w[m].
template <class Map, int K, int R, class F>
__device__ __forceinline__ void z_thread_sums(const F (&w)[1 << R], uint32_t tid, F (&zv)[K + 1]) {
    F W = 0;
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) W += w[m];
    static_for<0, R>([&](auto bc) {
        constexpr int b = decltype(bc)::value;
        F hi = 0;  // weight of the slots with bit b set (s = -1)
#pragma unroll
        for (int m = 0; m < (1 << R); ++m)
            if ((m >> b) & 1) hi += w[m];
        zv[Map::slot(b)] = W - 2 * hi;
    });
    static_for<0, K - R>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        zv[Map::thr(j)] = ((tid >> j) & 1u) ? -W : W;
    });
    zv[K] = W;
}

// Sum zv over the CTA and add the tile's contribution to zacc[q], q < nq:
// a qubit on a tile bit takes that bit's sum, a qubit outside the tile the
// tile's weight times its spin in the tile's base index; sg = -1 when the
// stored array is in the flipped frame (every spin negated).  zred holds
// NW * (K + 1) values.  Called by every thread; the accumulators are FP64 and
// each CTA adds its tiles in a fixed order, so the sums are reproducible.
template <int K, int NW, class F>
__device__ __forceinline__ void z_tile_add(F (&zv)[K + 1], F* zred, double* zacc, const TMap& tm, uint64_t zb,
                                           int nq, int sg, uint32_t tid) {
#pragma unroll
    for (int i = 0; i <= K; ++i) {
        F v = zv[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        zv[i] = v;
    }
    if ((tid & 31u) == 0) {
#pragma unroll
        for (int i = 0; i <= K; ++i) zred[(tid >> 5) * (K + 1) + i] = zv[i];
    }
    __syncthreads();
    if (tid < 32) {
        for (int q = (int)tid; q < nq; q += 32) {
            const int tb = tm.tile_bit(q);
            const int col = tb >= 0 ? tb : K;
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) s += (double)zred[w * (K + 1) + col];
            if (tb < 0 && ((zb >> q) & 1ull)) s = -s;
            zacc[q] += sg < 0 ? -s : s;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// The sweep
// ---------------------------------------------------------------------------
template <class Real, int K, int R, int NA, int KIND>
struct Sweep {
    using C2 = typename C2T<Real>::T;
    // layout tables as compile-time scalars (qs_layout.h)
    // KIND 2 (run-structured kind-0 tiles) uses the kind-0 layouts
    static constexpr int LK = KIND == 2 ? 0 : KIND;
    static constexpr int G = make_layout(K, R, LK).G;
    template <int g, int b> __host__ __device__ static constexpr int reg_bit() { return make_layout(K, R, LK).regs[g][b]; }
    template <int g, int j> __host__ __device__ static constexpr int thr_bit() { return make_layout(K, R, LK).tbits[g][j]; }
    template <int g> __host__ __device__ static constexpr int rot_lo() { return make_layout(K, R, LK).rot_lo[g]; }
    template <int g> __host__ __device__ static constexpr int rot_hi() { return make_layout(K, R, LK).rot_hi[g]; }
    static constexpr int NT = 1 << (K - R);
    static constexpr int NS = 1 << R;
    static constexpr int NW = NT / 32;
    static constexpr int NSLOT = 2 * kMaxRounds;
    static constexpr size_t TILE_BYTES = (size_t)sizeof(C2) << K;
    static constexpr size_t BUF_BYTES = (size_t)NA * TILE_BYTES;  // one region per array
    static constexpr size_t TT_OFF = BUF_BYTES + 64 + (size_t)NW * NSLOT * 8;  // two TileTabs
    static constexpr size_t SMEM_BYTES = TT_OFF + 2 * sizeof(TileTab);
    // T_ZEXP kernels: FP64 accumulators [kZSlots][kZQ], then the warp sums
    static constexpr size_t Z_BYTES = (size_t)kZSlots * kZQ * 8 + (size_t)NW * (K + 1) * sizeof(Real);
    static_assert(SMEM_BYTES % 8 == 0, "accumulators follow the tile tables");
    static_assert(K - R >= 5, "a tile needs at least one full warp");
    // compile-time tile bits of layout g for SlotCost::init_tile
    template <int g> struct Map {
        __host__ __device__ static constexpr int slot(int b) { return make_layout(K, R, LK).regs[g][b]; }
        __host__ __device__ static constexpr int thr(int j) { return make_layout(K, R, LK).tbits[g][j]; }
    };
    static_assert(G <= kMaxLay, "too many layouts");

    template <int g>
    __device__ static __forceinline__ uint32_t e_thread(uint32_t tid) {
        uint32_t e = 0;
        static_for<0, K - R>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            e |= ((tid >> j) & 1u) << thr_bit<g, j>();
        });
        return e;
    }
    template <int g>
    __device__ static __forceinline__ uint32_t e_slot(int m) {
        uint32_t e = 0;
        static_for<0, R>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            e |= (uint32_t)((m >> b) & 1) << reg_bit<g, b>();
        });
        return e;
    }

    // ---- shared-memory transposes ------------------------------------------
    template <int g>
    __device__ static __forceinline__ void sts(C2* tb, const C2 (&x)[NS], uint32_t tid) {
        const uint32_t pt = Swz<R>::phys(e_thread<g>(tid));
#pragma unroll
        for (int m = 0; m < NS; ++m) tb[pt ^ Swz<R>::phys(e_slot<g>(m))] = x[m];
    }
    template <int g>
    __device__ static __forceinline__ void lds(const C2* tb, C2 (&x)[NS], uint32_t tid) {
        const uint32_t pt = Swz<R>::phys(e_thread<g>(tid));
#pragma unroll
        for (int m = 0; m < NS; ++m) x[m] = tb[pt ^ Swz<R>::phys(e_slot<g>(m))];
    }
    template <int g>
    __device__ static __forceinline__ void lds_dense(const C2* src, C2 (&x)[NS], uint32_t tid) {
        const uint32_t et = e_thread<g>(tid);
#pragma unroll
        for (int m = 0; m < NS; ++m) x[m] = src[et | e_slot<g>(m)];
    }
    __device__ static __forceinline__ void sts_any(int g, C2* tb, const C2 (&x)[NS], uint32_t tid) {
        if (g == 0) sts<0>(tb, x, tid);
        else if (G > 1 && g == 1) sts<(G > 1 ? 1 : 0)>(tb, x, tid);
        else if (G > 2) sts<(G > 2 ? 2 : 0)>(tb, x, tid);
    }
    __device__ static __forceinline__ void lds_any(int g, const C2* tb, C2 (&x)[NS], uint32_t tid) {
        if (g == 0) lds<0>(tb, x, tid);
        else if (G > 1 && g == 1) lds<(G > 1 ? 1 : 0)>(tb, x, tid);
        else if (G > 2) lds<(G > 2 ? 2 : 0)>(tb, x, tid);
    }
    // In place: each array has its own region of the tile buffer.  A thread
    // rewrites exactly the slots it last read in layout `from`, so only the
    // barrier between the writes and the reads of layout `to` is needed.
    __device__ static __forceinline__ void transpose(int from, int to, C2* buf, C2 (&v)[NA][NS], uint32_t tid) {
#pragma unroll
        for (int a = 0; a < NA; ++a) sts_any(from, buf + ((size_t)a << K), v[a], tid);
        __syncthreads();
#pragma unroll
        for (int a = 0; a < NA; ++a) lds_any(to, buf + ((size_t)a << K), v[a], tid);
    }

    // ---- rotations ---------------------------------------------------------
    // Butterfly on register bit b:  a' = a + w (-i b),  b' = b + w (-i a).
    // Adjoint (NA = 2): before it, gacc += fpow * Im(conj(lam_a) psi_b +
    // conj(lam_b) psi_a), with fpow = |f|^{2r} for the r rotations of this
    // layer already applied (the stored states carry f^{-r}).
    template <int g>
    __device__ static __forceinline__ void rotate(C2 (&v)[NA][NS], Real w, int c, Real fabs2, Real& fpow,
                                                  Real& gacc) {
        static_for<0, R>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int tb = reg_bit<g, b>();
            constexpr int rk = rank_of(K, LK, tb);
            if constexpr (rk < rot_lo<g>() || rk >= rot_hi<g>()) return;  // not rotated in this layout
            if (KIND == 1 && tb < c) return;                             // carried bit
            Real part = 0;
#pragma unroll
            for (int m = 0; m < NS; ++m) {
                if (m & (1 << b)) continue;
                const int m2 = m | (1 << b);
                if (NA == 2) {
                    const C2 pa = v[0][m], pb = v[0][m2], la = v[NA - 1][m], lb = v[NA - 1][m2];
                    Real t0 = la.x * pb.y - la.y * pb.x;
                    t0 = fma_(lb.x, pa.y, t0);
                    t0 = fma_(-lb.y, pa.x, t0);
                    part += t0;
                }
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const C2 x = v[a][m], y = v[a][m2];
                    C2 nx, ny;
                    nx.x = fma_(w, y.y, x.x);
                    nx.y = fma_(-w, y.x, x.y);
                    ny.x = fma_(w, x.y, y.x);
                    ny.y = fma_(-w, x.x, y.y);
                    v[a][m] = nx;
                    v[a][m2] = ny;
                }
            }
            if (NA == 2) {
                gacc = fma_(part, fpow, gacc);
                fpow *= fabs2;
            }
        });
    }
    // General single-spin unitaries (the x + z exponentials of Eq. AQA4): the
    // target qubit q of register bit b gets (a, b) -> (u00 a + u01 b,
    // u10 a + u11 b) with u = U[8 q ..] (row major, re / im pairs, FP64).
    template <int g>
    __device__ static __forceinline__ void rotate_su2(C2 (&v)[NA][NS], const double* __restrict__ U, const TMap& tm,
                                                      int c) {
        static_for<0, R>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int tb = reg_bit<g, b>();
            constexpr int rk = rank_of(K, LK, tb);
            if constexpr (rk < rot_lo<g>() || rk >= rot_hi<g>()) return;  // not rotated in this layout
            if (KIND == 1 && tb < c) return;                             // carried bit
            const double* u = U + 8 * tm.gbit(tb);
            const Real u0r = (Real)__ldg(u), u0i = (Real)__ldg(u + 1), u1r = (Real)__ldg(u + 2),
                       u1i = (Real)__ldg(u + 3), u2r = (Real)__ldg(u + 4), u2i = (Real)__ldg(u + 5),
                       u3r = (Real)__ldg(u + 6), u3i = (Real)__ldg(u + 7);
#pragma unroll
            for (int m = 0; m < NS; ++m) {
                if (m & (1 << b)) continue;
                const int m2 = m | (1 << b);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const C2 x = v[a][m], y = v[a][m2];
                    C2 nx, ny;
                    nx.x = fma_(u0r, x.x, fma_(-u0i, x.y, fma_(u1r, y.x, -u1i * y.y)));
                    nx.y = fma_(u0r, x.y, fma_(u0i, x.x, fma_(u1r, y.y, u1i * y.x)));
                    ny.x = fma_(u2r, x.x, fma_(-u2i, x.y, fma_(u3r, y.x, -u3i * y.y)));
                    ny.y = fma_(u2r, x.y, fma_(u2i, x.x, fma_(u3r, y.y, u3i * y.x)));
                    v[a][m] = nx;
                    v[a][m2] = ny;
                }
            }
        });
    }
    __device__ static __forceinline__ void rotate_su2_any(int g, C2 (&v)[NA][NS], const double* U, const TMap& tm,
                                                          int c) {
        if (g == 0) rotate_su2<0>(v, U, tm, c);
        else if (G > 1 && g == 1) rotate_su2<(G > 1 ? 1 : 0)>(v, U, tm, c);
        else if (G > 2) rotate_su2<(G > 2 ? 2 : 0)>(v, U, tm, c);
    }
    __device__ static __forceinline__ void rotate_any(int g, C2 (&v)[NA][NS], Real w, int c, Real fabs2, Real& fpow,
                                                      Real& gacc) {
        if (g == 0) rotate<0>(v, w, c, fabs2, fpow, gacc);
        else if (G > 1 && g == 1) rotate<(G > 1 ? 1 : 0)>(v, w, c, fabs2, fpow, gacc);
        else if (G > 2) rotate<(G > 2 ? 2 : 0)>(v, w, c, fabs2, fpow, gacc);
    }

    // ---- phase -------------------------------------------------------------
    template <int g>
    __device__ static __forceinline__ void phase(C2 (&v)[NA][NS], const SweepTask& T, const TileTab& tt,
                                                 uint32_t tid, const C2* __restrict__ tab, int frame, Real& gacc) {
        SlotCost<R> sc;
        sc.template init_tile<Map<g>, K - R>(tt, T.cprog[g], tid, frame, T.cost_lo);
        const int top = T.tab_stride - 1;
        Real part = 0;
#pragma unroll
        for (int m = 0; m < NS; ++m) {
            const int ix = sc.tidx(m, top);
            const C2 f = __ldg(tab + ix);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const C2 x = v[a][m];
                C2 y;
                y.x = fma_(x.x, f.x, -x.y * f.y);
                y.y = fma_(x.x, f.y, x.y * f.x);
                v[a][m] = y;
            }
            if (NA == 2) {
                const Real im = v[NA - 1][m].x * v[0][m].y - v[NA - 1][m].y * v[0][m].x;
                part = fma_((Real)(ix + T.cost_lo), im, part);
            }
        }
        gacc += part;
    }

    // ---- spin expectations (single array) -------------------------------------
    template <int g>
    __device__ static __forceinline__ void zexp(const C2 (&v)[NA][NS], uint32_t tid, Real* zred, double* zacc,
                                                const TMap& tm, uint64_t zb, int nq, int sg) {
        Real w[NS], zv[K + 1];
#pragma unroll
        for (int m = 0; m < NS; ++m) w[m] = fma_(v[0][m].x, v[0][m].x, v[0][m].y * v[0][m].y);
        z_thread_sums<Map<g>, K, R>(w, tid, zv);
        z_tile_add<K, NW>(zv, zred, zacc, tm, zb, nq, sg, tid);
    }
    __device__ static __forceinline__ void zexp_any(int g, const C2 (&v)[NA][NS], uint32_t tid, Real* zred,
                                                    double* zacc, const TMap& tm, uint64_t zb, int nq, int sg) {
        if (g == 0) zexp<0>(v, tid, zred, zacc, tm, zb, nq, sg);
        else if (G > 1 && g == 1) zexp<(G > 1 ? 1 : 0)>(v, tid, zred, zacc, tm, zb, nq, sg);
        else if (G > 2) zexp<(G > 2 ? 2 : 0)>(v, tid, zred, zacc, tm, zb, nq, sg);
    }

    // global offset of the thread part of layout g
    template <int g>
    __device__ static __forceinline__ uint64_t zthread(uint64_t base, uint32_t tid, const TMap& tm) {
        const uint32_t e = e_thread<g>(tid);
        return base + (KIND == 0 ? (uint64_t)e : tm.gofs(e));
    }
    __device__ static __forceinline__ void phase_any(int g, C2 (&v)[NA][NS], const SweepTask& T, const TileTab& tt,
                                                     uint32_t tid, const C2* tab, int frame, Real& gacc) {
        if (g == 0) phase<0>(v, T, tt, tid, tab, frame, gacc);
        else if (G > 1 && g == 1) phase<(G > 1 ? 1 : 0)>(v, T, tt, tid, tab, frame, gacc);
        else if (G > 2) phase<(G > 2 ? 2 : 0)>(v, T, tt, tid, tab, frame, gacc);
    }

    // ---- layout-0 global offsets of the register slots ----------------------
    // kind 0: compile-time; kind 1: layout 0's registers are the top R tile
    // bits.  When they all lie in the last target run (every large shape)
    // the offset is one shift; otherwise the general map.
    template <class F>
    __device__ static __forceinline__ void for_slots(const TMap& tm, F&& f) {
        if (KIND == 0) {
#pragma unroll
            for (int m = 0; m < NS; ++m) f(m, (uint64_t)e_slot<0>(m));
        } else if (KIND == 2) {
            // runs of 2^kRunBits: layout 0's registers are tile bits
            // [K - 1 - R, K - 1); the cl of them inside the run stay in place,
            // the others lie on run 1 (consecutive global bits from g0)
            constexpr int lo = K - 1 - R, cl = kRunBits - lo;
            static_assert(cl >= 0 && cl <= R, "layout-0 registers straddle the run boundary");
            const uint64_t stride = 1ull << tm.g0;
            uint64_t hi = 0;
#pragma unroll
            for (int h = 0; h < (NS >> cl); ++h) {
#pragma unroll
                for (int l = 0; l < (1 << cl); ++l) f((h << cl) | l, hi + ((uint64_t)l << lo));
                hi += stride;
            }
        } else {
            constexpr int lo = K - R;  // regs of layout 0 are tile bits [K - R, K)
            if (tm.c + tm.n1 <= lo) {
                const int sh = tm.g1 + lo - tm.c - tm.n1;
#pragma unroll
                for (int m = 0; m < NS; ++m) f(m, (uint64_t)m << sh);
            } else {
#pragma unroll
                for (int m = 0; m < NS; ++m) f(m, tm.gofs((uint32_t)m << lo));
            }
        }
    }
};

template <class Real, int K, int R, int NA, int KIND, int V>
__global__ void __launch_bounds__(1 << (K - R), NA == 1 ? 2 : 1)
    sweep_kernel(const SweepTask* __restrict__ tasks, const int64_t* __restrict__ prefix, int ntasks, int64_t total,
                 int* __restrict__ err, int qlog) {
    using S = Sweep<Real, K, R, NA, KIND>;
    using C2 = typename S::C2;
    constexpr int NS = S::NS, NW = S::NW, NSLOT = S::NSLOT;
    constexpr bool kZ = V == V_ZFULL && NA == 1;
    constexpr bool kSU2 = V == V_SU2 && NA == 1;  // general single-spin unitaries instead of x rotations
    constexpr bool kGen = V == V_FULL || kZ || kSU2, kPhase = V != V_LEAN, kRead = V == V_FULL || kZ || kSU2;
    static_assert(KIND != 1 || make_layout(K, R, KIND).regs[0][0] == K - R, "layout 0 holds the top R tile bits");
    extern __shared__ __align__(128) unsigned char smraw[];
    C2* buf = reinterpret_cast<C2*>(smraw);                                      // [NA][2^K]
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw + S::BUF_BYTES);
    double* red = reinterpret_cast<double*>(smraw + S::BUF_BYTES + 64);
    TileTab* ttab = reinterpret_cast<TileTab*>(smraw + S::TT_OFF);  // [2]: by tile parity
    double* zacc = reinterpret_cast<double*>(smraw + S::SMEM_BYTES);   // kZ: [kZSlots][kZQ]
    Real* zred = reinterpret_cast<Real*>(smraw + S::SMEM_BYTES + (size_t)kZSlots * kZQ * 8);
    const uint32_t tid = threadIdx.x;
    C2 v[NA][NS];
    const bool zon = kZ && (tasks[0].flags & T_ZEXP);  // one task per launch

    auto find_task = [&](int64_t gt) -> int {
        if (ntasks == 1) return 0;
        int lo = 0, hi = ntasks - 1;  // last task whose prefix <= gt
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(prefix + mid) <= gt) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    bool pending = false;
    // Called by every thread; every thread arrives once on the barrier.
    // Contiguous tiles: thread 0 issues one TMA bulk copy per array.  Strided
    // and run-structured tiles: every thread issues 16-byte cp.async copies,
    // completing on the same barrier.
    auto issue = [&](int64_t gt) {
        const int ti = find_task(gt);
        const SweepTask& T = tasks[ti];
        if (kGen && (T.flags & T_GEN)) return;  // generated, nothing to load
        const int64_t tile = gt - __ldg(prefix + ti);
        if (KIND == 1) {
            constexpr int EPC = 16 / (int)sizeof(C2);                  // elements per 16-byte copy
            constexpr int CHUNKS = (1 << K) / EPC;
            const TMap tm{T.c, T.g0, T.n1, T.g1, K};
            const uint64_t base = tm.base(tile);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const C2* src = reinterpret_cast<const C2*>(a == 0 ? T.psi : T.lam) + base;
                C2* dst = buf + ((size_t)a << K);
                for (int q = tid; q < CHUNKS; q += S::NT) {
                    const uint32_t e = (uint32_t)q * EPC;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + e)),
                                 "l"(src + tm.gofs(e))
                                 : "memory");
                }
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(full)) : "memory");
            pending = true;
            return;
        }
        // kind 0 / 2: thread 0 arrives with the byte count, every other thread
        // arrives plainly.  Kind 0 (contiguous): one bulk copy per array by
        // thread 0.  Kind 2 (runs of 2^c): one bulk copy per run and array by
        // warp 0, after thread 0's byte count.
        if (tid == 0) mbar_expect_tx(full, (uint32_t)S::BUF_BYTES);
        else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(full)) : "memory");
        if (KIND == 0) {
            if (tid == 0) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const C2* src = reinterpret_cast<const C2*>(a == 0 ? T.psi : T.lam) + ((uint64_t)tile << K);
                    tma_load_1d(buf + ((size_t)a << K), src, (uint32_t)S::TILE_BYTES, full);
                }
            }
        } else if (tid < 32) {
            __syncwarp();
            const TMap tm{T.c, T.g0, T.n1, T.g1, K};
            // runs of 2^kRunBits with the batch bit above them and run 1 on the
            // top global bits: the tile index fills the bits in between
            const uint64_t base = (uint64_t)tile << (kRunBits + 1);
            constexpr uint32_t run = 1u << kRunBits;  // amplitudes per run (>= 16 bytes, aligned)
            for (uint32_t e0 = tid * run; e0 < (1u << K); e0 += 32 * run)
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const C2* src = reinterpret_cast<const C2*>(a == 0 ? T.psi : T.lam) + base + tm.gofs(e0);
                    tma_load_1d(buf + ((size_t)a << K) + e0, src, run * (uint32_t)sizeof(C2), full);
                }
        }
        pending = true;
    };

    if (tid == 0) {
        mbar_init(full, S::NT);  // one arrival per thread (with its copies, or with the byte count)
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (zon)
        for (int i = (int)tid; i < kZSlots * kZQ; i += S::NT) zacc[i] = 0.0;
    __syncthreads();
    // The CTA's k-th tile: groups of 2^qlog consecutive tiles (which share
    // HBM lines when rows are short) run back to back on one CTA.
    const int64_t qmask = (1ll << qlog) - 1;
    auto tile_at = [&](int64_t k) -> int64_t {
        return (((int64_t)blockIdx.x + (k >> qlog) * gridDim.x) << qlog) + (k & qmask);
    };
    if (tile_at(0) < total) issue(tile_at(0));

    uint32_t parity = 0;
    for (int64_t k = 0;; ++k) {
        const int64_t gt = tile_at(k);
        if (gt >= total) break;
        const int ti = find_task(gt);
        const SweepTask& T = tasks[ti];
        const int64_t tile = gt - __ldg(prefix + ti);
        const int c = T.c, flags = T.flags, nr = T.nrounds;
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        const uint64_t base = KIND == 0   ? ((uint64_t)tile << K)
                              : KIND == 2 ? ((uint64_t)tile << (kRunBits + 1))
                                          : tm.base(tile);
        // layouts that hold targets (kind 1 drops those entirely below c)
        int ga = S::G;
        if (KIND == 1) {
            ga = 1;
            if (S::G > 1 && K - 1 - S::template rot_lo<(1 < S::G ? 1 : 0)>() >= c) ga = 2;
            if (S::G > 2 && K - 1 - S::template rot_lo<(2 < S::G ? 2 : 0)>() >= c) ga = 3;
        }
        const bool gen = kGen && (flags & T_GEN);
        const int start = (gen && (nr & 1) && ga > 1) ? ga - 1 : 0;
        // transposes of this tile: ga - 1 per round, + 1 back to layout 0
        const int endl = ga == 1 ? 0 : ((start == 0) == ((nr & 1) == 0) ? 0 : ga - 1);
        const int ntr = nr * (ga - 1) + (endl != 0 ? 1 : 0);
        int done_tr = 0;
        const int64_t nx = tile_at(k + 1);
        // after the tile's last shared-memory read: reload the buffer
        auto release = [&]() {
            __syncthreads();
            if (nx < total) {
                if ((KIND == 0 && tid == 0) || (KIND == 2 && tid < 32)) fence_proxy_async();  // bulk-copy issuers
                issue(nx);
            }
        };
        const uint64_t g_thread = S::template zthread<0>(base, tid, tm);
        C2* arr[2] = {reinterpret_cast<C2*>(T.psi), reinterpret_cast<C2*>(T.lam)};
        // the tile's cost table: warp 0, published by the barrier below (the
        // other table of the pair may still be read for the previous tile)
        const TileTab& tt = ttab[k & 1];
        if ((kPhase || kRead) && tid < 32) tile_tab_fill(&ttab[k & 1], T.tprog, base, tid);

        int cur = start;
        if (gen) {
            __syncthreads();  // the previous tile's reads of the buffer are done
            const Real a0 = (Real)T.amp0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int m = 0; m < NS; ++m) v[a][m] = C2{a0, (Real)0};
            if (ntr == 0 && nx < total) issue(nx);
        } else {
            const int ok = mbar_wait_bounded(full, parity) ? 1 : 0;
            if (!__syncthreads_and(ok)) {  // the copies stay pending on this phase
                if (tid == 0) atomicExch(err, 1);
                break;
            }
            parity ^= 1u;
            if (tid == 0) pending = false;
#pragma unroll
            for (int a = 0; a < NA; ++a) S::template lds_dense<0>(buf + ((size_t)a << K), v[a], tid);
            if (ntr == 0) release();
            else __syncthreads();  // dense reads done before the swizzled writes
        }
        auto transpose = [&](int from, int to) {
            S::transpose(from, to, buf, v, tid);
            if (++done_tr == ntr) release();
        };

        const C2* tab = reinterpret_cast<const C2*>(T.tab);
        for (int r = 0; r < nr; ++r) {
            const SweepRound rd = T.rounds[r];
            const LayerDev ly = T.layers[rd.layer];
            Real gB = 0, gG = 0;
            const C2* ltab = tab + (int64_t)rd.layer * T.tab_stride;
            // the state after the previous layer (normalised: the scalars of a
            // layer's rotations sit in its own phase table)
            if (zon && rd.phase_pre && rd.layer > 0)
                S::zexp_any(cur, v, tid, zred, zacc + r * kZQ, tm, base, T.n, ly.frame ? -1 : 1);
            if (kPhase && rd.phase_pre) S::phase_any(cur, v, T, tt, tid, ltab, ly.frame, gG);
            const Real fabs2 = (Real)(ly.fabs * ly.fabs);
            Real fpow = 1;
            if (NA == 2)
                for (int i = 0; i < rd.r0; ++i) fpow *= fabs2;  // |f|^{2 r0}, no FP64 on the device
            const Real w = (Real)ly.w;
            const double* U = kSU2 ? T.su2 + (size_t)rd.layer * T.n * 8 : nullptr;
            if (cur == 0) {
                for (int g = 0; g < ga; ++g) {
                    if (g != cur) { transpose(cur, g); cur = g; }
                    if (kSU2) S::rotate_su2_any(g, v, U, tm, c);
                    else S::rotate_any(g, v, w, c, fabs2, fpow, gB);
                }
            } else {
                for (int g = ga - 1; g >= 0; --g) {
                    if (g != cur) { transpose(cur, g); cur = g; }
                    if (kSU2) S::rotate_su2_any(g, v, U, tm, c);
                    else S::rotate_any(g, v, w, c, fabs2, fpow, gB);
                }
            }
            if (kPhase && rd.phase_post) S::phase_any(cur, v, T, tt, tid, ltab, ly.frame, gG);
            if (NA == 2) {
                warp_sum_to((double)gB, red, 2 * r, NSLOT);
                warp_sum_to((double)gG, red, 2 * r + 1, NSLOT);
            }
        }
        if (cur != 0) { transpose(cur, 0); cur = 0; }

        if (zon && (flags & T_READOUT))
            S::template zexp<0>(v, tid, zred, zacc + kMaxRounds * kZQ, tm, base, T.n,
                                T.layers[T.end_layer].frame ? -1 : 1);
        if (kRead && (flags & (T_READOUT | T_WRITE_LAM))) {
            const int ef = T.layers[T.end_layer].frame;
            SlotCost<R> sc;
            sc.template init_tile<typename S::template Map<0>, K - R>(tt, T.cprog[0], tid, ef, T.cost_lo);
            Real E = 0, P = 0, N = 0;
            C2* lam = arr[1] + g_thread;
            const bool wl = (flags & T_WRITE_LAM) != 0;
            S::for_slots(tm, [&](int m, uint64_t off) {
                const C2 x = v[0][m];
                const int ix = sc.idx(m);
                const Real w2 = x.x * x.x + x.y * x.y;
                const Real cst = (Real)(ix + T.cost_lo);
                E = fma_(w2, cst, E);
                N += w2;
                const bool gnd = (ix == T.gidx);
                if (gnd) P += w2;
                if (wl) {
                    const Real o = (T.objective == 0) ? cst : (gnd ? (Real)1 : (Real)0);
                    lam[off] = C2{o * x.x, o * x.y};
                }
            });
            if (flags & T_READOUT) {
                warp_sum_to((double)E, red, 0, NSLOT);
                warp_sum_to((double)P, red, 1, NSLOT);
                warp_sum_to((double)N, red, 2, NSLOT);
            }
        }
        if (flags & T_STORE) {
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                C2* dst = arr[a] + g_thread;
                S::for_slots(tm, [&](int m, uint64_t off) { dst[off] = v[a][m]; });
            }
        }
        if ((kRead || NA == 2) && T.np > 0) {
            const int np = T.np;
            __syncthreads();
            if (tid < (uint32_t)np) {
                double s = 0.0;
                for (int w = 0; w < NW; ++w) s += red[w * NSLOT + tid];
                T.partials[(T.part_base + tile) * np + tid] = s;
            }
            __syncthreads();
        }
    }
    // On a timeout, wait (bounded) for a copy still in flight before the CTA's
    // shared memory goes away; if that wait also gives up, a copy may still
    // land in shared memory the SM hands to a later CTA: report it with the
    // sticky status 2 (the host then refuses to use the handle again).
    if (tid == 0 && pending && !mbar_wait_bounded(full, parity)) atomicMax(err, 2);
    if (zon) {
        __syncthreads();
        double* zp = tasks[0].zpart + (size_t)blockIdx.x * (kZSlots * kZQ);
        for (int i = (int)tid; i < kZSlots * kZQ; i += S::NT) zp[i] = zacc[i];
    }
}

template <class Real, int K, int R, int NA, int KIND, int V>
constexpr size_t sweep_smem() {
    using S = Sweep<Real, K, R, NA, KIND>;
    return S::SMEM_BYTES + (V == V_ZFULL ? S::Z_BYTES : 0);
}

template <class Real, int K, int R, int NA, int KIND, int V>
cudaError_t launch_sweep_cfg(const SweepLaunch& L, int grid, cudaStream_t st) {
    using S = Sweep<Real, K, R, NA, KIND>;
    auto kern = sweep_kernel<Real, K, R, NA, KIND, V>;
    constexpr size_t smem = sweep_smem<Real, K, R, NA, KIND, V>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int qlog = 0;
    while ((1 << (qlog + 1)) <= L.group) ++qlog;
    kern<<<grid, S::NT, smem, st>>>(L.tasks, L.tile_prefix, L.ntasks, L.total_tiles, L.err, qlog);
    return note_launch(cudaGetLastError());
}

template <class Real, int K, int R, int NA, int KIND, int V>
int grid_cfg() {
    using S = Sweep<Real, K, R, NA, KIND>;
    auto kern = sweep_kernel<Real, K, R, NA, KIND, V>;
    constexpr size_t smem = sweep_smem<Real, K, R, NA, KIND, V>();
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::NT, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

}  // namespace qs
