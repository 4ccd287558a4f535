// Packed-pair sweep: the strided complex64 forward sweeps (rotations only, or
// rotations with a layer boundary and its phase), layouts in qs_pair.h.
//
// Same tile walk as sweep_kernel (qs_sweep.cuh): persistent CTAs, three per SM
// (registers bounded to 168 per thread), each with one in-place 64 KB tile
// buffer, 16-byte cp.async copies of the strided tile
// completing on an mbarrier (bounded wait), the next tile's copies issued
// after the current tile's last shared-memory read.  The difference is the
// register format: pairs split by component and updated with packed f32x2
// FMAs (fma.rn.f32x2), transposes as 16-byte pair moves.
#include <cstring>

#include "qs_pair.h"
#include "qs_sweep.cuh"

namespace qs {

namespace {

// a * b + c on both halves: one packed f32x2 FMA (fma.rn.f32x2)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// A zero the compiler cannot see through: XORed into the per-thread shared
// memory base of a transpose so that the 16-32 slot addresses are formed at
// the access (one LOP3 each) instead of being hoisted out of the tile loop
// and held in registers for the whole kernel.
// Landing-buffer position of tile element e: the pack bit P flipped with
// tile bits 4 and 8 (and, for P = 2, bit 3 with tile bit 9).  A tile is read
// from the landing buffer into layout 0 or layout 1; the 8-byte reads of
// either (half-warp lanes on tile bits 0, 1 and 3, 4 or 9, 8 when P = 2;
// 0, 1, 2 and 4 or 8 when P = 3) then hit 16 distinct bank pairs, and a
// 16-byte copy (elements e, e + 1) stays whole because bit 0 is kept.
template <int P>
__device__ __forceinline__ uint32_t land(uint32_t e) {
    const uint32_t f = ((e >> 4) ^ (e >> 8)) & 1u;
    return P == 2 ? e ^ (f << 2) ^ (((e >> 9) & 1u) << 3) : e ^ (f << P);
}

__device__ __forceinline__ uint32_t opaque_zero() {
    uint32_t z;
    asm volatile("mov.u32 %0, 0;" : "=r"(z));
    return z;
}

// One 8-byte store of an amplitude whose parts sit in different pairs.  Two
// 4-byte stores would leave each 32-byte sector half written in between,
// which costs DRAM reads; the vector store writes whole sectors.
__device__ __forceinline__ void stg2(float2* p, float re, float im) {
    asm volatile("st.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(re), "f"(im) : "memory");
}

template <int C>
struct PairSweep {
    static constexpr int K = kPairK, NT = 128, NJ = 32, P = C;
    static constexpr int NB = 1;  // tile buffers per CTA
    static constexpr size_t BUF_BYTES = (size_t)8 << K;
    static constexpr size_t TT_OFF = NB * BUF_BYTES + 64;  // two TileTabs (by tile parity)
    static constexpr size_t KOFF_OFF = TT_OFF + 2 * sizeof(TileTab);  // 32 tile-copy offsets (uint64)
    // the launch's task and its rounds' layer parameters, copied once per CTA
    static constexpr size_t TASK_OFF = (KOFF_OFF + 32 * sizeof(uint64_t) + 15) & ~(size_t)15;
    static constexpr size_t LAY_OFF = (TASK_OFF + sizeof(SweepTask) + 15) & ~(size_t)15;
    static constexpr size_t SMEM_BYTES = LAY_OFF + kMaxRounds * sizeof(LayerDev);
    // V_ZPHASE: FP64 spin-expectation accumulators [kZSlots][kZQ], then the warp sums
    static constexpr size_t Z_BYTES = (size_t)kZSlots * kZQ * 8 + (size_t)(NT / 32) * (K + 1) * 4;
    static_assert(SMEM_BYTES % 8 == 0, "accumulators follow the tile tables");
    // compile-time tile bits of layout g: slot bit 0 is the pack bit
    template <int g> struct Map {
        __host__ __device__ static constexpr int slot(int b) { return b == 0 ? P : pair_layout(C).regs[g][b - 1]; }
        __host__ __device__ static constexpr int thr(int j) { return pair_layout(C).tbits[g][j]; }
    };

    template <int g, int t> __host__ __device__ static constexpr int tb() { return pair_layout(C).tbits[g][t]; }
    template <int g, int b> __host__ __device__ static constexpr int rb() { return pair_layout(C).regs[g][b]; }
    template <int g> __host__ __device__ static constexpr int rmask() { return pair_layout(C).rotmask[g]; }

    template <int g>
    __device__ static __forceinline__ uint32_t e_thread(uint32_t tid) {
        uint32_t e = 0;
        static_for<0, 7>([&](auto tc) {
            constexpr int t = decltype(tc)::value;
            e |= ((tid >> t) & 1u) << tb<g, t>();
        });
        return e;
    }
    template <int g>
    __host__ __device__ static constexpr uint32_t e_slot(int j) {
        uint32_t e = 0;
        for (int b = 0; b < 5; ++b) e |= (uint32_t)((j >> b) & 1) << pair_layout(C).regs[g][b];
        return e;
    }

    // ---- transposes (16-byte pair units, swizzled) ---------------------------
    template <int g>
    __device__ static __forceinline__ void sts(float4* tb4, const float2 (&X)[NJ], const float2 (&Y)[NJ],
                                               uint32_t tid) {
        const uint32_t pt = pair_phys(pair_unit(e_thread<g>(tid), P)) ^ opaque_zero();
#pragma unroll
        for (int j = 0; j < NJ; ++j)
            tb4[pt ^ pair_phys(pair_unit(e_slot<g>(j), P))] = make_float4(X[j].x, X[j].y, Y[j].x, Y[j].y);
    }
    template <int g>
    __device__ static __forceinline__ void lds(const float4* tb4, float2 (&X)[NJ], float2 (&Y)[NJ], uint32_t tid) {
        const uint32_t pt = pair_phys(pair_unit(e_thread<g>(tid), P)) ^ opaque_zero();
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const float4 v = tb4[pt ^ pair_phys(pair_unit(e_slot<g>(j), P))];
            X[j] = make_float2(v.x, v.y);
            Y[j] = make_float2(v.z, v.w);
        }
    }
    // from the landing buffer (tile order, one float2 per amplitude) into layout g
    template <int g>
    __device__ static __forceinline__ void lds_dense(const float2* src, float2 (&X)[NJ], float2 (&Y)[NJ],
                                                     uint32_t tid) {
        const uint32_t et = e_thread<g>(tid);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const float2 a = src[land<P>(et | e_slot<g>(j))];
            const float2 b = src[land<P>(et | e_slot<g>(j) | (1u << P))];
            X[j] = make_float2(a.x, b.x);
            Y[j] = make_float2(a.y, b.y);
        }
    }

    // from a tile landed by the two tensor-map copies (pair_tma_land order
    // for layout g) into layout g; the landing map is linear over XOR, so the
    // thread's part is formed once and each slot's part is a constant
    template <int g>
    __device__ static __forceinline__ void lds_tma(const float2* src, float2 (&X)[NJ], float2 (&Y)[NJ],
                                                   uint32_t tid) {
        uint32_t lt = 0;
        static_for<0, 7>([&](auto tc) {
            constexpr int t = decltype(tc)::value;
            constexpr uint32_t l = pair_tma_land(C, g, 1u << tb<g, t>());
            lt ^= ((tid >> t) & 1u) ? l : 0u;
        });
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const float2 a = src[lt ^ pair_tma_land(C, g, e_slot<g>(j))];
            const float2 b = src[lt ^ pair_tma_land(C, g, e_slot<g>(j) | (1u << P))];
            X[j] = make_float2(a.x, b.x);
            Y[j] = make_float2(a.y, b.y);
        }
    }

    // ---- rotations: a' = a + w (-i b), b' = b + w (-i a) ----------------------
    template <int g>
    __device__ static __forceinline__ void rotate(float2 (&X)[NJ], float2 (&Y)[NJ], float w) {
        const float2 w2 = make_float2(w, w), nw2 = make_float2(-w, -w);
        static_for<0, 5>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            if constexpr (((rmask<g>() >> b) & 1) != 0) {
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    if (j & (1 << b)) continue;
                    const int j2 = j | (1 << b);
                    const float2 xa = X[j], ya = Y[j], xb = X[j2], yb = Y[j2];
                    X[j] = ffma2(w2, yb, xa);
                    Y[j] = ffma2(nw2, xb, ya);
                    X[j2] = ffma2(w2, ya, xb);
                    Y[j2] = ffma2(nw2, xa, yb);
                }
            }
        });
        if (g == 0) {  // the pack bit: the two halves of every pair
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const float ar = X[j].x, br = X[j].y, ai = Y[j].x, bi = Y[j].y;
                X[j] = make_float2(fmaf(w, bi, ar), fmaf(w, ai, br));
                Y[j] = make_float2(fmaf(-w, br, ai), fmaf(-w, ar, bi));
            }
        }
    }

    // ---- <Z_q> of the tile in layout g: slot m = half | j << 1 ------------------
    template <int g>
    __device__ static __forceinline__ void zexp(const float2 (&X)[NJ], const float2 (&Y)[NJ], uint32_t tid,
                                                float* zred, double* zacc, const TMap& tm, uint64_t zb, int nq,
                                                int sg) {
        float w[2 * NJ], zv[K + 1];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            w[2 * j] = fmaf(X[j].x, X[j].x, Y[j].x * Y[j].x);
            w[2 * j + 1] = fmaf(X[j].y, X[j].y, Y[j].y * Y[j].y);
        }
        z_thread_sums<Map<g>, K, 6>(w, tid, zv);
        z_tile_add<K, NT / 32>(zv, zred, zacc, tm, zb, nq, sg, tid);
    }

    // ---- phase: slot m = lane | j << 1 (cost program of the layout) ------------
    // Q[m] comes from the kernel parameters; the layer's table (a generic
    // pointer) lies in shared memory when it was staged at kernel start, else
    // in global memory.
    template <int g>
    __device__ static __forceinline__ void phase(float2 (&X)[NJ], float2 (&Y)[NJ], const SweepTask& T,
                                                 const TileTab& tt, uint32_t tid, const float2* __restrict__ tab,
                                                 int frame, const PairQ& pq) {
        pair_phase<Map<g>, 7>(X, Y, T.cprog[g], tt, tid, frame, T.cost_lo, tab, T.tab_stride - 1, pq.q[g]);
    }
};

}  // namespace

// The two tensor-map copies of the tile whose base index (tile bits clear)
// is base into dst (one per value of the pack bit, 2^12 amplitudes each),
// completion on the barrier.  Coordinates: per dimension the index bits it
// spans; dimension 0 counts floats.
__device__ __forceinline__ void tma_load_tile(unsigned char* dst, const PairLoad& tm, uint64_t base, uint64_t* bar) {
    const uint64_t mp = reinterpret_cast<uint64_t>(&tm.map);
    const uint32_t mb = smem_u32(bar);
    const int rank = tm.rank;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const uint64_t bk = base | ((uint64_t)k << tm.kbit);
        const uint32_t d = smem_u32(dst + (size_t)k * 32768);
        const int c0 = 2 * (int)((bk >> tm.lo[0]) & ((1ull << tm.nb[0]) - 1ull));
        const int c1 = (int)((bk >> tm.lo[1]) & ((1ull << tm.nb[1]) - 1ull));
        const int c2 = (int)((bk >> tm.lo[2]) & ((1ull << tm.nb[2]) - 1ull));
        if (rank == 3) {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                "%3, %4}], [%5];" ::"r"(d),
                "l"(mp), "r"(c0), "r"(c1), "r"(c2), "r"(mb)
                : "memory");
            continue;
        }
        const int c3 = (int)((bk >> tm.lo[3]) & ((1ull << tm.nb[3]) - 1ull));
        if (rank == 4) {
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                "%3, %4, %5}], [%6];" ::"r"(d),
                "l"(mp), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mb)
                : "memory");
            continue;
        }
        const int c4 = (int)((bk >> tm.lo[4]) & ((1ull << tm.nb[4]) - 1ull));
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4, %5, %6}], [%7];" ::"r"(d),
            "l"(mp), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mb)
            : "memory");
    }
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Three CTAs per SM, each with NB = 1 in-place tile buffer: after tile k's
// last shared-memory read the buffer takes tile k + 1 (NB > 1 would keep
// more tiles in flight per CTA, at one CTA per SM; measured slower).
//
// CL = 4: clusters of four CTAs take the four tiles that differ in tile-index
// bits 0 and 1 (the neighbouring runs of one 128-byte line when c = 2) and
// issue their copies together, after a cluster barrier, so the HBM lines they
// share are fetched once.  Every CTA of a cluster walks the same number of
// tiles (the tile count and the grid are multiples of four) and passes the
// barrier once per tile, also after a timed-out wait.
// CTAs per SM: three (168 registers a thread); QS_PHASE_OCC sets it for the
// sweeps that apply a phase (2: 255 registers, no spills, 8 warps per SM).
#ifndef QS_PHASE_OCC
#define QS_PHASE_OCC 3
#endif
template <int V> struct PairOcc { static constexpr int value = (V == V_PHASE || V == V_ZPHASE) ? QS_PHASE_OCC : 3; };

// V_PHASE stages the layer table of its phase in shared memory when it has at
// most this many entries (the three CTAs of an SM still fit).
constexpr int kPairTabSmem = 1024;

// TM: the tile arrives as two tensor-map copies issued by thread 0 (one per
// value of the pack bit, in the landing order of the layout the tile is
// first read into; one launch = one task, the map of its state buffer in
// ld) instead of per-thread 16-byte cp.async copies.  The buffer is placed
// on a 1024-byte boundary (1 KB of slack in the dynamic shared memory).
template <int C, int V, int CL, bool TM>
__global__ void __launch_bounds__(128, PairOcc<V>::value)
    sweep_pair_kernel(const SweepTask* __restrict__ tasks, const int64_t* __restrict__ prefix, int ntasks,
                      int64_t total, int* __restrict__ err, const __grid_constant__ PairQ pq,
                      const __grid_constant__ PairLoad ld) {
    using S = PairSweep<C>;
    constexpr int K = S::K, NT = S::NT, NJ = S::NJ, P = S::P, NB = S::NB;
    constexpr bool kPhase = V != V_LEAN, kZ = V == V_ZPHASE, kSTab = V == V_PHASE;
    extern __shared__ __align__(128) unsigned char smdyn[];
    unsigned char* smraw = TM ? smdyn + ((1024u - (smem_u32(smdyn) & 1023u)) & 1023u) : smdyn;
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw + NB * S::BUF_BYTES);  // one barrier per buffer
    TileTab* ttab = reinterpret_cast<TileTab*>(smraw + S::TT_OFF);
    uint64_t* koff = reinterpret_cast<uint64_t*>(smraw + S::KOFF_OFF);
    // one task per launch (checked on the host): read from shared memory,
    // so the per-tile and per-round fields are short-latency loads
    const SweepTask& T = *reinterpret_cast<const SweepTask*>(smraw + S::TASK_OFF);
    LayerDev* slay = reinterpret_cast<LayerDev*>(smraw + S::LAY_OFF);
    double* zacc = reinterpret_cast<double*>(smraw + S::SMEM_BYTES);  // kZ: [kZSlots][kZQ]
    float* zred = reinterpret_cast<float*>(smraw + S::SMEM_BYTES + (size_t)kZSlots * kZQ * 8);
    float2* stab = reinterpret_cast<float2*>(smraw + S::SMEM_BYTES);  // kSTab: [kPairTabSmem]
    const uint32_t tid = threadIdx.x;
    const bool zon = kZ && (tasks[0].flags & T_ZEXP);
    uint32_t tpar = 0;  // parity of the CTA's tile count: which TileTab
    float2 X[NJ], Y[NJ];

    uint32_t pend = 0;   // buffers with copies in flight
    uint32_t phase = 0;  // per buffer: parity of its next completion
    // every thread: 16-byte cp.async copies of its share of the strided tile
    // gt into buffer b, completing on that buffer's barrier (one arrival per
    // thread)
    auto issue = [&](int64_t gt, int b) {
        if constexpr (TM) {
            if (tid == 0) {
                const TMap tm{T.c, T.g0, T.n1, T.g1, K};
                fence_proxy_async();  // the buffer's generic accesses before the async writes
                mbar_expect_tx(full + b, (uint32_t)S::BUF_BYTES);
                tma_load_tile(smraw + b * S::BUF_BYTES, ld, tm.base(gt), full + b);
            }
            pend |= 1u << b;
            return;
        }
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        // thread t copies elements e = 2t + 256k, k < 32: the landing map and
        // the global offset split into a per-thread part and the k part
        // (koff[k] = gofs(256 k), the same for every tile of the launch)
        const uint32_t e_t = 2u * tid;
        const float2* src = reinterpret_cast<const float2*>(T.psi) + tm.base(gt) + tm.gofs(e_t);
        const uint32_t sb = smem_u32(smraw + b * S::BUF_BYTES), lt = land<P>(e_t);
#pragma unroll
        for (int k = 0; k < 32; ++k)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + 8u * (lt ^ land<P>(256u * k))),
                         "l"(src + koff[k])
                         : "memory");
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(full + b)) : "memory");
        pend |= 1u << b;
    };

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(full + b, TM ? 1 : NT);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const int* src = reinterpret_cast<const int*>(tasks);
        int* dst = reinterpret_cast<int*>(smraw + S::TASK_OFF);
        for (int i = (int)tid; i < (int)(sizeof(SweepTask) / 4); i += NT) dst[i] = __ldg(src + i);
        const SweepTask& T0 = tasks[0];
        if ((int)tid < T0.nrounds) slay[tid] = T0.layers[T0.rounds[tid].layer];
        if (!TM && tid < 32) koff[tid] = TMap{T0.c, T0.g0, T0.n1, T0.g1, K}.gofs(256u * tid);
    }
    if (zon)
        for (int i = (int)tid; i < kZSlots * kZQ; i += NT) zacc[i] = 0.0;
    // the table of the (first) layer whose phase this sweep applies
    int slayer = -1;
    if (kSTab && ntasks == 1 && tasks[0].tab_stride <= kPairTabSmem) {
        const SweepTask& T0 = tasks[0];
        for (int r = 0; r < T0.nrounds; ++r)
            if (T0.rounds[r].phase_pre) {
                slayer = T0.rounds[r].layer;
                break;
            }
        if (slayer >= 0) {
            const float2* src = reinterpret_cast<const float2*>(T0.tab) + (int64_t)slayer * T0.tab_stride;
            for (int i = (int)tid; i < T0.tab_stride; i += NT) stab[i] = __ldg(src + i);
        }
    }
    __syncthreads();
    for (int b = 0; b < NB; ++b) {
        const int64_t g0 = (int64_t)blockIdx.x + (int64_t)b * gridDim.x;
        if (g0 < total) issue(g0, b);
    }

    bool failed = false;
    int b = 0;  // buffer of the current tile
    for (int64_t gt = blockIdx.x; gt < total; gt += gridDim.x, b = (b + 1 == NB ? 0 : b + 1)) {
        const int flags = T.flags, nr = T.nrounds;
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        const uint64_t base = tm.base(gt);
        const int64_t nx = gt + (int64_t)NB * gridDim.x;
        float2* buf = reinterpret_cast<float2*>(smraw + b * S::BUF_BYTES);
        float4* buf4 = reinterpret_cast<float4*>(buf);
        // a tile is read into layout 1 for an odd number of rounds and into
        // layout 0 for an even one; each round moves once to the other layout,
        // so the tile ends in layout 0 (its coalesced stores) after nr
        // transposes
        const int ntr = nr;
        int done_tr = 0;
        auto release = [&]() {
            if (CL > 1) cluster_sync_all();
            else __syncthreads();
            if (nx < total && !failed) issue(nx, b);
        };

        // the tile's cost table (warp 0), published by the barrier after the wait
        const TileTab& tt = ttab[tpar];
        if (kPhase && tid < 32) tile_tab_fill(&ttab[tpar], T.tprog, base, tid);
        tpar ^= 1u;
        // After a timed-out wait the CTA walks its remaining tiles without
        // waiting, loading or storing (the copies stay pending on this phase
        // until the exit drain): the barriers stay in step with the cluster
        // and the loop keeps a single path.
        const int ok = failed ? 0 : (mbar_wait_bounded(full + b, (phase >> b) & 1u) ? 1 : 0);
        if (__syncthreads_and(ok)) {
            phase ^= 1u << b;
            pend &= ~(1u << b);
        } else if (!failed) {
            if (tid == 0) atomicExch(err, 1);
            failed = true;
            if (CL == 1) break;  // no cluster to keep in step
        }
        int cur = nr & 1;
        if constexpr (TM) {
            if (cur) S::template lds_tma<1>(buf, X, Y, tid);
            else S::template lds_tma<0>(buf, X, Y, tid);
        } else {
            if (cur) S::template lds_dense<1>(buf, X, Y, tid);
            else S::template lds_dense<0>(buf, X, Y, tid);
        }
        __syncthreads();  // dense reads done before the swizzled writes
        if (ntr == 0) release();

        auto to_layout = [&](int g) {
            if (g == cur) return;
            if (cur == 0) S::template sts<0>(buf4, X, Y, tid);
            else S::template sts<1>(buf4, X, Y, tid);
            __syncthreads();
            if (g == 0) S::template lds<0>(buf4, X, Y, tid);
            else S::template lds<1>(buf4, X, Y, tid);
            cur = g;
            if (++done_tr == ntr) release();
        };
        auto do_phase = [&](const float2* ltab, int frame, bool staged) {
            const float2* t = (kSTab && staged) ? stab : ltab;
            if (cur == 0) S::template phase<0>(X, Y, T, tt, tid, t, frame, pq);
            else S::template phase<1>(X, Y, T, tt, tid, t, frame, pq);
        };
        const float2* tab = reinterpret_cast<const float2*>(T.tab);
        for (int r = 0; r < nr; ++r) {
            const SweepRound rd = T.rounds[r];
            const LayerDev ly = slay[r];
            const float2* ltab = tab + (int64_t)rd.layer * T.tab_stride;
            // the state after the previous layer, before this layer's phase
            if (zon && rd.phase_pre && rd.layer > 0) {
                double* za = zacc + r * kZQ;
                const int sg = ly.frame ? -1 : 1;
                if (cur == 0) S::template zexp<0>(X, Y, tid, zred, za, tm, base, T.n, sg);
                else S::template zexp<1>(X, Y, tid, zred, za, tm, base, T.n, sg);
            }
            if (kPhase && rd.phase_pre) do_phase(ltab, ly.frame, rd.layer == slayer);
            const float w = (float)ly.w;
            // zig-zag: a round starts in the current layout
            if (cur == 0) {
                S::template rotate<0>(X, Y, w);
                to_layout(1);
                S::template rotate<1>(X, Y, w);
            } else {
                S::template rotate<1>(X, Y, w);
                to_layout(0);
                S::template rotate<0>(X, Y, w);
            }
            // (forward plans apply a layer's phase before its rotations only:
            // no phase_post here, which keeps the register pressure down)
        }
        to_layout(0);

        if ((flags & T_STORE) && !failed) {
            float2* dst = reinterpret_cast<float2*>(T.psi) + base + tm.gofs(S::template e_thread<0>(tid));
            const uint64_t gP = tm.gofs(1u << P);
            if (T.c + T.n1 <= 8) {  // layout-0 registers (tile bits 8..12) in the second run: one shift
                const int sh = T.g1 + 8 - T.c - T.n1;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    float2* d = dst + ((uint64_t)j << sh);
                    stg2(d, X[j].x, Y[j].x);
                    stg2(d + gP, X[j].y, Y[j].y);
                }
            } else {  // the map is additive over disjoint bits: Gray-code walk over j
                uint64_t step[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) step[q] = tm.gofs(1u << (8 + q));
                uint64_t off = 0;
#pragma unroll
                for (int i = 0; i < NJ; ++i) {
                    const int j = i ^ (i >> 1);
                    if (i > 0) {
                        const int q = __ffs(i) - 1;
                        if ((j >> q) & 1) off += step[q];
                        else off -= step[q];
                    }
                    stg2(dst + off, X[j].x, Y[j].x);
                    stg2(dst + off + gP, X[j].y, Y[j].y);
                }
            }
        }
    }
    // before the shared memory goes away: wait (bounded) for copies in flight;
    // a drain that gives up is reported with the sticky status 2
    if (tid == 0)
        for (int q = 0; q < NB; ++q)
            if (((pend >> q) & 1u) && !mbar_wait_bounded(full + q, (phase >> q) & 1u)) atomicMax(err, 2);
    __syncthreads();
    if (zon) {
        double* zp = tasks[0].zpart + (size_t)blockIdx.x * (kZSlots * kZQ);
        for (int i = (int)tid; i < kZSlots * kZQ; i += NT) zp[i] = zacc[i];
    }
}

template <int C, int V, bool TM = false>
constexpr size_t pair_smem() {
    return PairSweep<C>::SMEM_BYTES + (V == V_ZPHASE ? PairSweep<C>::Z_BYTES : 0) +
           (V == V_PHASE ? (size_t)kPairTabSmem * sizeof(float2) : 0) + (TM ? 1024 : 0);
}

template <int C, int V, bool TM>
static cudaError_t launch_pair_tm(const SweepLaunch& L, int grid, cudaStream_t st) {
    constexpr size_t smem = pair_smem<C, V, TM>();
    if (V != V_LEAN && !L.pq) return cudaErrorInvalidValue;  // the phase needs the Q tables
    if (L.ntasks != 1 || (TM && (!L.load || !L.load->tma))) return cudaErrorInvalidValue;  // one task per launch
    const PairQ pq = L.pq ? *L.pq : PairQ{};
    PairLoad tm;
    if (L.load) tm = *L.load;
    else std::memset(&tm, 0, sizeof tm);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_pair_kernel<C, V, 1, TM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sweep_pair_kernel<C, V, 4, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (L.cluster == 4 && L.total_tiles % 4 == 0 && grid % 4 == 0 && grid >= 4) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(PairSweep<C>::NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 4;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, sweep_pair_kernel<C, V, 4, TM>, L.tasks, L.tile_prefix, L.ntasks,
                                           L.total_tiles, L.err, pq, tm);
        return note_launch(e);
    }
    sweep_pair_kernel<C, V, 1, TM><<<grid, PairSweep<C>::NT, smem, st>>>(L.tasks, L.tile_prefix, L.ntasks,
                                                                          L.total_tiles, L.err, pq, tm);
    return note_launch(cudaGetLastError());
}

template <int C, int V>
static cudaError_t launch_pair_cfg(const SweepLaunch& L, int grid, cudaStream_t st) {
    return L.load && L.load->tma ? launch_pair_tm<C, V, true>(L, grid, st) : launch_pair_tm<C, V, false>(L, grid, st);
}

cudaError_t launch_sweep_pair(const SweepLaunch& L, int grid, cudaStream_t st) {
    if (L.pairc == 2 && L.variant == V_LEAN) return launch_pair_cfg<2, V_LEAN>(L, grid, st);
    if (L.pairc == 2 && L.variant == V_PHASE) return launch_pair_cfg<2, V_PHASE>(L, grid, st);
    if (L.pairc == 3 && L.variant == V_LEAN) return launch_pair_cfg<3, V_LEAN>(L, grid, st);
    if (L.pairc == 3 && L.variant == V_PHASE) return launch_pair_cfg<3, V_PHASE>(L, grid, st);
    if (L.pairc == 2 && L.variant == V_ZPHASE) return launch_pair_cfg<2, V_ZPHASE>(L, grid, st);
    if (L.pairc == 3 && L.variant == V_ZPHASE) return launch_pair_cfg<3, V_ZPHASE>(L, grid, st);
    return cudaErrorInvalidValue;
}

// Persistent grid: as many four-CTA clusters as can be resident at once
// (a multiple of four), else one CTA per resident slot.
template <int V>
static int pair_grid_v() {
    auto kern = sweep_pair_kernel<2, V, 4, false>;
    constexpr size_t smem = pair_smem<2, V>();
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4);
    cfg.blockDim = dim3(PairSweep<2>::NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 4;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl > 0) return 4 * ncl;
    cudaGetLastError();
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_pair_kernel<2, V, 1, false>, PairSweep<2>::NT, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

int sweep_pair_grid(int variant) {
    if (variant == V_LEAN) return pair_grid_v<V_LEAN>();
    if (variant == V_ZPHASE) return pair_grid_v<V_ZPHASE>();
    return pair_grid_v<V_PHASE>();
}

}  // namespace qs
