// Packed-pair adjoint sweep: the reverse sweeps of the gradient over the
// strided complex64 shapes (c = 2 or 3), layouts in qs_pair.h.
//
// Same work as sweep_kernel with two arrays (qs_sweep.cuh): psi and lambda
// are rotated back one layer at a time; before every butterfly the term
// Im(conj(lambda_a) psi_b + conj(lambda_b) psi_a) of dF/dbeta is accumulated
// (scaled by |f|^{2r} for the r rotations of the layer already undone), and
// at an un-phase the term (C) Im(conj(lambda) psi) of dF/dgamma.  Both arrays
// are held as pairs split by component (X = re, Y = im of the two members,
// which differ in the pack bit), so the butterflies and the dF/dbeta products
// of every bit but the pack bit are packed f32x2 FMAs, and the transposes
// move 16-byte pairs.  One CTA of 256 threads per SM with three 64 KB
// buffers: the next tile's psi and lambda land in two of them while the
// current tile, already in registers, is transposed through the third (psi,
// then lambda), so the loads overlap all of a tile's arithmetic.
#include "qs_pair.h"
#include "qs_sweep.cuh"

namespace qs {

namespace {

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// A zero the compiler cannot see through: XORed into the per-thread shared
// memory base of a transpose so that the 16-32 slot addresses are formed at
// the access (one LOP3 each) instead of being hoisted out of the tile loop
// and held in registers for the whole kernel.
// Landing-buffer position of tile element e: the pack bit flipped with tile
// bit 4.  The 8-byte reads of layout 0 (half-warp lanes on tile bits 0, 1,
// 3 or 2, and 4) then hit 16 distinct bank pairs; a 16-byte copy (elements
// e, e + 1) stays whole because the pack bit is 2 or more.
template <int P>
__device__ __forceinline__ uint32_t land(uint32_t e) { return P == 0 ? e : e ^ (((e >> 4) & 1u) << P); }

__device__ __forceinline__ uint32_t opaque_zero() {
    uint32_t z;
    asm volatile("mov.u32 %0, 0;" : "=r"(z));
    return z;
}

__device__ __forceinline__ void stg2(float2* p, float re, float im) {
    asm volatile("st.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(re), "f"(im) : "memory");
}

// float partial sum over a warp, lane 0 stores it (as double) to red[warp * nslots + slot]
__device__ __forceinline__ void warp_sum_f(float v, double* red, int slot, int nslots) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) * nslots + slot] = (double)v;
}

template <int C>
struct PairAdj {
    static constexpr int K = kPairK, NT = 256, NJ = 16, P = pair_adj_layout(C).P, NW = NT / 32,
                         NSLOT = 2 * kMaxRounds;
    static constexpr size_t TILE_BYTES = (size_t)8 << K;
    static constexpr size_t TT_OFF = 3 * TILE_BYTES + 64 + (size_t)NW * NSLOT * 8;  // two TileTabs
    static constexpr size_t KOFF_OFF = TT_OFF + 2 * sizeof(TileTab);  // 16 tile-copy offsets (uint64)
    // the launch's task and its rounds' layer parameters, copied once per CTA
    static constexpr size_t TASK_OFF = (KOFF_OFF + 16 * sizeof(uint64_t) + 15) & ~(size_t)15;
    static constexpr size_t LAY_OFF = (TASK_OFF + sizeof(SweepTask) + 15) & ~(size_t)15;
    static constexpr size_t SMEM_BYTES = LAY_OFF + kMaxRounds * sizeof(LayerDev);
    // compile-time tile bits of layout g: slot bit 0 is the pack bit
    template <int g> struct Map {
        __host__ __device__ static constexpr int slot(int b) {
            return b == 0 ? pair_adj_layout(C).P : pair_adj_layout(C).regs[g][b - 1];
        }
        __host__ __device__ static constexpr int thr(int j) { return pair_adj_layout(C).tbits[g][j]; }
    };

    template <int g, int t> __host__ __device__ static constexpr int tb() { return pair_adj_layout(C).tbits[g][t]; }
    template <int g> __host__ __device__ static constexpr int rmask() { return pair_adj_layout(C).rotmask[g]; }

    template <int g>
    __device__ static __forceinline__ uint32_t e_thread(uint32_t tid) {
        uint32_t e = 0;
        static_for<0, 8>([&](auto tc) {
            constexpr int t = decltype(tc)::value;
            e |= ((tid >> t) & 1u) << tb<g, t>();
        });
        return e;
    }
    template <int g>
    __host__ __device__ static constexpr uint32_t e_slot(int j) {
        uint32_t e = 0;
        for (int b = 0; b < 4; ++b) e |= (uint32_t)((j >> b) & 1) << pair_adj_layout(C).regs[g][b];
        return e;
    }

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
    __device__ static __forceinline__ void lds_dense(const float2* src, float2 (&X)[NJ], float2 (&Y)[NJ],
                                                     uint32_t tid) {
        const uint32_t et = e_thread<0>(tid);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if constexpr (P == 0) {  // the two members are adjacent: one 16-byte read
                const float4 v = reinterpret_cast<const float4*>(src)[(et | e_slot<0>(j)) >> 1];
                X[j] = make_float2(v.x, v.z);
                Y[j] = make_float2(v.y, v.w);
            } else {
                const float2 a = src[land<P>(et | e_slot<0>(j))];
                const float2 b = src[land<P>(et | e_slot<0>(j) | (1u << P))];
                X[j] = make_float2(a.x, b.x);
                Y[j] = make_float2(a.y, b.y);
            }
        }
    }

    // Butterflies a' = a + w (-i b), b' = b + w (-i a) on psi (p) and lambda
    // (l), each bit preceded by its dF/dbeta term.
    template <int g>
    __device__ static __forceinline__ void rotate(float2 (&Xp)[NJ], float2 (&Yp)[NJ], float2 (&Xl)[NJ],
                                                  float2 (&Yl)[NJ], float w, float fabs2, float& fpow, float& gacc) {
        const float2 w2 = make_float2(w, w), nw2 = make_float2(-w, -w), z2 = make_float2(0.f, 0.f);
        static_for<0, 4>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            if constexpr (((rmask<g>() >> b) & 1) != 0) {
                float2 accP = z2, accN = z2;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    if (j & (1 << b)) continue;
                    const int j2 = j | (1 << b);
                    const float2 xpa = Xp[j], ypa = Yp[j], xpb = Xp[j2], ypb = Yp[j2];
                    const float2 xla = Xl[j], yla = Yl[j], xlb = Xl[j2], ylb = Yl[j2];
                    // Im(conj(la) pb) + Im(conj(lb) pa), both halves of the pairs
                    accP = ffma2(xla, ypb, accP);
                    accP = ffma2(xlb, ypa, accP);
                    accN = ffma2(yla, xpb, accN);
                    accN = ffma2(ylb, xpa, accN);
                    Xp[j] = ffma2(w2, ypb, xpa);
                    Yp[j] = ffma2(nw2, xpb, ypa);
                    Xp[j2] = ffma2(w2, ypa, xpb);
                    Yp[j2] = ffma2(nw2, xpa, ypb);
                    Xl[j] = ffma2(w2, ylb, xla);
                    Yl[j] = ffma2(nw2, xlb, yla);
                    Xl[j2] = ffma2(w2, yla, xlb);
                    Yl[j2] = ffma2(nw2, xla, ylb);
                }
                const float part = (accP.x + accP.y) - (accN.x + accN.y);
                gacc = fmaf(part, fpow, gacc);
                fpow *= fabs2;
            }
        });
        if (g == 0) {  // the pack bit: the two halves of every pair
            float part = 0.f;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const float par = Xp[j].x, pbr = Xp[j].y, pai = Yp[j].x, pbi = Yp[j].y;
                const float lar = Xl[j].x, lbr = Xl[j].y, lai = Yl[j].x, lbi = Yl[j].y;
                float t0 = lar * pbi - lai * pbr;
                t0 = fmaf(lbr, pai, t0);
                t0 = fmaf(-lbi, par, t0);
                part += t0;
                Xp[j] = make_float2(fmaf(w, pbi, par), fmaf(w, pai, pbr));
                Yp[j] = make_float2(fmaf(-w, pbr, pai), fmaf(-w, par, pbi));
                Xl[j] = make_float2(fmaf(w, lbi, lar), fmaf(w, lai, lbr));
                Yl[j] = make_float2(fmaf(-w, lbr, lai), fmaf(-w, lar, lbi));
            }
            gacc = fmaf(part, fpow, gacc);
            fpow *= fabs2;
        }
    }

    // both arrays from layout g: the map is additive over disjoint bits, so
    // the pair index is walked in Gray-code order, one per-bit step per pair
    template <int g>
    __device__ static __forceinline__ void store(float2* psi, float2* lam, const TMap& tm, uint64_t base,
                                                 const float2 (&Xp)[NJ], const float2 (&Yp)[NJ],
                                                 const float2 (&Xl)[NJ], const float2 (&Yl)[NJ], uint32_t tid) {
        const uint64_t gP = tm.gofs(1u << P);
        const uint64_t t0 = base + tm.gofs(e_thread<g>(tid));
        float2* dp = psi + t0;
        float2* dl = lam + t0;
        uint64_t step[4];
        static_for<0, 4>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            step[q] = tm.gofs(1u << pair_adj_layout(C).regs[g][q]);
        });
        uint64_t o = 0;
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            const int j = i ^ (i >> 1);
            if (i > 0) {
                const int q = __ffs(i) - 1;
                if ((j >> q) & 1) o += step[q];
                else o -= step[q];
            }
            stg2(dp + o, Xp[j].x, Yp[j].x);
            stg2(dp + o + gP, Xp[j].y, Yp[j].y);
            stg2(dl + o, Xl[j].x, Yl[j].x);
            stg2(dl + o + gP, Xl[j].y, Yl[j].y);
        }
    }

    // phase of the layer on both arrays, then the dF/dgamma term C Im(conj(l) p)
    // (slot m = half | j << 1 of the layout's cost program; Q[m] from the
    // kernel parameters; the table through a generic pointer, in shared
    // memory when it was staged at kernel start)
    template <int g>
    __device__ static __forceinline__ void phase(float2 (&Xp)[NJ], float2 (&Yp)[NJ], float2 (&Xl)[NJ],
                                                 float2 (&Yl)[NJ], const SweepTask& T, const TileTab& tt,
                                                 uint32_t tid, const float2* __restrict__ tab, int frame,
                                                 float& gacc, const PairAdjQ& pq) {
        SlotCost<5> sc;
        sc.template init_tile<Map<g>, 8>(tt, T.cprog[g], tid, frame, T.cost_lo);
        const int top = T.tab_stride - 1;
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int ia = SlotCost<5>::clamp_tab(sc.idx_noq(2 * j) + pq.q[g][2 * j], top);
            const int ib = SlotCost<5>::clamp_tab(sc.idx_noq(2 * j + 1) + pq.q[g][2 * j + 1], top);
            const float2 fa = tab[ia], fb = tab[ib];
            const float par = Xp[j].x, pbr = Xp[j].y, pai = Yp[j].x, pbi = Yp[j].y;
            const float lar = Xl[j].x, lbr = Xl[j].y, lai = Yl[j].x, lbi = Yl[j].y;
            const float npar = fmaf(par, fa.x, -pai * fa.y), npai = fmaf(par, fa.y, pai * fa.x);
            const float npbr = fmaf(pbr, fb.x, -pbi * fb.y), npbi = fmaf(pbr, fb.y, pbi * fb.x);
            const float nlar = fmaf(lar, fa.x, -lai * fa.y), nlai = fmaf(lar, fa.y, lai * fa.x);
            const float nlbr = fmaf(lbr, fb.x, -lbi * fb.y), nlbi = fmaf(lbr, fb.y, lbi * fb.x);
            Xp[j] = make_float2(npar, npbr);
            Yp[j] = make_float2(npai, npbi);
            Xl[j] = make_float2(nlar, nlbr);
            Yl[j] = make_float2(nlai, nlbi);
            part = fmaf((float)(ia + T.cost_lo), nlar * npai - nlai * npar, part);
            part = fmaf((float)(ib + T.cost_lo), nlbr * npbi - nlbi * npbr, part);
        }
        gacc += part;
    }
};

}  // namespace

// The un-phase of a reverse sweep reads its layer table from shared memory
// when it has at most this many entries.
constexpr int kAdjTabSmem = 1024;

template <int C>
__global__ void __launch_bounds__(256, 1)
    sweep_pair_adj_kernel(const SweepTask* __restrict__ tasks, const int64_t* __restrict__ prefix, int ntasks,
                          int64_t total, int* __restrict__ err, const __grid_constant__ PairAdjQ pq) {
    using S = PairAdj<C>;
    constexpr int K = S::K, NT = S::NT, NJ = S::NJ, P = S::P, NW = S::NW, NSLOT = S::NSLOT;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2* buf = reinterpret_cast<float2*>(smraw);  // landing: [psi tile][lambda tile]
    float4* wk4 = reinterpret_cast<float4*>(smraw + 2 * S::TILE_BYTES);  // transpose buffer
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw + 3 * S::TILE_BYTES);
    double* red = reinterpret_cast<double*>(smraw + 3 * S::TILE_BYTES + 64);
    TileTab* ttab = reinterpret_cast<TileTab*>(smraw + S::TT_OFF);
    uint64_t* koff = reinterpret_cast<uint64_t*>(smraw + S::KOFF_OFF);
    float2* stab = reinterpret_cast<float2*>(smraw + S::SMEM_BYTES);  // [kAdjTabSmem]
    // one task per launch (checked on the host): read from shared memory,
    // so the per-tile and per-round fields are short-latency loads
    const SweepTask& T = *reinterpret_cast<const SweepTask*>(smraw + S::TASK_OFF);
    LayerDev* slay = reinterpret_cast<LayerDev*>(smraw + S::LAY_OFF);
    const uint32_t tid = threadIdx.x;
    uint32_t tpar = 0;  // parity of the CTA's tile count: which TileTab
    float2 Xp[NJ], Yp[NJ], Xl[NJ], Yl[NJ];

    bool pending = false;
    // every thread: 16-byte cp.async copies of its share of both strided
    // tiles, completing on the barrier (one arrival per thread)
    auto issue = [&](int64_t tile) {
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        // thread t copies elements e = 2t + 512k, k < 16, of each array: the
        // landing map and the global offset split into a per-thread part and
        // the k part (koff[k] = gofs(512 k), the same for every tile)
        const uint32_t e_t = 2u * tid;
        const uint64_t off_t = tm.base(tile) + tm.gofs(e_t);
        const uint32_t lt = land<P>(e_t);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float2* src = reinterpret_cast<const float2*>(a == 0 ? T.psi : T.lam) + off_t;
            const uint32_t sb = smem_u32(buf + ((size_t)a << K));
#pragma unroll
            for (int k = 0; k < 16; ++k)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + 8u * (lt ^ land<P>(512u * k))),
                             "l"(src + koff[k])
                             : "memory");
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(full)) : "memory");
        pending = true;
    };

    if (tid == 0) {
        mbar_init(full, NT);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const int* src = reinterpret_cast<const int*>(tasks);
        int* dst = reinterpret_cast<int*>(smraw + S::TASK_OFF);
        for (int i = (int)tid; i < (int)(sizeof(SweepTask) / 4); i += NT) dst[i] = __ldg(src + i);
        const SweepTask& T0 = tasks[0];
        if ((int)tid < T0.nrounds) slay[tid] = T0.layers[T0.rounds[tid].layer];
        if (tid < 16) koff[tid] = TMap{T0.c, T0.g0, T0.n1, T0.g1, K}.gofs(512u * tid);
    }
    // the table of the (first) layer whose phase this sweep un-applies
    int slayer = -1;
    if (ntasks == 1 && tasks[0].tab_stride <= kAdjTabSmem) {
        const SweepTask& T0 = tasks[0];
        for (int r = 0; r < T0.nrounds; ++r)
            if (T0.rounds[r].phase_pre || T0.rounds[r].phase_post) {
                slayer = T0.rounds[r].layer;
                break;
            }
        if (slayer >= 0) {
            const float2* src = reinterpret_cast<const float2*>(T0.tab) + (int64_t)slayer * T0.tab_stride;
            for (int i = (int)tid; i < T0.tab_stride; i += NT) stab[i] = __ldg(src + i);
        }
    }
    __syncthreads();
    if ((int64_t)blockIdx.x < total) issue(blockIdx.x);

    uint32_t parity = 0;
    for (int64_t gt = blockIdx.x; gt < total; gt += gridDim.x) {
        const int flags = T.flags, nr = T.nrounds;
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        const uint64_t base = tm.base(gt);
        const int64_t nx = gt + gridDim.x;
        // the tile's cost table (warp 0), published by the barrier after the wait
        const TileTab& tt = ttab[tpar];
        if (tid < 32) tile_tab_fill(&ttab[tpar], T.tprog, base, tid);
        tpar ^= 1u;

        const int ok = mbar_wait_bounded(full, parity) ? 1 : 0;
        if (!__syncthreads_and(ok)) {  // the copies stay pending on this phase
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        parity ^= 1u;
        if (tid == 0) pending = false;
        S::lds_dense(buf, Xp, Yp, tid);
        S::lds_dense(buf + ((size_t)1 << K), Xl, Yl, tid);
        __syncthreads();  // landing buffers read: the next tile's copies may start
        if (nx < total) issue(nx);

        // psi and lambda through the one transpose buffer.  A thread rewrites
        // exactly the positions it last read, so only the reads of the new
        // layout by other threads need barriers.
        int cur = 0;
        auto to_layout = [&](int g) {
            if (g == cur) return;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                float2(&X)[NJ] = a == 0 ? Xp : Xl;
                float2(&Y)[NJ] = a == 0 ? Yp : Yl;
                if (a == 1) __syncthreads();  // psi's reads of the new layout are done
                if (cur == 0) S::template sts<0>(wk4, X, Y, tid);
                else if (cur == 1) S::template sts<1>(wk4, X, Y, tid);
                else S::template sts<2>(wk4, X, Y, tid);
                __syncthreads();
                if (g == 0) S::template lds<0>(wk4, X, Y, tid);
                else if (g == 1) S::template lds<1>(wk4, X, Y, tid);
                else S::template lds<2>(wk4, X, Y, tid);
            }
            cur = g;
        };
        auto rotate_cur = [&](float w, float fabs2, float& fpow, float& gB) {
            if (cur == 0) S::template rotate<0>(Xp, Yp, Xl, Yl, w, fabs2, fpow, gB);
            else if (cur == 1) S::template rotate<1>(Xp, Yp, Xl, Yl, w, fabs2, fpow, gB);
            else S::template rotate<2>(Xp, Yp, Xl, Yl, w, fabs2, fpow, gB);
        };
        auto do_phase = [&](const float2* ltab, int frame, float& gG, bool staged) {
            const float2* t = staged ? stab : ltab;
            if (cur == 0) S::template phase<0>(Xp, Yp, Xl, Yl, T, tt, tid, t, frame, gG, pq);
            else if (cur == 1) S::template phase<1>(Xp, Yp, Xl, Yl, T, tt, tid, t, frame, gG, pq);
            else S::template phase<2>(Xp, Yp, Xl, Yl, T, tt, tid, t, frame, gG, pq);
        };
        const float2* tab = reinterpret_cast<const float2*>(T.tab);
        for (int r = 0; r < nr; ++r) {
            const SweepRound rd = T.rounds[r];
            const LayerDev ly = slay[r];
            const float2* ltab = tab + (int64_t)rd.layer * T.tab_stride;
            float gB = 0.f, gG = 0.f;
            if (rd.phase_pre) do_phase(ltab, ly.frame, gG, rd.layer == slayer);
            const float fabs2 = (float)(ly.fabs * ly.fabs);
            float fpow = 1.f;
            for (int i = 0; i < rd.r0; ++i) fpow *= fabs2;  // |f|^{2 r0}
            const float w = (float)ly.w;
            // zig-zag over the three layouts, starting in the current one
            if (cur == 0) {
                rotate_cur(w, fabs2, fpow, gB);
                to_layout(1);
                rotate_cur(w, fabs2, fpow, gB);
                to_layout(2);
                rotate_cur(w, fabs2, fpow, gB);
            } else {
                rotate_cur(w, fabs2, fpow, gB);
                to_layout(1);
                rotate_cur(w, fabs2, fpow, gB);
                to_layout(0);
                rotate_cur(w, fabs2, fpow, gB);
            }
            if (rd.phase_post) do_phase(ltab, ly.frame, gG, rd.layer == slayer);
            warp_sum_f(gB, red, 2 * r, NSLOT);
            warp_sum_f(gG, red, 2 * r + 1, NSLOT);
        }
        // stored from the layout the rounds end in: 0 after an even number,
        // 2 after an odd one (both hold adjacent amplitudes on the low lanes)
        if (cur == 1) to_layout(0);
        if (flags & T_STORE) {
            float2* psi = reinterpret_cast<float2*>(T.psi);
            float2* lam = reinterpret_cast<float2*>(T.lam);
            if (cur == 0) S::template store<0>(psi, lam, tm, base, Xp, Yp, Xl, Yl, tid);
            else S::template store<2>(psi, lam, tm, base, Xp, Yp, Xl, Yl, tid);
        }
        if (T.np > 0) {
            const int np = T.np;
            __syncthreads();
            if (tid < (uint32_t)np) {
                double s = 0.0;
                for (int w = 0; w < NW; ++w) s += red[w * NSLOT + tid];
                T.partials[(T.part_base + gt) * np + tid] = s;
            }
            __syncthreads();
        }
    }
    // a drain that gives up is reported with the sticky status 2
    if (tid == 0 && pending && !mbar_wait_bounded(full, parity)) atomicMax(err, 2);
}

template <int C>
constexpr size_t pair_adj_smem() { return PairAdj<C>::SMEM_BYTES + (size_t)kAdjTabSmem * sizeof(float2); }

template <int C>
static cudaError_t launch_pair_adj_cfg(const SweepLaunch& L, int grid, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_pair_adj_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)pair_adj_smem<C>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (!L.paq || L.ntasks != 1) return cudaErrorInvalidValue;  // the un-phase's Q tables; one task per launch
    sweep_pair_adj_kernel<C><<<grid, PairAdj<C>::NT, pair_adj_smem<C>(), st>>>(L.tasks, L.tile_prefix, L.ntasks,
                                                                                L.total_tiles, L.err, *L.paq);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_sweep_pair_adj(const SweepLaunch& L, int grid, cudaStream_t st) {
    if (L.pairc == 1) return launch_pair_adj_cfg<1>(L, grid, st);
    if (L.pairc == 2) return launch_pair_adj_cfg<2>(L, grid, st);
    if (L.pairc == 3) return launch_pair_adj_cfg<3>(L, grid, st);
    return cudaErrorInvalidValue;
}

int sweep_pair_adj_grid() {
    cudaFuncSetAttribute(sweep_pair_adj_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pair_adj_smem<2>());
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_pair_adj_kernel<2>, PairAdj<2>::NT,
                                                  pair_adj_smem<2>());
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

}  // namespace qs
