// Packed-pair sweep of the run-structured shape A (complex64 states of 33 and
// 34 qubits): tile bits [0, 8) are one 2 KB run, [8, 12) the four top qubits,
// bit 12 the batch bit; the targets are tile bits [0, 12).  Forward
// rotations, with the phase of a layer boundary (V_PHASE) or without
// (V_LEAN); layouts in qs_pair.h (pair_runs_layout).
//
// Same tile walk as sweep_pair_kernel (qs_sweep_pair.cu): three persistent
// CTAs per SM, one in-place 64 KB tile buffer each, the next tile's copies
// issued after the current tile's last shared-memory read, bounded waits.
// The tile arrives as 32 bulk copies (cp.async.bulk) of one 2 KB run each,
// issued by warp 0 and completing on the tile's mbarrier.  A pair is two
// adjacent amplitudes (the pack bit is tile bit 0), split by component into
// X = (re_a, re_b), Y = (im_a, im_b): the butterflies of the other register
// bits are packed f32x2 FMAs.  Layout 0 rotates the pack bit and run bits
// 6..10, layout 1 run bits 1..5 and, with lane shuffles, tile bit 11.
#include "qs_pair.h"
#include "qs_sweep.cuh"

namespace qs {

namespace {

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// A zero the compiler cannot see through: XORed into the per-thread shared
// memory base of a transpose so that the slot addresses are formed at the
// access instead of being held in registers for the whole kernel.
__device__ __forceinline__ uint32_t opaque_zero() {
    uint32_t z;
    asm volatile("mov.u32 %0, 0;" : "=r"(z));
    return z;
}

struct RunsSweep {
    static constexpr int K = kPairK, NT = 128, NJ = 32, P = 0;
    static constexpr size_t BUF_BYTES = (size_t)8 << K;
    static constexpr size_t TT_OFF = BUF_BYTES + 64;  // two TileTabs (by tile parity)
    // the launch's task and its rounds' layer parameters, copied once per CTA
    static constexpr size_t TASK_OFF = (TT_OFF + 2 * sizeof(TileTab) + 15) & ~(size_t)15;
    static constexpr size_t LAY_OFF = (TASK_OFF + sizeof(SweepTask) + 15) & ~(size_t)15;
    static constexpr size_t RED_OFF = LAY_OFF + kMaxRounds * sizeof(LayerDev);  // readout warp sums [4][3]
    static constexpr size_t SMEM_BYTES = RED_OFF + (NT / 32) * 3 * sizeof(double);
    static_assert(SMEM_BYTES % 16 == 0, "the staged phase table follows the tile tables");
    static_assert(kRunBits == 8 && K == 13, "layouts of pair_runs_layout");
    template <int g> struct Map {
        __host__ __device__ static constexpr int slot(int b) { return b == 0 ? P : pair_runs_layout().regs[g][b - 1]; }
        __host__ __device__ static constexpr int thr(int j) { return pair_runs_layout().tbits[g][j]; }
    };
    template <int g, int t> __host__ __device__ static constexpr int tb() { return pair_runs_layout().tbits[g][t]; }

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
        for (int b = 0; b < 5; ++b) e |= (uint32_t)((j >> b) & 1) << pair_runs_layout().regs[g][b];
        return e;
    }

    // ---- transposes (16-byte pair units, swizzled) -------------------------
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
    // from the landing buffer (tile order) into layout 0: one 16-byte read per
    // pair, a warp's lanes on run bits 1..5 (512 contiguous bytes)
    __device__ static __forceinline__ void lds_dense0(const float2* src, float2 (&X)[NJ], float2 (&Y)[NJ],
                                                      uint32_t tid) {
        const uint32_t et = e_thread<0>(tid);
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const float4 v = s4[(et | e_slot<0>(j)) >> 1];
            X[j] = make_float2(v.x, v.z);
            Y[j] = make_float2(v.y, v.w);
        }
    }

    // ---- rotations: a' = a + w (-i b), b' = b + w (-i a) --------------------
    template <int g>
    __device__ static __forceinline__ void rotate(float2 (&X)[NJ], float2 (&Y)[NJ], float w) {
        const float2 w2 = make_float2(w, w), nw2 = make_float2(-w, -w);
        static_for<0, 5>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
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
        });
        if (g == 0) {  // the pack bit: the two halves of every pair
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const float ar = X[j].x, br = X[j].y, ai = Y[j].x, bi = Y[j].y;
                X[j] = make_float2(fmaf(w, bi, ar), fmaf(w, ai, br));
                Y[j] = make_float2(fmaf(-w, br, ai), fmaf(-w, ar, bi));
            }
        } else {  // tile bit 11 on lane bit 0: the partner amplitude is in lane ^ 1
            // both members update alike: re' = re + w im_other, im' = im - w re_other
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                float2 xo, yo;
                xo.x = __shfl_xor_sync(0xffffffffu, X[j].x, 1);
                xo.y = __shfl_xor_sync(0xffffffffu, X[j].y, 1);
                yo.x = __shfl_xor_sync(0xffffffffu, Y[j].x, 1);
                yo.y = __shfl_xor_sync(0xffffffffu, Y[j].y, 1);
                X[j] = ffma2(w2, yo, X[j]);
                Y[j] = ffma2(nw2, xo, Y[j]);
            }
        }
    }

    // ---- phase: slot m = half | j << 1; Q[m] from the kernel parameters, the
    // layer table through a generic pointer (shared memory when staged) ------
    template <int g>
    __device__ static __forceinline__ void phase(float2 (&X)[NJ], float2 (&Y)[NJ], const SweepTask& T,
                                                 const TileTab& tt, uint32_t tid, const float2* __restrict__ tab,
                                                 int frame, const PairQ& pq) {
        pair_phase<Map<g>, 7>(X, Y, T.cprog[g], tt, tid, frame, T.cost_lo, tab, T.tab_stride - 1, pq.q[g]);
    }
};

constexpr int kRunsTabSmem = 1024;  // V_PHASE: staged layer table entries

}  // namespace

#ifndef QS_PHASE_OCC
#define QS_PHASE_OCC 3
#endif
template <int V>
__global__ void __launch_bounds__(128, V == V_PHASE ? QS_PHASE_OCC : 3)
    sweep_runs_kernel(const SweepTask* __restrict__ tasks, const int64_t* __restrict__ prefix, int ntasks,
                      int64_t total, int* __restrict__ err, const __grid_constant__ PairQ pq) {
    using S = RunsSweep;
    constexpr int K = S::K, NT = S::NT, NJ = S::NJ;
    // V_RUNS_GEN: |+> generated in registers, no load; V_RUNS_READ: E, P and
    // the norm of the tile after its rounds, as per-tile partials
    constexpr bool kGen = V == V_RUNS_GEN, kRead = V == V_RUNS_READ;
    constexpr bool kPhase = V != V_LEAN;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2* buf = reinterpret_cast<float2*>(smraw);
    float4* buf4 = reinterpret_cast<float4*>(smraw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw + S::BUF_BYTES);
    TileTab* ttab = reinterpret_cast<TileTab*>(smraw + S::TT_OFF);
    float2* stab = reinterpret_cast<float2*>(smraw + S::SMEM_BYTES);  // kPhase: [kRunsTabSmem]
    // one task per launch (checked on the host): read from shared memory,
    // so the per-tile and per-round fields are short-latency loads
    const SweepTask& T = *reinterpret_cast<const SweepTask*>(smraw + S::TASK_OFF);
    LayerDev* slay = reinterpret_cast<LayerDev*>(smraw + S::LAY_OFF);
    double* red = reinterpret_cast<double*>(smraw + S::RED_OFF);  // kRead: warp sums [NT / 32][3]
    const uint32_t tid = threadIdx.x;
    uint32_t tpar = 0;
    float2 X[NJ], Y[NJ];

    bool pending = false;
    // thread 0 arrives with the byte count, every other thread plainly; warp 0
    // issues one 2 KB bulk copy per lane (32 runs)
    auto issue = [&](int64_t tile) {
        if (tid == 0) mbar_expect_tx(full, (uint32_t)S::BUF_BYTES);
        else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(full)) : "memory");
        if (tid < 32) {
            __syncwarp();
            fence_proxy_async();  // the buffer's generic reads before the async writes
            const TMap tm{T.c, T.g0, T.n1, T.g1, K};
            const uint64_t base = (uint64_t)tile << (kRunBits + 1);
            constexpr uint32_t run = 1u << kRunBits;
            const uint32_t e0 = tid * run;
            const float2* src = reinterpret_cast<const float2*>(T.psi) + base + tm.gofs(e0);
            tma_load_1d(buf + e0, src, run * (uint32_t)sizeof(float2), full);
        }
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
        if ((int)tid < tasks[0].nrounds) slay[tid] = tasks[0].layers[tasks[0].rounds[tid].layer];
    }
    // the table of the (first) layer whose phase this sweep applies
    int slayer = -1;
    if (kPhase && ntasks == 1 && tasks[0].tab_stride <= kRunsTabSmem) {
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
    if (!kGen && (int64_t)blockIdx.x < total) issue(blockIdx.x);

    uint32_t parity = 0;
    for (int64_t gt = blockIdx.x; gt < total; gt += gridDim.x) {
        const int flags = T.flags, nr = T.nrounds;
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        const uint64_t base = (uint64_t)gt << (kRunBits + 1);
        const int64_t nx = gt + gridDim.x;
        // the tile's cost table (warp 0), published by the barrier after the wait
        const TileTab& tt = ttab[tpar];
        if (kPhase && tid < 32) tile_tab_fill(&ttab[tpar], T.tprog, base, tid);
        tpar ^= 1u;
        if constexpr (kGen) {
            // |+>^n: every amplitude 2^{-n/2}, real
            __syncthreads();  // the tile table is published
            const float a0 = (float)T.amp0;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                X[j] = make_float2(a0, a0);
                Y[j] = make_float2(0.f, 0.f);
            }
        } else {
            const int ok = mbar_wait_bounded(full, parity) ? 1 : 0;
            if (!__syncthreads_and(ok)) {  // the copies stay pending on this phase
                if (tid == 0) atomicExch(err, 1);
                break;
            }
            parity ^= 1u;
            pending = false;
            S::lds_dense0(buf, X, Y, tid);
            __syncthreads();  // dense reads done before the swizzled writes
        }
        // each round moves once to the other layout; an odd count moves back
        const int ntr = nr + (nr & 1);
        int done_tr = 0, cur = 0;
        auto release = [&]() {
            __syncthreads();
            if (!kGen && nx < total) issue(nx);
        };
        if (ntr == 0) release();
        auto to_layout = [&](int g) {
            if (g == cur) return;
            if (cur == 0) S::sts<0>(buf4, X, Y, tid);
            else S::sts<1>(buf4, X, Y, tid);
            __syncthreads();
            if (g == 0) S::lds<0>(buf4, X, Y, tid);
            else S::lds<1>(buf4, X, Y, tid);
            cur = g;
            if (++done_tr == ntr) release();
        };
        auto do_phase = [&](const float2* ltab, int frame, bool staged) {
            const float2* t = (kPhase && staged) ? stab : ltab;
            if (cur == 0) S::phase<0>(X, Y, T, tt, tid, t, frame, pq);
            else S::phase<1>(X, Y, T, tt, tid, t, frame, pq);
        };
        const float2* tab = reinterpret_cast<const float2*>(T.tab);
        for (int r = 0; r < nr; ++r) {
            const SweepRound rd = T.rounds[r];
            const LayerDev ly = slay[r];
            const float2* ltab = tab + (int64_t)rd.layer * T.tab_stride;
            if (kPhase && rd.phase_pre) do_phase(ltab, ly.frame, rd.layer == slayer);
            const float w = (float)ly.w;
            if (cur == 0) {
                S::rotate<0>(X, Y, w);
                to_layout(1);
                S::rotate<1>(X, Y, w);
            } else {
                S::rotate<1>(X, Y, w);
                to_layout(0);
                S::rotate<0>(X, Y, w);
            }
            // (forward plans apply a layer's phase before its rotations only)
        }
        to_layout(0);

        if (kRead && (flags & T_READOUT)) {
            float E = 0.f, Pg = 0.f, N = 0.f;
            pair_readout<typename S::template Map<0>, 7>(X, Y, T.cprog[0], tt, tid, T.layers[T.end_layer].frame,
                                                         T.cost_lo, T.gidx, pq.q[0], E, Pg, N);
            warp_sum_to((double)E, red, 0, 3);
            warp_sum_to((double)Pg, red, 1, 3);
            warp_sum_to((double)N, red, 2, 3);
        }
        if (flags & T_STORE) {
            // layout 0: slot bits are run bits 6, 7 (in the run) and tile bits
            // 8..10 (global bits g0..g0 + 2); lanes on run bits 1..5
            float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float2*>(T.psi) + base +
                                                    tm.gofs(S::e_thread<0>(tid)));
            const int sh = tm.g0;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const uint64_t off = ((uint64_t)(j & 3) << 6) + ((uint64_t)(j >> 2) << sh);
                dst[off >> 1] = make_float4(X[j].x, Y[j].x, X[j].y, Y[j].y);
            }
        }
        if (kRead && T.np > 0) {  // the tile's partials: E, P, norm
            __syncthreads();
            if (tid < (uint32_t)T.np) {
                double sum = 0.0;
                for (int w = 0; w < NT / 32; ++w) sum += red[w * 3 + tid];
                T.partials[(T.part_base + gt) * T.np + tid] = sum;
            }
            __syncthreads();
        }
    }
    // before the shared memory goes away: wait (bounded) for copies in flight;
    // a drain that gives up is reported with the sticky status 2
    if (tid == 0 && pending && !mbar_wait_bounded(full, parity)) atomicMax(err, 2);
    __syncthreads();
}

template <int V>
static size_t runs_smem() {
    return RunsSweep::SMEM_BYTES + (V != V_LEAN ? (size_t)kRunsTabSmem * sizeof(float2) : 0);
}

template <int V>
static cudaError_t launch_runs_cfg(const SweepLaunch& L, int grid, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(sweep_runs_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)runs_smem<V>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (V != V_LEAN && !L.pq) return cudaErrorInvalidValue;  // the phase and the readout need the Q tables
    if (L.ntasks != 1) return cudaErrorInvalidValue;           // one task per launch
    const PairQ pq = L.pq ? *L.pq : PairQ{};
    sweep_runs_kernel<V><<<grid, RunsSweep::NT, runs_smem<V>(), st>>>(L.tasks, L.tile_prefix, L.ntasks,
                                                                      L.total_tiles, L.err, pq);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_sweep_runs(const SweepLaunch& L, int grid, cudaStream_t st) {
    if (L.variant == V_PHASE) return launch_runs_cfg<V_PHASE>(L, grid, st);
    if (L.variant == V_LEAN) return launch_runs_cfg<V_LEAN>(L, grid, st);
    if (L.variant == V_RUNS_GEN) return launch_runs_cfg<V_RUNS_GEN>(L, grid, st);
    if (L.variant == V_RUNS_READ) return launch_runs_cfg<V_RUNS_READ>(L, grid, st);
    return cudaErrorInvalidValue;
}

int sweep_runs_grid(int variant) {
    auto grid_v = [](auto kern, size_t smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RunsSweep::NT, smem);
        if (per_sm < 1) per_sm = 1;
        return per_sm * sms;
    };
    return variant == V_LEAN ? grid_v(sweep_runs_kernel<V_LEAN>, runs_smem<V_LEAN>())
                             : grid_v(sweep_runs_kernel<V_PHASE>, runs_smem<V_PHASE>());
}

}  // namespace qs
