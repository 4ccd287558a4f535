// Persistent work-queue sweep of a batch: every sweep of every instance in
// one launch (the forward of all instances), or every reverse sweep (the
// adjoint of all instances), instead of one launch per wave of sweeps.
//
// Work items are the tiles of a task list ordered wave by wave (the w-th
// sweep of every instance, then the (w + 1)-th), so the sweep a tile depends
// on normally finished long before.  CTAs take items from one counter in that
// order (atomicAdd), which is deadlock-free without co-residency: a CTA only
// waits for items with smaller indices, all handed to CTAs that are running.
// Each instance has a tile counter; a tile of an instance's sweep w may be
// read once the counter holds every tile of its sweeps 0..w-1 (a sweep reads
// amplitudes that every tile of the previous sweep wrote), and adds one after
// its stores, one tile later (release: barrier, fence, relaxed add; acquire: a relaxed load
// by thread 0 that sees the count, an acq_rel fence, then a barrier, and a
// proxy fence before the bulk copy of a contiguous tile).  Thread 0 takes
// items three ahead and pipelines their lookups (item -> task table, then the
// task's dependency, then a poll of its counter) over the tiles in between,
// so neither the counter nor the lookups sit on a tile's critical path.  Every
// wait is bounded: a dependency that does not arrive in time sets the error
// word, which every other waiting CTA also checks.
//
// The tile work is that of sweep_kernel (qs_sweep.cuh) with every feature
// selected at run time (|+> generation, phase, readout, lambda, adjoint
// accumulations) and the tile kind (contiguous or strided) chosen per item.
#include "qs_sweep.cuh"

namespace qs {

namespace {

constexpr int kQK = 13;  // tile bits (complex64)

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// With a relaxed load that saw the producer's count, the acquire half of the
// synchronisation (loads after it see the producer's stores).
__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Thread 0: wait until done[dep] >= need, giving up after limit ns of device
// time or as soon as another CTA has reported an error; fences on success.
__device__ bool dep_wait(int dep, int need, const unsigned* done, const int* err, uint64_t limit) {
    if (need > 0 && ld_relaxed_u32(done + dep) < (unsigned)need) {
        const uint64_t t0 = globaltimer();
        for (uint32_t it = 0;; ++it) {
            __nanosleep(256);
            if (ld_relaxed_u32(done + dep) >= (unsigned)need) break;
            if ((it & 15u) == 15u) {
                if (*(volatile const int*)err != 0) return false;
                if (globaltimer() - t0 > limit) return false;
            }
        }
    }
    fence_acquire_gpu();
    return true;
}

}  // namespace

template <int NA, int R>
struct QueueCfg {
    using S0 = Sweep<float, kQK, R, NA, 0>;
    using S1 = Sweep<float, kQK, R, NA, 1>;
    static_assert(S0::SMEM_BYTES == S1::SMEM_BYTES && S0::NT == S1::NT, "both tile kinds share one buffer layout");
};

template <int NA, int R>
__global__ void __launch_bounds__(1 << (kQK - R), NA == 1 ? 2 : 1)
    queue_kernel(const SweepTask* __restrict__ tasks, const int64_t* __restrict__ prefix,
                 const int* __restrict__ item_task, const int2* __restrict__ depneed, int64_t total,
                 unsigned long long* __restrict__ next, unsigned* __restrict__ done, int* __restrict__ err,
                 uint64_t limit) {
    constexpr int K = kQK;
    using S0 = typename QueueCfg<NA, R>::S0;
    using C2 = float2;
    constexpr int NT = S0::NT, NS = S0::NS, NW = S0::NW, NSLOT = S0::NSLOT;
    extern __shared__ __align__(128) unsigned char smraw[];
    C2* buf = reinterpret_cast<C2*>(smraw);  // [NA][2^K]
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw + S0::BUF_BYTES);
    double* red = reinterpret_cast<double*>(smraw + S0::BUF_BYTES + 64);
    TileTab* ttab = reinterpret_cast<TileTab*>(smraw + S0::TT_OFF);  // [2]: by tile parity
    __shared__ long long s_item[2];  // [0] the current item, [1] the next one
    __shared__ int s_task[2];        // their tasks
    __shared__ long long s_nxt[2];   // the item after the next, by tile parity (written at release)
    __shared__ int s_flag, s_flag2;
    const uint32_t tid = threadIdx.x;
    C2 v[NA][NS];

    bool pending = false;
    // Every thread arrives once on the barrier (a generated tile loads nothing).
    // Contiguous tiles: thread 0 issues one bulk copy per array (after a proxy
    // fence: the data was written by other CTAs through the generic proxy).
    // Strided tiles: every thread issues 16-byte cp.async copies.
    auto issue = [&](int64_t gt, int ti) {
        const SweepTask& T = tasks[ti];
        if (T.flags & T_GEN) return;
        const int64_t tile = gt - __ldg(prefix + ti);
        if (T.kind == 1) {
            constexpr int EPC = 2;  // complex64 elements per 16-byte copy
            const TMap tm{T.c, T.g0, T.n1, T.g1, K};
            const uint64_t base = tm.base(tile);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const C2* src = reinterpret_cast<const C2*>(a == 0 ? T.psi : T.lam) + base;
                C2* dst = buf + ((size_t)a << K);
                for (int q = tid; q < (1 << K) / EPC; q += NT) {
                    const uint32_t e = (uint32_t)q * EPC;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + e)),
                                 "l"(src + tm.gofs(e))
                                 : "memory");
                }
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(full)) : "memory");
        } else {
            if (tid == 0) {
                fence_proxy_async_all();
                mbar_expect_tx(full, (uint32_t)S0::BUF_BYTES);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const C2* src = reinterpret_cast<const C2*>(a == 0 ? T.psi : T.lam) + ((uint64_t)tile << K);
                    tma_load_1d(buf + ((size_t)a << K), src, (uint32_t)S0::TILE_BYTES, full);
                }
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(full)) : "memory");
            }
        }
        pending = true;
    };

    // Thread 0 signals a tile's completion one tile later (at the next tile's
    // release, when its stores have long drained, so the fence is cheap), and
    // at once before any blocking wait: a CTA never waits on its own tile.
    int pend = -1;
    auto flush = [&]() {
        if (pend >= 0) {
            fence_acquire_gpu();  // acq_rel: the tile's stores before the count
            atomicAdd(done + pend, 1u);
            pend = -1;
        }
    };
    // Thread 0's pipeline of items (software-pipelined so that no load sits on
    // a tile's critical path): i1 the next item with its task t1 and
    // (dep, need) dn1, i2 the one after with its task t2 (loaded during the
    // tile), i3 the one after that (the counter's result, used next tile).
    long long i1 = 0, i2 = 0, i3 = 0;
    int t1 = -1, t2 = -1;
    int2 dn1 = make_int2(0, 0), dn2 = make_int2(0, 0);
    unsigned poll1 = 0;
    if (tid == 0) {
        mbar_init(full, NT);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const long long i0 = (long long)atomicAdd(next, 1ull);
        i1 = (long long)atomicAdd(next, 1ull);
        i2 = (long long)atomicAdd(next, 1ull);
        const int t0 = i0 < total ? __ldg(item_task + i0) : -1;
        t1 = i1 < total ? __ldg(item_task + i1) : -1;
        if (t1 >= 0) dn1 = __ldg(depneed + t1);
        s_item[0] = i0;
        s_item[1] = i1;
        s_task[0] = t0;
        if (t0 >= 0) {
            const int2 dn0 = __ldg(depneed + t0);
            s_flag = dep_wait(dn0.x, dn0.y, done, err, limit) ? 1 : 0;
        } else {
            s_flag = 1;
        }
    }
    __syncthreads();
    int64_t cur = s_item[0], nx = s_item[1];
    int cti = s_task[0];
    bool failed = false;
    if (cur < total) {
        if (s_flag) issue(cur, cti);
        else {
            if (tid == 0) atomicExch(err, 1);
            failed = true;
        }
    }
    uint32_t parity = 0, tpar = 0, kpar = 0;
    while (cur < total && !failed) {
        const SweepTask& T = tasks[cti];
        const int64_t tile = cur - __ldg(prefix + cti);
        const int flags = T.flags, nr = T.nrounds;
        const bool gen = (flags & T_GEN) != 0;
        if (tid == 0) {
            s_task[1] = t1;                                       // the next item's task (known)
            i3 = (long long)atomicAdd(next, 1ull);                // used after the next tile
            t2 = i2 < total ? __ldg(item_task + i2) : -1;         // used at this tile's release
            poll1 = (t1 >= 0 && dn1.y > 0) ? ld_relaxed_u32(done + dn1.x) : 0u;  // used at release
        }
        // the tile's cost table (warp 0), published by the barrier below
        const TileTab& tt = ttab[tpar];
        const TMap tm{T.c, T.g0, T.n1, T.g1, K};
        const uint64_t base = T.kind == 1 ? tm.base(tile) : ((uint64_t)tile << K);
        if (tid < 32 && (flags & T_TAB)) tile_tab_fill(&ttab[tpar], T.tprog, base, tid);
        tpar ^= 1u;
        if (!gen) {
            const int ok = mbar_wait_bounded(full, parity) ? 1 : 0;
            if (!__syncthreads_and(ok)) {  // the copies stay pending on this phase
                if (tid == 0) atomicExch(err, 1);
                failed = true;
                break;
            }
            parity ^= 1u;
            pending = false;
        } else {
            __syncthreads();  // the previous tile's reads of the buffer are done
        }
        const int nti = s_task[1];
        bool nx_issued = false;
        // after the tile's last read of the buffer: load the next item now if
        // the tiles it reads are already written (else after this tile)
        auto release = [&]() {
            if (tid == 0) {
                flush();  // the previous tile
                const bool ok = t1 >= 0 && (dn1.y <= 0 || poll1 >= (unsigned)dn1.y ||
                                            ld_relaxed_u32(done + dn1.x) >= (unsigned)dn1.y);
                if (ok) fence_acquire_gpu();
                s_flag = ok ? 1 : 0;
                s_nxt[kpar] = i2;                        // read by every thread after this tile
                if (t2 >= 0) dn2 = __ldg(depneed + t2);  // used at the next tile's start
            }
            __syncthreads();
            if (s_flag) {
                issue(nx, nti);
                nx_issued = true;
            }
        };
        auto body = [&](auto kc) {
            constexpr int KIND = decltype(kc)::value;
            using S = Sweep<float, K, R, NA, KIND>;
            constexpr int G = S::G;
            int ga = G;
            if (KIND == 1) {
                ga = 1;
                if (G > 1 && K - 1 - S::template rot_lo<(1 < G ? 1 : 0)>() >= T.c) ga = 2;
                if (G > 2 && K - 1 - S::template rot_lo<(2 < G ? 2 : 0)>() >= T.c) ga = 3;
            }
            const int start = (gen && (nr & 1) && ga > 1) ? ga - 1 : 0;
            const int endl = ga == 1 ? 0 : ((start == 0) == ((nr & 1) == 0) ? 0 : ga - 1);
            const int ntr = nr * (ga - 1) + (endl != 0 ? 1 : 0);
            int done_tr = 0;
            int cur_l = start;
            if (gen) {
                const float a0 = (float)T.amp0;
#pragma unroll
                for (int a = 0; a < NA; ++a)
#pragma unroll
                    for (int m = 0; m < NS; ++m) v[a][m] = C2{a0, 0.f};
                if (ntr == 0) release();
            } else {
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
                float gB = 0.f, gG = 0.f;
                const C2* ltab = tab + (int64_t)rd.layer * T.tab_stride;
                if (rd.phase_pre) S::phase_any(cur_l, v, T, tt, tid, ltab, ly.frame, gG);
                const float fabs2 = (float)(ly.fabs * ly.fabs);
                float fpow = 1.f;
                if (NA == 2)
                    for (int i = 0; i < rd.r0; ++i) fpow *= fabs2;
                const float w = (float)ly.w;
                if (cur_l == 0) {
                    for (int g = 0; g < ga; ++g) {
                        if (g != cur_l) { transpose(cur_l, g); cur_l = g; }
                        S::rotate_any(g, v, w, T.c, fabs2, fpow, gB);
                    }
                } else {
                    for (int g = ga - 1; g >= 0; --g) {
                        if (g != cur_l) { transpose(cur_l, g); cur_l = g; }
                        S::rotate_any(g, v, w, T.c, fabs2, fpow, gB);
                    }
                }
                if (rd.phase_post) S::phase_any(cur_l, v, T, tt, tid, ltab, ly.frame, gG);
                if (NA == 2) {
                    warp_sum_to((double)gB, red, 2 * r, NSLOT);
                    warp_sum_to((double)gG, red, 2 * r + 1, NSLOT);
                }
            }
            if (cur_l != 0) transpose(cur_l, 0);

            const uint64_t g_thread = S::template zthread<0>(base, tid, tm);
            C2* arr[2] = {reinterpret_cast<C2*>(T.psi), reinterpret_cast<C2*>(T.lam)};
            if (flags & (T_READOUT | T_WRITE_LAM)) {
                const int ef = T.layers[T.end_layer].frame;
                SlotCost<R> sc;
                sc.template init_tile<typename S::template Map<0>, K - R>(tt, T.cprog[0], tid, ef, T.cost_lo);
                float E = 0.f, P = 0.f, N = 0.f;
                C2* lam = arr[1] + g_thread;
                const bool wl = (flags & T_WRITE_LAM) != 0;
                S::for_slots(tm, [&](int m, uint64_t off) {
                    const C2 x = v[0][m];
                    const int ix = sc.idx(m);
                    const float w2 = x.x * x.x + x.y * x.y;
                    const float cst = (float)(ix + T.cost_lo);
                    E = fmaf(w2, cst, E);
                    N += w2;
                    const bool gnd = (ix == T.gidx);
                    if (gnd) P += w2;
                    if (wl) {
                        const float o = (T.objective == 0) ? cst : (gnd ? 1.f : 0.f);
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
        };
        if (T.kind == 1) body(std::integral_constant<int, 1>{});
        else body(std::integral_constant<int, 0>{});

        if (T.np > 0) {
            const int np = T.np;
            __syncthreads();
            if (tid < (uint32_t)np) {
                double s = 0.0;
                for (int w = 0; w < NW; ++w) s += red[w * NSLOT + tid];
                T.partials[(T.part_base + tile) * np + tid] = s;
            }
        }
        // The tile's completion is signalled at the next tile's release (the
        // barriers in between order every thread's stores before thread 0's
        // fence), or here before a blocking wait.  No barrier otherwise.
        const bool need_issue = nx < total && !nx_issued;
        if (need_issue) {
            __syncthreads();  // the tile's stores, before thread 0's flush
            if (tid == 0) {
                pend = T.dep;
                flush();
                s_flag2 = dep_wait(dn1.x, dn1.y, done, err, limit) ? 1 : 0;
            }
            __syncthreads();
        } else if (tid == 0) {
            pend = T.dep;
        }
        if (tid == 0) {  // advance the pipeline: the next item's successor becomes "next"
            i1 = i2;
            t1 = t2;
            dn1 = dn2;
            i2 = i3;
        }
        cur = nx;
        cti = nti;
        nx = s_nxt[kpar];
        kpar ^= 1u;
        if (need_issue) {
            if (!s_flag2) {
                if (tid == 0) atomicExch(err, 1);
                failed = true;
                break;
            }
            issue(cur, cti);
        }
    }
    __syncthreads();  // the last tile's stores, before thread 0's flush
    if (tid == 0) flush();
    // a copy still in flight must land before the shared memory goes away; a
    // drain that gives up is reported with the sticky status 2
    if (tid == 0 && pending && !mbar_wait_bounded(full, parity)) atomicMax(err, 2);
}

template <int NA, int R>
static size_t queue_smem() {
    return QueueCfg<NA, R>::S0::SMEM_BYTES;
}

template <int NA, int R>
static cudaError_t launch_queue_cfg(const QueueLaunch& Q, int grid, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(queue_kernel<NA, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)queue_smem<NA, R>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    queue_kernel<NA, R><<<grid, 1 << (kQK - R), queue_smem<NA, R>(), st>>>(
        Q.tasks, Q.tile_prefix, Q.item_task, Q.depneed, Q.total_tiles, Q.next, Q.done, Q.err, Q.wait_ns);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_queue(const QueueLaunch& Q, int grid, cudaStream_t st) {
    if (Q.total_tiles <= 0 || Q.ntasks <= 0) return cudaSuccess;
    if (grid > Q.total_tiles) grid = (int)Q.total_tiles;
    if (grid < 1) grid = 1;
    return Q.adjoint ? launch_queue_cfg<2, 5>(Q, grid, st) : launch_queue_cfg<1, 6>(Q, grid, st);
}

template <int NA, int R>
static int queue_grid_cfg() {
    cudaFuncSetAttribute(queue_kernel<NA, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)queue_smem<NA, R>());
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel<NA, R>, 1 << (kQK - R), queue_smem<NA, R>());
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

int queue_grid(int adjoint) { return adjoint ? queue_grid_cfg<2, 5>() : queue_grid_cfg<1, 6>(); }

}  // namespace qs
