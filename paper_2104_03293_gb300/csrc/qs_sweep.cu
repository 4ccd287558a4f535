// Tiled HBM sweep kernel: one read + one write of the state per launch, with
// the x-rotations of K - c tile bits (Eq. twocomponentupdates applied to
// e^{-i beta X}, Sec. III.A.1), the diagonal phase e^{-i gamma H_C}
// (Eq. HC, computed from the bit pattern, no 2^n diagonal), the readout
// (<H_C>, ground probability, norm) and the adjoint accumulations fused in.
//
// Work decomposition (one CTA = one tile of 2^K amplitudes at a time):
//   * tile bits: the c lowest index bits (carried, never rotated here) plus
//     the target run [g0, g0 + K - c); the other n - K bits select the tile.
//   * each thread holds 2^R amplitudes in registers; a "layout" g puts the
//     tile bits [lo_g, lo_g + R) in the register slot index and the other
//     K - R bits in the thread index (lane bits lowest).  Layout 0 has the
//     top R tile bits in registers, so lanes walk the contiguous low bits:
//     global loads and stores are coalesced in layout 0.
//   * a round rotates every target bit once: the register bits of the
//     current layout in registers, then a shared-memory transpose into the
//     next layout, and so on.  Rounds alternate direction (0,1,..) then
//     (..,1,0) so consecutive rounds share the layout at their boundary.
//   * the butterfly is the tangent form a' = a + w (-i b), |w| <= 1, whose
//     scalar factor per rotation (cos beta, or -i sin beta with a bit flip of
//     the whole basis frame) is folded into the layer's phase table.
#include <cuda_runtime.h>

#include "qs_internal.h"

namespace qs {

template <class Real> struct C2T;
template <> struct C2T<float> { using T = float2; };
template <> struct C2T<double> { using T = double2; };

// Shared-memory swizzle: phys(e) = e ^ ((e >> S) & 31), S = max(R, 5).  It is
// linear, so phys(thread part | slot part) = phys(thread) ^ phys(slot), and
// it makes every layout's shared-memory accesses conflict-free for the
// configurations in kernel_cfg (checked on the host by the test-suite).
template <int R> struct Swz {
    static constexpr int S = R > 5 ? R : 5;
    __host__ __device__ static constexpr uint32_t phys(uint32_t e) { return e ^ ((e >> S) & 31u); }
};

template <int K, int R, int g> struct Lay {
    static constexpr int lo = (K - (g + 1) * R) > 0 ? (K - (g + 1) * R) : 0;
    static constexpr int hi = K - g * R;  // rotation range of this group is [max(lo,c), hi)
    __device__ static __forceinline__ uint32_t e_thread(uint32_t tid) {
        return (tid & ((1u << lo) - 1u)) | ((tid >> lo) << (lo + R));
    }
};

// Tile-local index -> global offset for a shape with c carried bits and
// target run starting at g0.
__device__ __forceinline__ uint64_t gofs(uint32_t e, int c, int g0) {
    uint32_t cm = (1u << c) - 1u;
    return (uint64_t)(e & cm) | ((uint64_t)(e >> c) << g0);
}

// Global offset of register slot m in layout 0, whose register bits are the
// tile bits [lo, lo + R), lo = K - R.  Tile bits below c are carried low index
// bits (global bit = tile bit), the rest are targets (global = g0 + tile - c).
// When no register bit is carried (cs = 0, every large shape) the offset is a
// single shift; for_slots hoists that test out of the unrolled slot loop.
struct SlotMap {
    int cs;   // register bits that are carried bits
    int lo;   // K - R
    int sh;   // shift of the target part
    __device__ __forceinline__ SlotMap(int K, int R, int c, int g0) {
        lo = K - R;
        cs = c > lo ? c - lo : 0;
        sh = cs ? g0 : g0 + lo - c;
    }
    __device__ __forceinline__ uint64_t general(int m) const {
        return (((uint64_t)m & ((1ull << cs) - 1ull)) << lo) | (((uint64_t)m >> cs) << sh);
    }
};

template <int NS, class F>
__device__ __forceinline__ void for_slots(const SlotMap& sm, F&& f) {
    if (sm.cs == 0) {
#pragma unroll
        for (int m = 0; m < NS; ++m) f(m, (uint64_t)m << sm.sh);
    } else {
#pragma unroll
        for (int m = 0; m < NS; ++m) f(m, sm.general(m));
    }
}

__device__ __forceinline__ uint64_t tile_base(int64_t t, int c, int g0, int K) {
    int mid = g0 - c;
    uint64_t midm = (mid > 0) ? ((1ull << mid) - 1ull) : 0ull;
    return (((uint64_t)t & midm) << c) | (((uint64_t)t >> mid) << (g0 + K - c));
}

// ---------------------------------------------------------------------------
// Cost program evaluation (see build_cost_prog).  Returns C_out and the
// per-register-bit fields fb (already negated when the frame is flipped).
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ int eval_cost(const int32_t* __restrict__ cp, uint64_t z, int (&fb)[R],
                                         const int32_t*& q) {
    const int nf = __ldg(cp + 1), ne = __ldg(cp + 2), const0 = __ldg(cp + 3), qoff = __ldg(cp + 4);
    const int32_t* t = cp + 12;
    int acc = 0;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) {
        int i = __ldg(t + 2 * k), h = __ldg(t + 2 * k + 1);
        acc += h * (int)((z >> i) & 1ull);
    }
    t += 2 * nf;
#pragma unroll 4
    for (int k = 0; k < ne; ++k) {
        int ij = __ldg(t + 2 * k), J = __ldg(t + 2 * k + 1);
        acc += J * (int)(((z >> (ij & 255)) ^ (z >> (ij >> 8))) & 1ull);
    }
    t += 2 * ne;
#pragma unroll
    for (int b = 0; b < R; ++b) {
        int fb0 = __ldg(t), cnt = __ldg(t + 1);
        t += 2;
        int a2 = 0;
        for (int k = 0; k < cnt; ++k) {
            int j = __ldg(t + 2 * k), J = __ldg(t + 2 * k + 1);
            a2 += J * (int)((z >> j) & 1ull);
        }
        t += 2 * cnt;
        fb[b] = fb0 - 2 * a2;
    }
    q = cp + qoff;
    return const0 - 2 * acc;
}

// Cost of every register slot: idx(m) = C(slot m) - cost_lo, from two
// partial-sum tables over the low / high halves of the register bits plus the
// layout's intra-register coupling table Q.
template <int R>
struct SlotCost {
    static constexpr int R1 = R / 2, R2 = R - R1;
    int plo[1 << R1], phi[1 << R2];
    const int32_t* q;
    __device__ __forceinline__ void init(const int32_t* __restrict__ cp, uint64_t zt, int flip, int cost_lo) {
        int fb[R];
        int cout = eval_cost<R>(cp, zt, fb, q);
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
    __device__ __forceinline__ int idx(int m) const {
        return plo[m & ((1 << R1) - 1)] + phi[m >> R1] + __ldg(q + m);
    }
    // table index, kept inside [0, top] so that no cost can address memory
    // outside the phase table
    __device__ __forceinline__ int tidx(int m, int top) const { return min(max(idx(m), 0), top); }
};

template <class Real> __device__ __forceinline__ Real fma_(Real a, Real b, Real c) { return fma(a, b, c); }

// Sum a per-thread value over the CTA into red[slot] (deterministic order).
template <int NT>
__device__ __forceinline__ void block_sum(double v, double* red_warp, int slot, int nslots) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red_warp[warp * nslots + slot] = v;
}

template <class Real, int K, int R, int NA>
struct SweepImpl {
    using C2 = typename C2T<Real>::T;
    static constexpr int NT = 1 << (K - R);
    static constexpr int NS = 1 << R;
    static constexpr int G = (K + R - 1) / R;
    static constexpr int NW = NT / 32;
    static_assert(K - R >= 5, "a tile needs at least one full warp");
    static_assert(G <= kMaxLayouts, "too many layouts");

    // ---- shared-memory transposes ------------------------------------------
    template <int g>
    __device__ static __forceinline__ void sts(C2* sm, const C2 (&v)[NA][NS], uint32_t tid) {
        using L = Lay<K, R, g>;
        const uint32_t pt = Swz<R>::phys(L::e_thread(tid));
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int m = 0; m < NS; ++m)
                sm[(a << K) + (pt ^ Swz<R>::phys((uint32_t)m << L::lo))] = v[a][m];
    }
    template <int g>
    __device__ static __forceinline__ void lds(const C2* sm, C2 (&v)[NA][NS], uint32_t tid) {
        using L = Lay<K, R, g>;
        const uint32_t pt = Swz<R>::phys(L::e_thread(tid));
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int m = 0; m < NS; ++m)
                v[a][m] = sm[(a << K) + (pt ^ Swz<R>::phys((uint32_t)m << L::lo))];
    }
    __device__ static __forceinline__ void sts_any(int g, C2* sm, const C2 (&v)[NA][NS], uint32_t tid) {
        if (g == 0) sts<0>(sm, v, tid);
        else if (G > 1 && g == 1) sts<(G > 1 ? 1 : 0)>(sm, v, tid);
        else if (G > 2) sts<(G > 2 ? 2 : 0)>(sm, v, tid);
    }
    __device__ static __forceinline__ void lds_any(int g, const C2* sm, C2 (&v)[NA][NS], uint32_t tid) {
        if (g == 0) lds<0>(sm, v, tid);
        else if (G > 1 && g == 1) lds<(G > 1 ? 1 : 0)>(sm, v, tid);
        else if (G > 2) lds<(G > 2 ? 2 : 0)>(sm, v, tid);
    }
    __device__ static __forceinline__ void transpose(int from, int to, C2* sm, C2 (&v)[NA][NS], uint32_t tid) {
        sts_any(from, sm, v, tid);
        __syncthreads();
        lds_any(to, sm, v, tid);
    }

    // ---- rotations ---------------------------------------------------------
    // Forward / inverse butterfly on register bit b of group g:
    //   a' = a + w (-i b),  b' = b + w (-i a).
    // Adjoint: before the butterfly, acc += Im(conj(lam_a) psi_b + conj(lam_b) psi_a),
    // scaled by fpow = |f|^{2r} (r = rotations of this layer applied so far).
    template <int g>
    __device__ static __forceinline__ void rotate(C2 (&v)[NA][NS], Real w, int c, Real fabs2, Real& fpow,
                                                  Real& gacc) {
        using L = Lay<K, R, g>;
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int tb = L::lo + b;
            if (tb < c || tb >= L::hi) continue;
            Real part = 0;
#pragma unroll
            for (int m = 0; m < NS; ++m) {
                if (m & (1 << b)) continue;
                const int m2 = m | (1 << b);
                if (NA == 2) {
                    const C2 pa = v[0][m], pb = v[0][m2], la = v[1][m], lb = v[1][m2];
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
        }
    }
    __device__ static __forceinline__ void rotate_any(int g, C2 (&v)[NA][NS], Real w, int c, Real fabs2,
                                                      Real& fpow, Real& gacc) {
        if (g == 0) rotate<0>(v, w, c, fabs2, fpow, gacc);
        else if (G > 1 && g == 1) rotate<(G > 1 ? 1 : 0)>(v, w, c, fabs2, fpow, gacc);
        else if (G > 2) rotate<(G > 2 ? 2 : 0)>(v, w, c, fabs2, fpow, gacc);
    }

    // ---- phase -------------------------------------------------------------
    // v *= tab[idx(m)] for every slot; adjoint: gacc += C * Im(conj(lam) psi)
    // after the multiplication.
    template <int g>
    __device__ static __forceinline__ void phase(C2 (&v)[NA][NS], const SweepTask& T, uint64_t base, uint32_t tid,
                                                 const C2* __restrict__ tab, int frame, Real& gacc) {
        using L = Lay<K, R, g>;
        const uint64_t zt = base + gofs(L::e_thread(tid), T.c, T.g0);
        const uint64_t fm = frame ? ((1ull << T.n) - 1ull) : 0ull;
        SlotCost<R> sc;
        sc.init(T.cprog[g], zt ^ fm, frame, T.cost_lo);
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
                const Real im = v[1][m].x * v[0][m].y - v[1][m].y * v[0][m].x;
                part = fma_((Real)(ix + T.cost_lo), im, part);
            }
        }
        gacc += part;
    }
    __device__ static __forceinline__ void phase_any(int g, C2 (&v)[NA][NS], const SweepTask& T, uint64_t base,
                                                     uint32_t tid, const C2* tab, int frame, Real& gacc) {
        if (g == 0) phase<0>(v, T, base, tid, tab, frame, gacc);
        else if (G > 1 && g == 1) phase<(G > 1 ? 1 : 0)>(v, T, base, tid, tab, frame, gacc);
        else if (G > 2) phase<(G > 2 ? 2 : 0)>(v, T, base, tid, tab, frame, gacc);
    }
};

template <class Real, int K, int R, int NA>
__global__ void __launch_bounds__(1 << (K - R))
    sweep_kernel(const SweepTask* __restrict__ tasks, const int64_t* __restrict__ prefix, int ntasks, int64_t total) {
    using S = SweepImpl<Real, K, R, NA>;
    using C2 = typename S::C2;
    constexpr int NS = S::NS, NT = S::NT, NW = S::NW;
    constexpr int NSLOT = 2 * kMaxRounds;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* sm = reinterpret_cast<C2*>(smraw);
    __shared__ double red[NW * NSLOT];
    const uint32_t tid = threadIdx.x;
    C2 v[NA][NS];

    for (int64_t gt = blockIdx.x; gt < total; gt += gridDim.x) {
        int ti = 0;
        if (ntasks > 1) {  // last task whose prefix <= gt
            int lo = 0, hi = ntasks - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (__ldg(prefix + mid) <= gt) lo = mid; else hi = mid - 1;
            }
            ti = lo;
        }
        const SweepTask& T = tasks[ti];
        const int64_t tile = gt - __ldg(prefix + ti);
        const int c = T.c, g0 = T.g0, flags = T.flags, nr = T.nrounds;
        const uint64_t base = tile_base(tile, c, g0, K);
        // number of layouts holding targets: groups g with hi_g > c
        int ga = 1;
        if (S::G > 1 && K - R > c) ga = 2;
        if (S::G > 2 && K - 2 * R > c) ga = 3;

        // layout-0 global address of slot 0 and the slot offsets
        const uint64_t g_thread = base + gofs(tid, c, g0);
        const SlotMap smap(K, R, c, g0);
        C2* arr[2] = {reinterpret_cast<C2*>(T.psi), reinterpret_cast<C2*>(T.lam)};

        int cur = 0;
        if (flags & T_GEN) {
            cur = ((nr & 1) && ga > 1) ? ga - 1 : 0;
            const Real a0 = (Real)T.amp0;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int m = 0; m < NS; ++m) v[a][m] = C2{a0, (Real)0};
        } else {
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const C2* src = arr[a] + g_thread;
                for_slots<NS>(smap, [&](int m, uint64_t off) { v[a][m] = src[off]; });
            }
        }

        const C2* tab = reinterpret_cast<const C2*>(T.tab);
        for (int r = 0; r < nr; ++r) {
            const SweepRound rd = T.rounds[r];
            const LayerDev ly = T.layers[rd.layer];
            Real gB = 0, gG = 0;
            const C2* ltab = tab + (int64_t)rd.layer * T.tab_stride;
            if (rd.phase_pre) S::phase_any(cur, v, T, base, tid, ltab, ly.frame, gG);
            const Real fabs2 = (Real)(ly.fabs * ly.fabs);
            Real fpow = 1;
            if (NA == 2) fpow = (Real)pow(ly.fabs, 2.0 * rd.r0);
            const Real w = (Real)ly.w;
            if (cur == 0) {
                for (int g = 0; g < ga; ++g) {
                    if (g != cur) { S::transpose(cur, g, sm, v, tid); cur = g; }
                    S::rotate_any(g, v, w, c, fabs2, fpow, gB);
                }
            } else {
                for (int g = ga - 1; g >= 0; --g) {
                    if (g != cur) { S::transpose(cur, g, sm, v, tid); cur = g; }
                    S::rotate_any(g, v, w, c, fabs2, fpow, gB);
                }
            }
            if (rd.phase_post) S::phase_any(cur, v, T, base, tid, ltab, ly.frame, gG);
            if (NA == 2) {
                block_sum<NT>((double)gB, red, 2 * r, NSLOT);
                block_sum<NT>((double)gG, red, 2 * r + 1, NSLOT);
            }
        }
        if (cur != 0) { S::transpose(cur, 0, sm, v, tid); cur = 0; }

        if (flags & (T_READOUT | T_WRITE_LAM)) {
            const int ef = T.layers[T.end_layer].frame;
            const uint64_t fm = ef ? ((1ull << T.n) - 1ull) : 0ull;
            SlotCost<R> sc;
            sc.init(T.cprog[0], g_thread ^ fm, ef, T.cost_lo);
            Real E = 0, P = 0, N = 0;
            C2* lam = arr[1] + g_thread;
            const bool wl = (flags & T_WRITE_LAM) != 0;
            for_slots<NS>(smap, [&](int m, uint64_t off) {
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
                block_sum<NT>((double)E, red, 0, NSLOT);
                block_sum<NT>((double)P, red, 1, NSLOT);
                block_sum<NT>((double)N, red, 2, NSLOT);
            }
        }
        if (flags & T_STORE) {
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                C2* dst = arr[a] + g_thread;
                for_slots<NS>(smap, [&](int m, uint64_t off) { dst[off] = v[a][m]; });
            }
        }
        const int np = T.np;
        if (np > 0) {
            __syncthreads();
            if (tid < (uint32_t)np) {
                double s = 0.0;
                for (int w = 0; w < NW; ++w) s += red[w * NSLOT + tid];
                T.partials[(T.part_base + tile) * np + tid] = s;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <class Real, int K, int R, int NA>
static cudaError_t launch_one(const SweepLaunch& L, int grid, cudaStream_t st) {
    using C2 = typename C2T<Real>::T;
    const size_t smem = (size_t)NA * ((size_t)1 << K) * sizeof(C2);
    auto kern = sweep_kernel<Real, K, R, NA>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kern<<<grid, 1 << (K - R), smem, st>>>(L.tasks, L.tile_prefix, L.ntasks, L.total_tiles);
    return note_launch(cudaGetLastError());
}

template <class Real, int K, int R, int NA>
static int grid_one() {
    using C2 = typename C2T<Real>::T;
    const size_t smem = (size_t)NA * ((size_t)1 << K) * sizeof(C2);
    auto kern = sweep_kernel<Real, K, R, NA>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 1 << (K - R), smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sms;
}

cudaError_t launch_sweep(const SweepLaunch& L, int grid, cudaStream_t st) {
    const int dtype = L.dtype, adjoint = L.adjoint, K = L.K;
    if (L.total_tiles <= 0) return cudaSuccess;
    if (grid > L.total_tiles) grid = (int)L.total_tiles;
#define QS_LAUNCH(Real, K_, R_, NA_) launch_one<Real, K_, R_, NA_>(L, grid, st)
    if (dtype == 0 && !adjoint && K == 12) return QS_LAUNCH(float, 12, 6, 1);
    if (dtype == 0 && !adjoint && K == 13) return QS_LAUNCH(float, 13, 6, 1);
    if (dtype == 0 && adjoint && K == 12) return QS_LAUNCH(float, 12, 5, 2);
    if (dtype == 0 && adjoint && K == 13) return QS_LAUNCH(float, 13, 5, 2);
    if (dtype == 1 && !adjoint && K == 11) return QS_LAUNCH(double, 11, 5, 1);
    if (dtype == 1 && !adjoint && K == 12) return QS_LAUNCH(double, 12, 5, 1);
    if (dtype == 1 && adjoint && K == 11) return QS_LAUNCH(double, 11, 4, 2);
    if (dtype == 1 && adjoint && K == 12) return QS_LAUNCH(double, 12, 4, 2);
#undef QS_LAUNCH
    return cudaErrorInvalidValue;
}

int sweep_grid(int K, int adjoint, int dtype) {
    if (dtype == 0 && !adjoint && K == 12) return grid_one<float, 12, 6, 1>();
    if (dtype == 0 && !adjoint && K == 13) return grid_one<float, 13, 6, 1>();
    if (dtype == 0 && adjoint && K == 12) return grid_one<float, 12, 5, 2>();
    if (dtype == 0 && adjoint && K == 13) return grid_one<float, 13, 5, 2>();
    if (dtype == 1 && !adjoint && K == 11) return grid_one<double, 11, 5, 1>();
    if (dtype == 1 && !adjoint && K == 12) return grid_one<double, 12, 5, 1>();
    if (dtype == 1 && adjoint && K == 11) return grid_one<double, 11, 4, 2>();
    if (dtype == 1 && adjoint && K == 12) return grid_one<double, 12, 4, 2>();
    return 0;
}

}  // namespace qs
