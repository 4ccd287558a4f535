// Support kernels: per-layer preparation from the angles, deterministic
// reductions, the full-enumeration ground-state search, the plain per-gate
// path, and the on-device Adam update.
#include <atomic>
#include <cmath>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/qs.h"
#include "qs_api_common.h"
#include "qs_internal.h"

namespace qs {

static std::atomic<int64_t> g_launches{0};

cudaError_t note_launch(cudaError_t e, int kernels) {
    if (e == cudaSuccess) g_launches.fetch_add(kernels, std::memory_order_relaxed);
    return e;
}

int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }

template <class Real> struct R2;
template <> struct R2<float> { using T = float2; };
template <> struct R2<double> { using T = double2; };

// ---------------------------------------------------------------------------
// Layer preparation.
//
// Forward layer k is e^{-i beta H_D} e^{-i gamma H_C} (Eq. QAOA_state).  The
// mixer acts as n x-rotations Rx = c - i s X (c = cos beta, s = sin beta).
// The sweep kernel applies the unnormalised butterfly (1 - i w X):
//   |s| <= |c|:  Rx = c (1 - i t X),            w = t = s / c          (var 0)
//   |s| >  |c|:  Rx = (-i s) X (1 + i u X),     w = -u, u = c / s      (var 1)
// var 1 also applies X to every qubit of the layer: the stored array then
// holds psi in the bit-flipped frame, tracked as a per-layer frame bit.  The
// scalar f per rotation is |f| = 1 / sqrt(1 + w^2) computed from the float w
// that the kernel uses, so the product of a layer stays exactly unitary, with
// phase sign(c) (var 0) or -i sign(s) (var 1).  f^n goes into the phase table
//   tab[k][j] = f^n exp(-i gamma (cost_lo + j) 2^-shift).
// Reverse (mode 1) uses Rx(-beta) = c + i s X: w -> -w, f -> conj(f), and the
// table holds f_rev^n exp(+i gamma C).  Plain (mode 2): table = exp(-i gamma C),
// layers carry (c, s) for the normalised rotation.
// ---------------------------------------------------------------------------
template <class Real>
__device__ void prep_layers(const double* gamma, const double* beta, int p, int nphys, int cost_lo, int range,
                            int shift, const int* frame0, int mode, LayerDev* layers, void* tabv, int stride) {
    using C2 = typename R2<Real>::T;
    C2* tab = reinterpret_cast<C2*>(tabv);
    __shared__ int s_frame[QS_MAX_LAYERS_PREP + 1];
    __shared__ double s_fre[QS_MAX_LAYERS_PREP], s_fim[QS_MAX_LAYERS_PREP];
    const double scale = ldexp(1.0, -shift);
    if (threadIdx.x == 0) {
        int fr = frame0 ? *frame0 : 0;
        for (int k = 0; k < p; ++k) {
            double s, c;
            sincos(beta[k], &s, &c);
            LayerDev L;
            L.var = fabs(s) > fabs(c) ? 1 : 0;
            double wd = L.var ? -(c / s) : (s / c);
            if (mode == 1) wd = -wd;
            // the complex64 kernels use w rounded to float: f must match it
            const double wq = (sizeof(Real) == 4) ? (double)(float)wd : wd;
            L.w = wq;
            L.fabs = 1.0 / sqrt(1.0 + wq * wq);
            L.c = c;
            L.s = s;
            L.frame = fr;
            // layer scalar f^n
            double mag = pow(L.fabs, (double)nphys), re, im;
            if (mode == 2) { re = 1.0; im = 0.0; }
            else if (!L.var) { double sg = (c < 0 && (nphys & 1)) ? -1.0 : 1.0; re = sg * mag; im = 0.0; }
            else {
                // (-i sign(s))^n forward, (+i sign(s))^n reverse
                int q = nphys & 3;                       // i^q phase of (+-i)^n
                double sgn = (s < 0) ? -1.0 : 1.0;
                double sgnn = (nphys & 1) ? sgn : 1.0;    // sign(s)^n
                int e = (mode == 1) ? q : ((4 - q) & 3); // (+i)^n or (-i)^n = i^{-n}
                double cr = (e == 0) ? 1.0 : (e == 2 ? -1.0 : 0.0);
                double ci = (e == 1) ? 1.0 : (e == 3 ? -1.0 : 0.0);
                re = sgnn * mag * cr; im = sgnn * mag * ci;
            }
            s_fre[k] = re; s_fim[k] = im;
            layers[k] = L;
            s_frame[k] = fr;
            if (mode != 2 && L.var) fr ^= 1;
        }
        LayerDev E;
        E.w = 0.0; E.frame = fr; E.fabs = 1.0; E.c = 1.f; E.s = 0.f; E.var = 0;
        layers[p] = E;
    }
    __syncthreads();
    const double sgn = (mode == 1) ? 1.0 : -1.0;
    for (int k = 0; k < p; ++k) {
        const double g = gamma[k] * scale;
        const double fr = s_fre[k], fi = s_fim[k];
        for (int j = threadIdx.x; j < range; j += blockDim.x) {
            double sn, cs;
            sincos(sgn * g * (double)(cost_lo + j), &sn, &cs);
            C2 v;
            v.x = (Real)(fr * cs - fi * sn);
            v.y = (Real)(fr * sn + fi * cs);
            tab[(int64_t)k * stride + j] = v;
        }
    }
}

template <class Real>
__global__ void prep_kernel(const double* gamma, const double* beta, int p, int nphys, int cost_lo, int range,
                            int shift, const int* frame0, int mode, LayerDev* layers, void* tab, int stride) {
    prep_layers<Real>(gamma, beta, p, nphys, cost_lo, range, shift, frame0, mode, layers, tab, stride);
}

template <class Real>
__global__ void prep_batch_kernel(const PrepTask* tasks) {
    const PrepTask t = tasks[blockIdx.x];
    prep_layers<Real>(t.gamma, t.beta, t.p, t.nphys, t.cost_lo, t.range, t.shift, t.frame0, t.reverse, t.layers,
                      t.tab, t.tab_stride);
}

cudaError_t launch_prep(int dtype, int p, const double* gamma, const double* beta, int nphys, int cost_lo,
                        int range, int shift, const int* frame0, int mode, LayerDev* layers, void* tab,
                        int tab_stride, cudaStream_t st) {
    if (p > QS_MAX_LAYERS_PREP) return cudaErrorInvalidValue;
    if (dtype == 0)
        prep_kernel<float><<<1, 256, 0, st>>>(gamma, beta, p, nphys, cost_lo, range, shift, frame0, mode, layers,
                                             tab, tab_stride);
    else
        prep_kernel<double><<<1, 256, 0, st>>>(gamma, beta, p, nphys, cost_lo, range, shift, frame0, mode, layers,
                                              tab, tab_stride);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_prep_batch(int dtype, const PrepTask* tasks, int ntasks, cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    if (dtype == 0) prep_batch_kernel<float><<<ntasks, 256, 0, st>>>(tasks);
    else prep_batch_kernel<double><<<ntasks, 256, 0, st>>>(tasks);
    return note_launch(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Deterministic reduction of per-tile partials: one block per task, fixed
// strided order per thread, fixed tree across threads.
// ---------------------------------------------------------------------------
__global__ void reduce_kernel(const ReduceTask* tasks) {
    const ReduceTask t = tasks[blockIdx.x];
    __shared__ double sh[256];
    for (int s = 0; s < t.count; ++s) {
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < t.ntiles; i += blockDim.x) acc += t.partials[i * t.np + t.off + s];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (t.accumulate) t.out[s] += t.mult * sh[0];
            else t.out[s] = t.mult * sh[0];
        }
        __syncthreads();
    }
}

cudaError_t launch_reduce(const ReduceTask* tasks, int ntasks, cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    reduce_kernel<<<ntasks, 256, 0, st>>>(tasks);
    return note_launch(cudaGetLastError());
}

// Segmented: block b runs tasks [seg[b], seg[b + 1]) one after another, so
// tasks that add into the same output are summed in a fixed order by one
// block (no two blocks write one output).
__global__ void reduce_seg_kernel(const ReduceTask* tasks, const int* seg) {
    __shared__ double sh[256];
    for (int k = seg[blockIdx.x]; k < seg[blockIdx.x + 1]; ++k) {
        const ReduceTask t = tasks[k];
        for (int s = 0; s < t.count; ++s) {
            double acc = 0.0;
            for (int64_t i = threadIdx.x; i < t.ntiles; i += blockDim.x) acc += t.partials[i * t.np + t.off + s];
            sh[threadIdx.x] = acc;
            __syncthreads();
            for (int w = blockDim.x / 2; w > 0; w >>= 1) {
                if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                if (t.accumulate) t.out[s] += t.mult * sh[0];
                else t.out[s] = t.mult * sh[0];
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_reduce_seg(const ReduceTask* tasks, const int* seg, int nseg, cudaStream_t st) {
    if (nseg <= 0) return cudaSuccess;
    reduce_seg_kernel<<<nseg, 256, 0, st>>>(tasks, seg);
    return note_launch(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Full enumeration (the t_FE ground-state search of Table III): every thread
// evaluates 64 consecutive basis states (register bits = qubits 0..5) with
// the cost-program decomposition; integer min / max / lowest argmin / count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int enum_eval_all(const int32_t* __restrict__ cp, uint64_t zt, int (&cst)[64]) {
    const int nf = __ldg(cp + 1), ne = __ldg(cp + 2), const0 = __ldg(cp + 3), qoff = __ldg(cp + 4);
    const int32_t* t = cp + 12;
    int acc = 0;
    for (int k = 0; k < nf; ++k) acc += __ldg(t + 2 * k + 1) * (int)((zt >> __ldg(t + 2 * k)) & 1ull);
    t += 2 * nf;
    for (int k = 0; k < ne; ++k) {
        int ij = __ldg(t + 2 * k), J = __ldg(t + 2 * k + 1);
        acc += J * (int)(((zt >> (ij & 255)) ^ (zt >> (ij >> 8))) & 1ull);
    }
    t += 2 * ne;
    int fb[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        int fb0 = __ldg(t), cnt = __ldg(t + 1);
        t += 2;
        int a2 = 0;
        for (int k = 0; k < cnt; ++k) a2 += __ldg(t + 2 * k + 1) * (int)((zt >> __ldg(t + 2 * k)) & 1ull);
        t += 2 * cnt;
        fb[b] = fb0 - 2 * a2;
    }
    const int cout = const0 - 2 * acc;
    int lin[64];
    int s0 = cout;
#pragma unroll
    for (int b = 0; b < 6; ++b) s0 += fb[b];
    lin[0] = s0;
#pragma unroll
    for (int b = 0; b < 6; ++b)
#pragma unroll
        for (int k = 0; k < (1 << b); ++k) lin[k | (1 << b)] = lin[k] - 2 * fb[b];
#pragma unroll
    for (int m = 0; m < 64; ++m) cst[m] = lin[m] + __ldg(cp + qoff + m);
    return 0;
}

struct EnumAcc {
    long long mn, mx, arg, cnt;
};

__device__ __forceinline__ void enum_merge(EnumAcc& a, const EnumAcc& b) {
    if (b.mn < a.mn) { a.mn = b.mn; a.arg = b.arg; a.cnt = b.cnt; }
    else if (b.mn == a.mn) { a.cnt += b.cnt; if (b.arg < a.arg) a.arg = b.arg; }
    if (b.mx > a.mx) a.mx = b.mx;
}

__global__ void enumerate_kernel(const int32_t* __restrict__ cp, int n, long long* scratch) {
    const uint64_t N = 1ull << n;
    const uint64_t nblk = (N + 63) >> 6;
    EnumAcc a{0x7fffffffffffffffLL, -0x7fffffffffffffffLL, 0x7fffffffffffffffLL, 0};
    const int valid = n >= 6 ? 64 : (1 << n);
    for (uint64_t blk = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; blk < nblk;
         blk += (uint64_t)gridDim.x * blockDim.x) {
        int cst[64];
        const uint64_t zt = blk << 6;
        enum_eval_all(cp, zt, cst);
#pragma unroll
        for (int m = 0; m < 64; ++m) {
            if (m >= valid) break;
            const long long c = cst[m];
            if (c < a.mn) { a.mn = c; a.arg = (long long)(zt + m); a.cnt = 1; }
            else if (c == a.mn) a.cnt++;  // ascending z within a thread: first hit is lowest
            if (c > a.mx) a.mx = c;
        }
    }
    __shared__ EnumAcc sh[256];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            EnumAcc x = sh[threadIdx.x];
            enum_merge(x, sh[threadIdx.x + w]);
            sh[threadIdx.x] = x;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[4 * blockIdx.x + 0] = sh[0].mn;
        scratch[4 * blockIdx.x + 1] = sh[0].mx;
        scratch[4 * blockIdx.x + 2] = sh[0].arg;
        scratch[4 * blockIdx.x + 3] = sh[0].cnt;
    }
}

__global__ void enumerate_final(const long long* scratch, int nblocks, long long* out) {
    __shared__ EnumAcc sh[256];
    EnumAcc a{0x7fffffffffffffffLL, -0x7fffffffffffffffLL, 0x7fffffffffffffffLL, 0};
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        EnumAcc b{scratch[4 * i], scratch[4 * i + 1], scratch[4 * i + 2], scratch[4 * i + 3]};
        enum_merge(a, b);
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            EnumAcc x = sh[threadIdx.x];
            enum_merge(x, sh[threadIdx.x + w]);
            sh[threadIdx.x] = x;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0].mn; out[1] = sh[0].mx; out[2] = sh[0].arg; out[3] = sh[0].cnt;
    }
}

cudaError_t launch_enumerate(const int32_t* cprog, int n, int64_t* scratch, int64_t nscratch, int64_t* out,
                             cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nblk = ((1ll << n) + 63) >> 6;
    int64_t blocks = (nblk + 255) / 256;
    int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks > nscratch / 4) blocks = nscratch / 4;
    if (blocks < 1) return cudaErrorInvalidValue;
    enumerate_kernel<<<(int)blocks, 256, 0, st>>>(cprog, n, reinterpret_cast<long long*>(scratch));
    enumerate_final<<<1, 256, 0, st>>>(reinterpret_cast<long long*>(scratch), (int)blocks,
                                       reinterpret_cast<long long*>(out));
    return note_launch(cudaGetLastError(), 2);
}

// ---------------------------------------------------------------------------
// Plain path: one launch per gate (Eq. twocomponentupdates per qubit, one
// diagonal phase launch per layer), normalised rotations, no fusion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int plain_cost(const int32_t* __restrict__ terms, int nf, int ne, int const0,
                                          uint64_t z) {
    int acc = 0;
    for (int k = 0; k < nf; ++k) acc += __ldg(terms + 2 * k + 1) * (int)((z >> __ldg(terms + 2 * k)) & 1ull);
    const int32_t* t = terms + 2 * nf;
    for (int k = 0; k < ne; ++k) {
        int ij = __ldg(t + 2 * k), J = __ldg(t + 2 * k + 1);
        acc += J * (int)(((z >> (ij & 255)) ^ (z >> (ij >> 8))) & 1ull);
    }
    return const0 - 2 * acc;
}

template <class Real>
__global__ void plain_init_kernel(typename R2<Real>::T* psi, uint64_t N, Real a) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
        psi[i] = typename R2<Real>::T{a, (Real)0};
}

template <class Real>
__global__ void plain_phase_kernel(typename R2<Real>::T* psi, uint64_t N, const int32_t* terms, int nf, int ne,
                                   int const0, const LayerDev* layer, const typename R2<Real>::T* tab, int cost_lo,
                                   int range) {
    const uint64_t fm = layer->frame ? (N - 1) : 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int c = plain_cost(terms, nf, ne, const0, i ^ fm);
        const auto f = tab[min(max(c - cost_lo, 0), range - 1)];  // never outside the table
        const auto x = psi[i];
        psi[i] = typename R2<Real>::T{x.x * f.x - x.y * f.y, x.x * f.y + x.y * f.x};
    }
}

// Pairs (z, z + 2^q), bit q of z clear: [a', b'] = [[c, -is], [-is, c]] [a, b].
template <class Real>
__global__ void plain_rx_kernel(typename R2<Real>::T* psi, uint64_t N, int q, const LayerDev* layer) {
    const Real c = (Real)layer->c, s = (Real)layer->s;
    const uint64_t half = N >> 1, lowm = (1ull << q) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < half;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t z = ((i & ~lowm) << 1) | (i & lowm);
        const auto a = psi[z], b = psi[z | (1ull << q)];
        psi[z] = typename R2<Real>::T{c * a.x + s * b.y, c * a.y - s * b.x};
        psi[z | (1ull << q)] = typename R2<Real>::T{c * b.x + s * a.y, c * b.y - s * a.x};
    }
}

template <class Real>
__global__ void plain_readout_kernel(const typename R2<Real>::T* psi, uint64_t N, const int32_t* terms, int nf,
                                     int ne, int const0, int cmin, const int* frame, double* partials) {
    const uint64_t fm = (frame && *frame) ? (N - 1) : 0;
    double E = 0, P = 0, Nn = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int c = plain_cost(terms, nf, ne, const0, i ^ fm);
        const auto x = psi[i];
        const double w = (double)x.x * x.x + (double)x.y * x.y;
        E += w * c;
        Nn += w;
        if (c == cmin) P += w;
    }
    __shared__ double sh[3][256];
    sh[0][threadIdx.x] = E; sh[1][threadIdx.x] = P; sh[2][threadIdx.x] = Nn;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) partials[blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

static int plain_grid(uint64_t work) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (work + 255) / 256;
    uint64_t cap = (uint64_t)sms * 16;
    return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

int64_t plain_readout_blocks(int nphys) {
    uint64_t N = 1ull << nphys;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (N + 255) / 256, cap = (uint64_t)sms * 8;
    return (int64_t)(blocks < cap ? blocks : cap);
}

cudaError_t launch_plain_init(int dtype, void* psi, int nphys, cudaStream_t st) {
    const uint64_t N = 1ull << nphys;
    const double a = pow(2.0, -0.5 * nphys);
    if (dtype == 0) plain_init_kernel<float><<<plain_grid(N), 256, 0, st>>>((float2*)psi, N, (float)a);
    else plain_init_kernel<double><<<plain_grid(N), 256, 0, st>>>((double2*)psi, N, a);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_plain_phase(int dtype, void* psi, int nphys, const int32_t* terms, int nf, int ne, int const0,
                               const LayerDev* layer, const void* tab, int cost_lo, int range, cudaStream_t st) {
    const uint64_t N = 1ull << nphys;
    if (dtype == 0)
        plain_phase_kernel<float><<<plain_grid(N), 256, 0, st>>>((float2*)psi, N, terms, nf, ne, const0, layer,
                                                                 (const float2*)tab, cost_lo, range);
    else
        plain_phase_kernel<double><<<plain_grid(N), 256, 0, st>>>((double2*)psi, N, terms, nf, ne, const0, layer,
                                                                  (const double2*)tab, cost_lo, range);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_plain_rx(int dtype, void* psi, int nphys, int q, const LayerDev* layer, cudaStream_t st) {
    const uint64_t N = 1ull << nphys;
    if (dtype == 0) plain_rx_kernel<float><<<plain_grid(N / 2), 256, 0, st>>>((float2*)psi, N, q, layer);
    else plain_rx_kernel<double><<<plain_grid(N / 2), 256, 0, st>>>((double2*)psi, N, q, layer);
    return note_launch(cudaGetLastError());
}

cudaError_t launch_plain_readout(int dtype, const void* psi, int nphys, const int32_t* terms, int nf, int ne,
                                 int const0, int cmin, const int* frame, double* partials, int64_t nblocks,
                                 cudaStream_t st) {
    const uint64_t N = 1ull << nphys;
    if (dtype == 0)
        plain_readout_kernel<float><<<(int)nblocks, 256, 0, st>>>((const float2*)psi, N, terms, nf, ne, const0,
                                                                  cmin, frame, partials);
    else
        plain_readout_kernel<double><<<(int)nblocks, 256, 0, st>>>((const double2*)psi, N, terms, nf, ne, const0,
                                                                   cmin, frame, partials);
    return note_launch(cudaGetLastError());
}

// In-place reversal psi[z] <-> psi[~z]: brings a flipped frame back to the
// canonical basis order.
template <class Real>
__global__ void flip_kernel(typename R2<Real>::T* psi, uint64_t N) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N / 2;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = (N - 1) ^ i;
        const auto a = psi[i], b = psi[j];
        psi[i] = b;
        psi[j] = a;
    }
}

cudaError_t launch_flip_all(int dtype, void* psi, int nphys, cudaStream_t st) {
    const uint64_t N = 1ull << nphys;
    if (dtype == 0) flip_kernel<float><<<plain_grid(N / 2), 256, 0, st>>>((float2*)psi, N);
    else flip_kernel<double><<<plain_grid(N / 2), 256, 0, st>>>((double2*)psi, N);
    return note_launch(cudaGetLastError());
}

__global__ void set_frame_kernel(int* frame, const LayerDev* layers, int p) { *frame = layers[p].frame; }

cudaError_t launch_set_frame(int* frame_dev, const LayerDev* layers, int p, cudaStream_t st) {
    set_frame_kernel<<<1, 1, 0, st>>>(frame_dev, layers, p);
    return note_launch(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Adam (bias-corrected, minimisation) over a flat angle vector.
// ---------------------------------------------------------------------------
__global__ void adam_kernel(double* theta, const double* grad, double* m, double* v, int64_t count, const int* step,
                            double lr, double b1, double b2, double eps) {
    const int t = *step;
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double g = grad[i];
        const double mi = b1 * m[i] + (1.0 - b1) * g;
        const double vi = b2 * v[i] + (1.0 - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
    }
}

cudaError_t launch_adam(double* theta, const double* grad, double* m, double* v, int64_t count, const int* step,
                        double lr, double b1, double b2, double eps, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int blocks = (int)((count + 255) / 256);
    adam_kernel<<<blocks, 256, 0, st>>>(theta, grad, m, v, count, step, lr, b1, b2, eps);
    return note_launch(cudaGetLastError());
}

__global__ void step_inc_kernel(int* step) { *step += 1; }

cudaError_t launch_step_inc(int* step, cudaStream_t st) {
    step_inc_kernel<<<1, 1, 0, st>>>(step);
    return note_launch(cudaGetLastError());
}

__global__ void copy_kernel(const double* s, double* d, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

cudaError_t launch_gather_grad(const double* dsrc, double* ddst, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    copy_kernel<<<(int)((count + 255) / 256), 256, 0, st>>>(dsrc, ddst, count);
    return note_launch(cudaGetLastError());
}


// ---------------------------------------------------------------------------
// Allocation-free ground-state enumeration.
//
// The same enumeration kernels as above, with their scratch (the cost
// program, the per-block partials and the four result words) in one
// file-scope device array instead of memory from cudaMalloc, for callers
// that cannot allocate device memory.  The array is shared by every call in
// the process: calls that overlap on the GPU (concurrent host threads, or
// several streams) race on it.  No word of it has to start at zero: a call
// writes the cost program, every partial slot it reads and the result words
// before reading them.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNaMaxBlocks = 2048;                         // partial slots (4 int64 each)
constexpr int kNaProgWords = 8448;                         // int32 words of cost program
constexpr size_t kNaPartOff = 256;                         // bytes; result words at 0
constexpr size_t kNaProgOff = kNaPartOff + (size_t)kNaMaxBlocks * 4 * sizeof(int64_t);
constexpr size_t kNaBytes = kNaProgOff + (size_t)kNaProgWords * sizeof(int32_t);
static_assert(kNaBytes == QS_NOALLOC_SCRATCH_BYTES, "scratch size disagrees with qs.h");

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
int na_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "qs_enumerate_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(QS_EINVAL, "qs_enumerate_noalloc: device %d >= %d", dev, kNaMaxDevices);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_error(e, "qs_enumerate_noalloc: cudaGetSymbolAddress");
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return QS_OK;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" int qs_enumerate_noalloc(int n, const double* hfield, int n_edges, const int32_t* edges, const double* J,
                                    void* cuda_stream, int64_t* cmin, int64_t* cmax, int64_t* argmin,
                                    int64_t* ground_count, int* scale_shift) {
    // Validation: the rules of qs_set_ising, checked without host allocation.
    if (n < 1 || n > QS_NOALLOC_MAX_QUBITS)
        return set_error(QS_EINVAL, "qs_enumerate_noalloc: n = %d outside [1, %d]", n, QS_NOALLOC_MAX_QUBITS);
    if (n_edges < 0 || n_edges > QS_MAX_EDGES)
        return set_error(QS_EINVAL, "qs_enumerate_noalloc: n_edges = %d outside [0, %d]", n_edges, QS_MAX_EDGES);
    if (!hfield) return set_error(QS_EINVAL, "qs_enumerate_noalloc: hfield is NULL");
    if (n_edges > 0 && (!edges || !J)) return set_error(QS_EINVAL, "qs_enumerate_noalloc: edges or J is NULL");
    uint64_t seen[QS_NOALLOC_MAX_QUBITS] = {};
    for (int e = 0; e < n_edges; ++e) {
        const int i = edges[2 * e], j = edges[2 * e + 1];
        if (i < 0 || j < 0 || i >= n || j >= n) return set_error(QS_EINVAL, "qs_enumerate_noalloc: edge %d out of range", e);
        if (i >= j) return set_error(QS_EINVAL, "qs_enumerate_noalloc: edge %d does not satisfy i < j", e);
        if ((seen[i] >> j) & 1) return set_error(QS_EINVAL, "qs_enumerate_noalloc: duplicate edge %d", e);
        seen[i] |= 1ull << j;
        if (!std::isfinite(J[e])) return set_error(QS_EINVAL, "qs_enumerate_noalloc: non-finite coupling %d", e);
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(hfield[i])) return set_error(QS_EINVAL, "qs_enumerate_noalloc: non-finite field %d", i);
    int shift = -1;
    for (int s = 0; s <= 3 && shift < 0; ++s) {
        const double sc = std::ldexp(1.0, s);
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) ok = std::nearbyint(hfield[i] * sc) == hfield[i] * sc;
        for (int e = 0; e < n_edges && ok; ++e) ok = std::nearbyint(J[e] * sc) == J[e] * sc;
        if (ok) shift = s;
    }
    if (shift < 0) return set_error(QS_ENOTINT, "qs_enumerate_noalloc: weights are not integer multiples of 2^-s, s <= 3");
    const double sc = std::ldexp(1.0, shift);
    double bound = 0;
    for (int i = 0; i < n; ++i) bound += std::fabs(hfield[i] * sc);
    for (int e = 0; e < n_edges; ++e) bound += std::fabs(J[e] * sc);
    if (bound > (double)(1 << 24)) return set_error(QS_ENOTINT, "qs_enumerate_noalloc: cost range exceeds 2^24 units");
    auto hi = [&](int i) { return (int32_t)(hfield[i] * sc); };
    auto Ji = [&](int e) { return (int32_t)(J[e] * sc); };

    // Cost program with register qubits 0..5 (the layout enum_eval_all reads):
    // header, outside fields, outside couplings, per-register field and
    // coupling lists, and the 64-entry table of register-register couplings.
    int32_t prog[kNaProgWords];
    int len = 12;
    auto push = [&](int32_t v) {
        if (len < kNaProgWords) prog[len] = v;
        ++len;
    };
    const int nreg = n < 6 ? n : 6;
    for (int b = 0; b < 12; ++b) prog[b] = 0;
    prog[0] = 6;
    for (int b = 0; b < 6; ++b) prog[5 + b] = b < nreg ? b : -1;
    int64_t const0 = 0;
    int nf = 0, ne = 0;
    for (int i = nreg; i < n; ++i) {
        if (hi(i) == 0) continue;
        push(i);
        push(hi(i));
        const0 += hi(i);
        ++nf;
    }
    for (int e = 0; e < n_edges; ++e) {
        const int i = edges[2 * e], j = edges[2 * e + 1];
        if (i < nreg || j < nreg || Ji(e) == 0) continue;
        push(i | (j << 8));
        push(Ji(e));
        const0 += Ji(e);
        ++ne;
    }
    for (int b = 0; b < 6; ++b) {
        if (b >= nreg) {
            push(0);
            push(0);
            continue;
        }
        int64_t fb0 = hi(b);
        int cnt = 0;
        for (int e = 0; e < n_edges; ++e) {
            const int i = edges[2 * e], j = edges[2 * e + 1];
            if ((i == b && j >= nreg) || (j == b && i >= nreg)) cnt += Ji(e) != 0;
        }
        const int at = len;
        push(0);
        push(cnt);
        for (int e = 0; e < n_edges; ++e) {
            const int i = edges[2 * e], j = edges[2 * e + 1];
            int other = -1;
            if (i == b && j >= nreg) other = j;
            else if (j == b && i >= nreg) other = i;
            if (other < 0 || Ji(e) == 0) continue;
            fb0 += Ji(e);
            push(other);
            push(Ji(e));
        }
        if (at < kNaProgWords) prog[at] = (int32_t)fb0;
    }
    const int qoff = len;
    for (int m = 0; m < 64; ++m) {
        int64_t q = 0;
        for (int e = 0; e < n_edges; ++e) {
            const int i = edges[2 * e], j = edges[2 * e + 1];
            if (i >= nreg || j >= nreg) continue;
            q += (int64_t)Ji(e) * (((m >> i) & 1) ? -1 : 1) * (((m >> j) & 1) ? -1 : 1);
        }
        push((int32_t)q);
    }
    if (len > kNaProgWords)
        return set_error(QS_EINVAL, "qs_enumerate_noalloc: cost program needs %d words, the scratch holds %d", len,
                         kNaProgWords);
    prog[1] = nf;
    prog[2] = ne;
    prog[3] = (int32_t)const0;
    prog[4] = qoff;

    unsigned char* base = nullptr;
    if (int rc = na_scratch(&base)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int32_t* dprog = reinterpret_cast<int32_t*>(base + kNaProgOff);
    int64_t* dpart = reinterpret_cast<int64_t*>(base + kNaPartOff);
    int64_t* dout = reinterpret_cast<int64_t*>(base);
    // pageable source: the copy has been staged when cudaMemcpyAsync returns
    cudaError_t e = cudaMemcpyAsync(dprog, prog, (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "qs_enumerate_noalloc: program upload");
    e = launch_enumerate(dprog, n, dpart, (int64_t)kNaMaxBlocks * 4, dout, st);
    if (e != cudaSuccess) return cuda_error(e, "qs_enumerate_noalloc: enumerate launch");
    int64_t res[4];
    e = cudaMemcpyAsync(res, dout, sizeof res, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "qs_enumerate_noalloc: enumerate");
    if (cmin) *cmin = res[0];
    if (cmax) *cmax = res[1];
    if (argmin) *argmin = res[2];
    if (ground_count) *ground_count = res[3];
    if (scale_shift) *scale_shift = shift;
    return QS_OK;
}
