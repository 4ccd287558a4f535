// C ABI of include/qs.h: single-state handles.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <complex>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/qs.h"
#include "qs_api_common.h"
#include "qs_layout.h"
#include "qs_pair.h"

namespace qs {

thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_error(cudaError_t e, const char* where) {
    return set_error(QS_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// DevBuf / Uploader
// ---------------------------------------------------------------------------
int DevBuf::reserve(size_t bytes) {
    if (bytes <= cap) return QS_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        return set_error(QS_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    cap = want;
    return QS_OK;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
}

Uploader::~Uploader() {
    if (ev) cudaEventDestroy(ev);
    if (host) cudaFreeHost(host);
    dev.release();
}

int Uploader::upload(const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return QS_OK;
    if (ev) {
        cudaError_t e = cudaEventSynchronize(ev);
        if (e != cudaSuccess) return cuda_error(e, "upload wait");
    } else {
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_error(e, "cudaEventCreate");
    }
    if (bytes > host_cap) {
        if (host) cudaFreeHost(host);
        host = nullptr;
        host_cap = 0;
        size_t want = bytes * 2;
        cudaError_t e = cudaMallocHost(&host, want);
        if (e != cudaSuccess) return set_error(QS_ENOMEM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
        host_cap = want;
    }
    if (bytes > dev.cap) {
        // the device copy may still be read by queued work: drain first
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_error(e, "upload grow");
    }
    if (int rc = dev.reserve(bytes)) return rc;
    std::memcpy(host, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dev.ptr, host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "upload");
    e = cudaEventRecord(ev, st);
    if (e != cudaSuccess) return cuda_error(e, "upload event");
    return QS_OK;
}

// ---------------------------------------------------------------------------
// Instance: validated Ising + device cost programs + ground-state data.
// ---------------------------------------------------------------------------
int Instance::set(int n_, int nphys_, int dtype_, const double* hfield, int n_edges, const int32_t* edges,
                  const double* J, cudaStream_t st, DevBuf& enum_scratch, ShapeRule rule) {
    IsingInt I;
    std::string err;
    int rc = validate_ising(n_, hfield, n_edges, edges, J, I, err);
    if (rc) return set_error(rc == 5 ? QS_ENOTINT : QS_EINVAL, "qs_set_ising: %s", err.c_str());
    n = n_;
    nphys = nphys_;
    dtype = dtype_;
    shift = I.shift;
    // pad h to nphys qubits (idle qubits carry no terms)
    std::vector<int32_t> h(nphys, 0);
    for (int i = 0; i < n; ++i) h[i] = I.h[i];
    std::vector<int32_t> blob;
    auto add = [&](const std::vector<int32_t>& p) {
        size_t off = blob.size();
        blob.insert(blob.end(), p.begin(), p.end());
        while (blob.size() % 4) blob.push_back(0);
        return off;
    };
    // per shape: the tile program; per kernel layout: the layout program
    // (the tile bits of its register-slot and thread-index bits)
    for (int cfgi = 0; cfgi < 2; ++cfgi) {
        const KernelCfg cfg = kernel_cfg(dtype, cfgi == 1);
        shapes[cfgi] = make_shapes(nphys, cfg, page_bit_for(dtype), rule);
        for (size_t s = 0; s < shapes[cfgi].size(); ++s) {
            const Shape& sh = shapes[cfgi][s];
            tprog_off[cfgi][s] = add(build_tile_prog(sh, h, I.ei, I.ej, I.J));
            const LayoutTab L = make_layout(sh.K, cfg.R, sh.kind);
            for (int g = 0; g < kMaxLayouts; ++g) {
                if (g >= L.G) { prog_off[cfgi][s][g] = prog_off[cfgi][s][0]; continue; }
                prog_off[cfgi][s][g] = add(build_layout_prog(sh, I.ei, I.ej, I.J, L.regs[g], cfg.R, L.tbits[g],
                                                             sh.K - cfg.R));
            }
        }
    }
    for (size_t s = 0; s < shapes[0].size(); ++s) {
        const Shape& sh = shapes[0][s];
        const int pc = pair_choice(dtype, 0, sh.kind, sh.c, V_PHASE);
        if (!pc) continue;
        const PairLayout PL = pair_layout(sh.c);
        const PairRunsLayout RL = pair_runs_layout();
        for (int g = 0; g < 2; ++g) {
            int slot[6];
            slot[0] = pc == 1 ? 0 : PL.P;  // slot bit 0: the pack bit; bits 1..5: regs[g]
            for (int b = 0; b < 5; ++b) slot[1 + b] = pc == 1 ? RL.regs[g][b] : PL.regs[g][b];
            const int* tb = pc == 1 ? RL.tbits[g] : PL.tbits[g];
            const std::vector<int32_t> lp = build_layout_prog(sh, I.ei, I.ej, I.J, slot, 6, tb, 7);
            for (int m = 0; m < 64; ++m) pair_q[s].q[g][m] = lp[m];
            prog_pair[s][g] = add(lp);
        }
    }
    for (size_t s = 0; s < shapes[1].size(); ++s) {
        const Shape& sh = shapes[1][s];
        const int pc = pair_choice(dtype, 1, sh.kind, sh.c, 0);
        if (!pc) continue;
        const PairAdjLayout PL = pair_adj_layout(pc);
        for (int g = 0; g < 3; ++g) {
            int slot[5];
            slot[0] = PL.P;  // slot bit 0: the pack bit; bits 1..4: regs[g]
            for (int b = 0; b < 4; ++b) slot[1 + b] = PL.regs[g][b];
            const std::vector<int32_t> lp = build_layout_prog(sh, I.ei, I.ej, I.J, slot, 5, PL.tbits[g], 8);
            for (int m = 0; m < 32; ++m) pair_adj_q[s].q[g][m] = lp[m];
            prog_pair_adj[s][g] = add(lp);
        }
    }
    {
        int regq[6];
        for (int b = 0; b < 6; ++b) regq[b] = b < n ? b : -1;
        enum_off = add(build_cost_prog(n, I.h, I.ei, I.ej, I.J, regq, 6));
    }
    {
        int regq[6] = {-1, -1, -1, -1, -1, -1};
        std::vector<int32_t> pp = build_cost_prog(nphys, h, I.ei, I.ej, I.J, regq, 0);
        plain_nf = pp[1];
        plain_ne = pp[2];
        plain_const0 = pp[3];
        std::vector<int32_t> terms(pp.begin() + 12, pp.begin() + 12 + 2 * (plain_nf + plain_ne));
        plain_off = add(terms.empty() ? std::vector<int32_t>{0, 0} : terms);
    }
    if (int r2 = progs.reserve(blob.size() * sizeof(int32_t))) return r2;
    cudaError_t e = cudaMemcpyAsync(progs.ptr, blob.data(), blob.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "qs_set_ising upload");
    // ground-state search (bit exact) on the device
    if (int r2 = enum_scratch.reserve(8 * 1024 * 4 * sizeof(int64_t) + 4 * sizeof(int64_t))) return r2;
    int64_t* sc = reinterpret_cast<int64_t*>(enum_scratch.ptr);
    e = launch_enumerate(prog(enum_off), n, sc + 4, 8 * 1024 * 4, sc, st);
    if (e != cudaSuccess) return cuda_error(e, "enumerate launch");
    int64_t res[4];
    e = cudaMemcpyAsync(res, sc, sizeof res, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "enumerate");
    cmin = res[0];
    cmax = res[1];
    argmin = res[2];
    count = res[3];
    // the phase table spans [cost_lo, cost_lo + range): the cost range of the
    // padded state equals that of the n-qubit problem
    cost_lo = (int)cmin;
    range = (int)(cmax - cmin + 1);
    if (range < 1) range = 1;
    if (range > (1 << 22)) return set_error(QS_ENOTINT, "qs_set_ising: cost range %d exceeds the phase table limit", range);
    valid = true;
    return QS_OK;
}

}  // namespace qs

using namespace qs;

// ---------------------------------------------------------------------------
// Single-state handle
// ---------------------------------------------------------------------------
struct qs_state {
    int n = 0, nphys = 0, dtype = 0, path = QS_PATH_TILED;
    size_t elem = 8;
    cudaStream_t st = nullptr;
    void* psi = nullptr;
    bool own_psi = false;
    void* lam = nullptr;
    bool own_lam = false;
    Instance inst;
    DevBuf enum_scratch, layers_f, layers_r, tab_f, tab_r, partials, out, frame, err, zpart, zout;
    Uploader up, up_ang, up_su2;
    double theta_pad = 0.0;   // global phase of the idle padding qubits
    bool have_readout = false;
    int grid[2][7] = {};  // [adjoint][kernel kind; 3, 4, 5 = packed-pair kernel, phase / lean / zexp; 6 = runs]
    bool poisoned = false;  // a kernel exited with a tile copy possibly still in flight
    int device = 0;
    ShapeRule rule;                      // tile-shape plan (qs_set_shape_rule / qs_autotune)
    int ctas_per_sm = 0;                 // launch rule: persistent CTAs per SM (0 = as many as fit)
    int pair_cluster = 4;                // launch rule: strided packed-pair sweeps in 4-CTA clusters or not
    int pair_tma = 0;                    // launch rule: strided packed-pair forward tiles by tensor-map copies
    int pair_l2 = 0;                     // launch rule: L2 promotion of the tensor-map tile copies (0 none, 1 128 B, 2 256 B)
    int sms = 0;                         // multiprocessors of the device
    std::vector<double> ising_h, ising_J;  // the last qs_set_ising input, to re-plan
    std::vector<int32_t> ising_e;
};

static int check_handle(qs_handle h) {
    if (!h) return set_error(QS_EINVAL, "NULL handle");
    if (h->poisoned)
        return set_error(QS_ESTATE, "the handle is unusable after a tile copy outlived its kernel; destroy it and "
                                    "create a new one");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    return QS_OK;
}

static int ensure_frame(qs_handle h) {
    if (h->frame.ptr) return QS_OK;
    if (int rc = h->frame.reserve(sizeof(int))) return rc;
    if (int rc = h->err.reserve(sizeof(int))) return rc;
    cudaError_t e = cudaMemsetAsync(h->frame.ptr, 0, sizeof(int), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err.ptr, 0, sizeof(int), h->st);
    return e == cudaSuccess ? QS_OK : cuda_error(e, "frame init");
}

// After a synchronisation: report (and clear) a timed-out device wait.
static int check_device_error(qs_handle h) {
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, h->err.ptr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "error word");
    if (v) {
        cudaMemset(h->err.ptr, 0, sizeof(int));
        h->have_readout = false;
        if (v >= 2) {
            // the exit drain gave up too: a copy may have landed in shared
            // memory after its kernel ended, so nothing on this handle (or
            // computed after that kernel) can be trusted
            h->poisoned = true;
            return set_error(QS_ETIMEOUT, "a sweep kernel gave up waiting for a tile copy and for its drain; the "
                                          "state and later results are invalid and the handle is unusable");
        }
        return set_error(QS_ETIMEOUT, "a sweep kernel gave up waiting for a tile copy; the state is invalid");
    }
    return QS_OK;
}

static int grid_for(qs_handle h, int kind, int adjoint);

extern "C" {

int qs_create(qs_handle* out, int n, int dtype, void* cuda_stream, void* device_buf, size_t buf_bytes) {
    if (!out) return set_error(QS_EINVAL, "qs_create: out is NULL");
    *out = nullptr;
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_create: bad dtype %d", dtype);
    const int nmax = dtype == QS_C64 ? QS_MAX_QUBITS_C64 : QS_MAX_QUBITS_C128;
    if (n < 1 || n > nmax) return set_error(QS_EINVAL, "qs_create: n = %d outside [1, %d]", n, nmax);
    if (device_buf && (reinterpret_cast<uintptr_t>(device_buf) & 255))
        return set_error(QS_EINVAL, "qs_create: device_buf must be 256-byte aligned");
    std::unique_ptr<qs_state> h(new qs_state);
    h->n = n;
    h->nphys = n < kMinPhysQubits ? kMinPhysQubits : n;
    h->dtype = dtype;
    h->elem = dtype == QS_C64 ? 8 : 16;
    h->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    const size_t need = ((size_t)1 << h->nphys) * h->elem;
    if (device_buf) {
        if (buf_bytes < need)
            return set_error(QS_ENOMEM, "qs_create: device_buf holds %zu bytes, %zu needed", buf_bytes, need);
        h->psi = device_buf;
    } else {
        e = cudaMalloc(&h->psi, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(QS_ENOMEM, "qs_create: cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
        }
        h->own_psi = true;
    }
    if (int rc = ensure_frame(h.get())) {
        if (h->own_psi) cudaFree(h->psi);
        return rc;
    }
    *out = h.release();
    return QS_OK;
}

int qs_destroy(qs_handle h) {
    if (!h) return QS_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->st);
    if (h->own_psi && h->psi) cudaFree(h->psi);
    if (h->own_lam && h->lam) cudaFree(h->lam);
    delete h;
    return QS_OK;
}

int qs_set_path(qs_handle h, int path) {
    if (int rc = check_handle(h)) return rc;
    if (path != QS_PATH_TILED && path != QS_PATH_PLAIN) return set_error(QS_EINVAL, "qs_set_path: bad path");
    h->path = path;
    return QS_OK;
}

int qs_set_ising(qs_handle h, const double* hfield, int n_edges, const int32_t* edges, const double* J) {
    if (int rc = check_handle(h)) return rc;
    Instance tmp;
    if (int rc = tmp.set(h->n, h->nphys, h->dtype, hfield, n_edges, edges, J, h->st, h->enum_scratch, h->rule))
        return rc;
    h->inst = std::move(tmp);
    h->have_readout = false;
    h->ising_h.assign(hfield, hfield + h->n);
    h->ising_e.assign(edges, edges + 2 * (size_t)n_edges);
    h->ising_J.assign(J, J + n_edges);
    return QS_OK;
}

static_assert(kPlanRuleInts == QS_PLAN_RULE_INTS, "plan rule length");

// cuTensorMapEncodeTiled from the driver, through the runtime (no link-time
// dependence on libcuda); null when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tile loads of a strided packed-pair forward sweep over psi whose tiles are
// first read into layout g: tensor-map copies (with the rule's L2
// promotion) when the rule asks for them and the shape fits
// (pair_tma_dims), else cp.async.
static PairLoad make_pair_load(qs_handle h, const Shape& s, void* psi, int g) {
    PairLoad L;
    std::memset(&L, 0, sizeof L);
    L.l2 = h->pair_l2;
    PairTmaDims d;
    auto enc = h->pair_tma ? tensor_map_encoder() : nullptr;
    if (!enc || !pair_tma_dims(s, h->nphys, g, d)) return L;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], es[5] = {1, 1, 1, 1, 1};
    for (int i = 0; i < d.rank; ++i) {
        // dimension 0 in floats (two per amplitude), the others in amplitudes
        dims[i] = (cuuint64_t)1 << (d.width[i] + (i == 0 ? 1 : 0));
        box[i] = 1u << (d.box[i] + (i == 0 ? 1 : 0));
        if (i > 0) strides[i - 1] = (cuuint64_t)8 << d.start[i];
        L.lo[i] = d.start[i];
        L.nb[i] = d.width[i];
    }
    const CUtensorMapL2promotion promo = h->pair_l2 == 2   ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                                         : h->pair_l2 == 1 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                           : CU_TENSOR_MAP_L2_PROMOTION_NONE;
    const CUresult r = enc(&L.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)d.rank, psi, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return L;
    L.rank = d.rank;
    L.kbit = d.kbit;
    L.tma = 1;
    return L;
}

// Rebuild the instance's shapes and cost programs under h->rule.
static int replan(qs_handle h) {
    if (!h->inst.valid) return QS_OK;
    Instance tmp;
    const int m = (int)h->ising_J.size();
    if (int rc = tmp.set(h->n, h->nphys, h->dtype, h->ising_h.data(), m, h->ising_e.data(), h->ising_J.data(), h->st,
                         h->enum_scratch, h->rule))
        return rc;
    h->inst = std::move(tmp);
    h->have_readout = false;
    return QS_OK;
}

int qs_set_shape_rule(qs_handle h, int runs_a, int split) {
    if (int rc = check_handle(h)) return rc;
    if (runs_a < -1 || runs_a > 1 || split < -1 || split >= h->nphys + 1)
        return set_error(QS_EINVAL, "qs_set_shape_rule: runs_a in {-1, 0, 1}, split in [-1, n]");
    h->rule = ShapeRule{runs_a, split, h->rule.cmin, h->rule.order};
    return replan(h);
}

int qs_set_plan_rule(qs_handle h, const int* rule) {
    if (int rc = check_handle(h)) return rc;
    if (!rule) return set_error(QS_EINVAL, "qs_set_plan_rule: rule is NULL");
    const int runs_a = rule[0], split = rule[1], cmin = rule[2], cps = rule[3], cl = rule[4], tma = rule[5],
              l2 = rule[6], order = rule[7];
    if (runs_a < -1 || runs_a > 1 || split < -1 || split >= h->nphys + 1 || !(cmin == -1 || cmin == 2 || cmin == 3) ||
        cps < 0 || cps > 32 || !(cl == 1 || cl == 4) || tma < 0 || tma > 1 || l2 < 0 || l2 > 2 || order < 0 ||
        order > 1)
        return set_error(QS_EINVAL, "qs_set_plan_rule: runs_a in {-1, 0, 1}, split in [-1, n], cmin in {-1, 2, 3}, "
                                    "ctas_per_sm in [0, 32], pair_cluster in {1, 4}, pair_tma in {0, 1}, pair_l2 in "
                                    "{0, 1, 2}, order in {0, 1}");
    const ShapeRule nr{runs_a, split, cmin, order};
    const bool reshape = !same_shapes(nr, h->rule);
    h->rule = nr;
    h->ctas_per_sm = cps;
    h->pair_cluster = cl;
    h->pair_tma = tma;
    h->pair_l2 = l2;
    return reshape ? replan(h) : QS_OK;
}

int qs_get_plan_rule(qs_handle h, int* rule) {
    if (int rc = check_handle(h)) return rc;
    if (!rule) return set_error(QS_EINVAL, "qs_get_plan_rule: rule is NULL");
    rule[0] = h->rule.runs_a;
    rule[1] = h->rule.split;
    rule[2] = h->rule.cmin;
    rule[3] = h->ctas_per_sm;
    rule[4] = h->pair_cluster;
    rule[5] = h->pair_tma;
    rule[6] = h->pair_l2;
    rule[7] = h->rule.order;
    return QS_OK;
}

// Device time of an evolve of p_trial layers under the handle's plan: the
// faster of two runs after one warm-up.
static int time_evolve(qs_handle h, int p_trial, const double* g, const double* b, cudaEvent_t e0, cudaEvent_t e1,
                       double* ms_out) {
    double best = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, h->st);
        if (int rc = qs_evolve(h, p_trial, g, b, 1)) return rc;
        cudaEventRecord(e1, h->st);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return cuda_error(ce, "qs_autotune");
        if (int rc = check_device_error(h)) return rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, (double)ms);  // rep 0 is the warm-up
    }
    *ms_out = best;
    return QS_OK;
}

int qs_autotune_ex(qs_handle h, int p_trial, int max_cand, int* ncand, int* cand_rules, double* cand_ms,
                   int* best_rule, double* best_ms) {
    if (int rc = check_handle(h)) return rc;
    if (!h->inst.valid) return set_error(QS_ESTATE, "qs_autotune: call qs_set_ising first");
    if (p_trial < 1 || p_trial > 64) return set_error(QS_EINVAL, "qs_autotune: p_trial outside [1, 64]");
    if (max_cand > 0 && (!cand_rules || !cand_ms)) return set_error(QS_EINVAL, "qs_autotune: NULL candidate arrays");
    struct Cand {
        ShapeRule r;
        int cps, cl, tma, l2;
        double ms;
    };
    std::vector<Cand> done;
    std::vector<double> g(p_trial, 0.3), b(p_trial, 0.7);
    const Cand keep{h->rule, h->ctas_per_sm, h->pair_cluster, h->pair_tma, h->pair_l2, 0.0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) return cuda_error(ce, "qs_autotune: events");
    int rc = QS_OK;
    auto apply = [&](const Cand& c) {
        h->rule = c.r;
        h->ctas_per_sm = c.cps;
        h->pair_cluster = c.cl;
        h->pair_tma = c.tma;
        h->pair_l2 = c.l2;
    };
    double best = 1e300;
    Cand pick{ShapeRule{0, page_bit_for(h->dtype), -1}, 0, 4, 0, 0, 1e300};
    auto measure = [&](Cand c) {
        const bool reshape = !same_shapes(c.r, h->rule);
        apply(c);
        c.ms = 1e300;
        if (reshape && (rc = replan(h))) return;
        if ((rc = time_evolve(h, p_trial, g.data(), b.data(), e0, e1, &c.ms))) return;
        done.push_back(c);
        if (c.ms < best) {
            best = c.ms;
            pick = c;
        }
    };
    // stage 1, tile shapes: contiguous shape A with the page-bit split and,
    // for complex64 states of 24 qubits and more, the run-structured A with
    // three split bits; strided rows of 2^2 or 2^3 amplitudes
    std::vector<ShapeRule> shapes{ShapeRule{0, page_bit_for(h->dtype), -1}};
    if (h->dtype == QS_C64 && h->nphys >= 24)
        for (int sp : {20, 22, 24}) shapes.push_back(ShapeRule{1, sp, -1});
    const size_t ns = shapes.size();
    for (size_t i = 0; i < ns; ++i) shapes.push_back(ShapeRule{shapes[i].runs_a, shapes[i].split, 3});
    for (const ShapeRule& r : shapes) {
        measure(Cand{r, 0, 4, 0, 0, 0.0});
        if (rc) break;
    }
    // the best shapes with the strided shapes in reverse order (another
    // shape's sweeps merged around the phases)
    if (!rc && pick.r.order == 0) {
        ShapeRule r = pick.r;
        r.order = 1;
        measure(Cand{r, 0, 4, 0, 0, 0.0});
    }
    // stage 2, launch: one CTA per SM fewer than fit, and (complex64) the
    // strided packed-pair sweeps without their 4-CTA clusters
    if (!rc) {
        int full = 0;
        for (int k = 0; k < 3; ++k) full = std::max(full, grid_for(h, k, 0));
        if (!h->sms) cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
        const int per_sm = h->sms > 0 ? full / h->sms : 0;
        std::vector<std::pair<int, int>> launch;
        if (per_sm > 1) launch.push_back({per_sm - 1, 4});
        if (h->dtype == QS_C64) launch.push_back({0, 1});
        const Cand base = pick;
        for (auto [cps, cl] : launch) {
            measure(Cand{base.r, cps, cl, 0, 0, 0.0});
            if (rc) break;
        }
    }
    // stage 3 (complex64), the strided packed-pair tile loads: tensor-map
    // copies with the default or 256-byte L2 promotion
    if (!rc && h->dtype == QS_C64) {
        const Cand base = pick;
        const int loads[2][2] = {{1, 0}, {1, 2}};
        for (const auto& ld : loads) {
            measure(Cand{base.r, base.cps, base.cl, ld[0], ld[1], 0.0});
            if (rc) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply(rc ? keep : pick);
    if (int rc2 = replan(h)) return rc ? rc : rc2;
    if (rc) return rc;
    if (ncand) *ncand = (int)done.size();
    for (int i = 0; i < (int)done.size() && i < max_cand; ++i) {
        const Cand& c = done[i];
        const int v[kPlanRuleInts] = {c.r.runs_a, c.r.split, c.r.cmin, c.cps, c.cl, c.tma, c.l2, c.r.order};
        for (int k = 0; k < kPlanRuleInts; ++k) cand_rules[kPlanRuleInts * i + k] = v[k];
        cand_ms[i] = c.ms;
    }
    if (best_rule) {
        const int v[kPlanRuleInts] = {pick.r.runs_a, pick.r.split, pick.r.cmin, pick.cps,
                                      pick.cl,         pick.tma,    pick.l2,     pick.r.order};
        for (int k = 0; k < kPlanRuleInts; ++k) best_rule[k] = v[k];
    }
    if (best_ms) *best_ms = best;
    return QS_OK;
}

int qs_autotune(qs_handle h, int p_trial, int* runs_a, int* split, double* best_ms) {
    int rule[kPlanRuleInts];
    if (int rc = qs_autotune_ex(h, p_trial, 0, nullptr, nullptr, nullptr, rule, best_ms)) return rc;
    if (runs_a) *runs_a = rule[0];
    if (split) *split = rule[1];
    return QS_OK;
}

}  // extern "C"

// Grid size of the persistent sweep kernel for a tile shape.
static int grid_for(qs_handle h, int kind, int adjoint) {
    int& g = h->grid[adjoint][kind];
    if (h->ctas_per_sm > 0) {  // the launch rule caps the persistent grid
        if (!h->sms) cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
        int full = g;
        if (!full) {
            const int keep = h->ctas_per_sm;
            h->ctas_per_sm = 0;
            full = grid_for(h, kind, adjoint);
            h->ctas_per_sm = keep;
        }
        return std::min(full, h->ctas_per_sm * h->sms);
    }
    if (!g)
        g = kind < 3    ? sweep_grid(h->dtype, adjoint, kind)
            : adjoint   ? sweep_pair_adj_grid()
            : kind == 6 ? sweep_runs_grid(V_PHASE)
                        : sweep_pair_grid(kind == 4 ? V_LEAN : kind == 5 ? V_ZPHASE : V_PHASE);
    return g;
}

// Grid of a forward sweep launch (the persistent grid, clamped as in
// launch_sweep to the number of tiles).
static int forward_grid(qs_handle h, const SweepLaunch& L) {
    int g = L.pairc == 1 ? grid_for(h, 6, 0)
            : L.pairc    ? grid_for(h, L.variant == V_LEAN ? 4 : L.variant == V_ZPHASE ? 5 : 3, 0)
                         : grid_for(h, L.kind, 0);
    if (g > L.total_tiles) g = (int)L.total_tiles;
    return g < 1 ? 1 : g;
}

// Upload the angles and prepare forward (and optionally reverse) layers.
static int prepare_layers(qs_handle h, int p, const double* gamma, const double* beta, bool from_plus, bool reverse,
                          bool plain) {
    Instance& I = h->inst;
    std::vector<double> ang(2 * (size_t)(p > 0 ? p : 1), 0.0);
    for (int k = 0; k < p; ++k) { ang[k] = gamma[k]; ang[p + k] = beta[k]; }
    if (int rc = h->up_ang.upload(ang.data(), ang.size() * sizeof(double), h->st)) return rc;
    cudaError_t e;
    const double* dg = reinterpret_cast<const double*>(h->up_ang.dev.ptr);
    const double* db = dg + p;
    const size_t tsz = (size_t)(p > 0 ? p : 1) * I.range * h->elem * 2;
    if (int rc = h->layers_f.reserve((size_t)(p + 1) * sizeof(LayerDev))) return rc;
    if (int rc = h->tab_f.reserve(tsz)) return rc;
    const int* f0 = from_plus ? nullptr : reinterpret_cast<const int*>(h->frame.ptr);
    e = launch_prep(h->dtype, p, dg, db, h->nphys, I.cost_lo, I.range, I.shift, f0, plain ? 2 : 0,
                    reinterpret_cast<LayerDev*>(h->layers_f.ptr), h->tab_f.ptr, I.range, h->st);
    if (e != cudaSuccess) return cuda_error(e, "prep");
    if (reverse) {
        if (int rc = h->layers_r.reserve((size_t)(p + 1) * sizeof(LayerDev))) return rc;
        if (int rc = h->tab_r.reserve(tsz)) return rc;
        e = launch_prep(h->dtype, p, dg, db, h->nphys, I.cost_lo, I.range, I.shift, f0, 1,
                        reinterpret_cast<LayerDev*>(h->layers_r.ptr), h->tab_r.ptr, I.range, h->st);
        if (e != cudaSuccess) return cuda_error(e, "prep reverse");
    }
    return QS_OK;
}

static SweepTask make_task(qs_handle h, const Shape& sh, const PlanSweep& ps, int cfgi, int shape_idx, void* lam,
                           const LayerDev* layers, const void* tab, int p, double* partials, int objective) {
    Instance& I = h->inst;
    SweepTask t;
    std::memset(&t, 0, sizeof t);
    t.psi = h->psi;
    t.lam = lam;
    t.layers = layers;
    t.tab = tab;
    for (int g = 0; g < kMaxLayouts; ++g) t.cprog[g] = I.prog(I.prog_off[cfgi][shape_idx][g]);
    t.tprog = I.prog(I.tprog_off[cfgi][shape_idx]);
    t.partials = partials;
    t.ntiles = sh.ntiles;
    t.part_base = 0;
    t.n = h->nphys;
    t.c = sh.c;
    t.g0 = sh.g0;
    t.flags = ps.flags;
    t.nrounds = ps.nr;
    t.objective = objective;
    t.tab_stride = I.range;
    t.cost_lo = I.cost_lo;
    t.gidx = (int)(I.cmin - I.cost_lo);
    t.end_layer = p;
    t.amp0 = std::pow(2.0, -0.5 * h->nphys);
    t.np = (ps.flags & T_ADJOINT) ? 2 * ps.nr : ((ps.flags & T_READOUT) ? 3 : 0);
    for (int r = 0; r < ps.nr; ++r) t.rounds[r] = ps.r[r];
    t.kind = sh.kind;
    t.n1 = sh.n1;
    t.g1 = sh.g1;
    return t;
}

// Blob uploaded once per call: tasks, per-launch tile prefixes, reduce tasks,
// each record 64-byte aligned.
struct CallBlob {
    std::vector<unsigned char> bytes;
    size_t add(const void* p, size_t n) {
        size_t off = (bytes.size() + 63) & ~size_t(63);
        bytes.resize(off + n);
        std::memcpy(bytes.data() + off, p, n);
        return off;
    }
};

// Run the tiled schedule: forward sweeps (+ readout), and for a gradient the
// reverse sweeps with their per-layer reductions.
//
// zexp: every sweep holding a layer boundary (a phase of layer k >= 1) or the
// readout also records <Z_q> of the state after layer k - 1 (resp. p - 1)
// into per-CTA records, reduced after the sweep into h->zout[layer][n].
// Kernel of a forward sweep: the variant (sweep_variant) and the packed-pair
// kernel (pair_choice; 0 = the generic sweep kernel).  The first and the
// readout sweep of the run-structured shape A run on its packed-pair kernel
// (V_RUNS_GEN, V_RUNS_READ) when they do nothing else.
static void forward_kernel(qs_handle h, const Shape& sh, const PlanSweep& s, int& variant, int& pairc) {
    variant = sweep_variant(s.flags, s.nr, s.r);
    pairc = pair_choice(h->dtype, 0, sh.kind, sh.c, variant);
    const int fl = s.flags & (T_GEN | T_READOUT | T_WRITE_LAM | T_ADJOINT | T_ZEXP | T_SU2);
    if (variant == V_FULL && (fl == T_GEN || fl == T_READOUT) &&
        pair_choice(h->dtype, 0, sh.kind, sh.c, V_PHASE) == 1) {
        variant = fl == T_GEN ? V_RUNS_GEN : V_RUNS_READ;
        pairc = 1;
    }
}

static int run_tiled(qs_handle h, int p, bool from_plus, int mode_grad, int objective, bool zexp = false,
                     const double* su2 = nullptr) {
    Instance& I = h->inst;
    const std::vector<Shape>& shf = I.shapes[0];
    const std::vector<Shape>& sha = I.shapes[1];
    std::vector<PlanSweep> fwd = plan_forward((int)shf.size(), p, from_plus);
    std::vector<PlanSweep> rev;
    if (mode_grad) {
        fwd.back().flags |= T_WRITE_LAM;
        rev = plan_reverse(fwd, sha, p);
    }
    if (su2)
        for (auto& s : fwd) s.flags |= T_SU2;
    if (zexp) {
        for (auto& s : fwd) {
            bool rec = (s.flags & T_READOUT) != 0;
            for (int r = 0; r < s.nr; ++r) rec = rec || (s.r[r].phase_pre && s.r[r].layer > 0);
            if (rec) s.flags |= T_ZEXP;
        }
        int gmax = 1;
        for (int k = 0; k < 7; ++k) gmax = std::max(gmax, k < 3 ? grid_for(h, k, 0) : (h->dtype == 0 ? grid_for(h, k, 0) : 1));
        if (int rc = h->zpart.reserve((size_t)gmax * kZSlots * kZQ * sizeof(double))) return rc;
        if (int rc = h->zout.reserve((size_t)std::max(p, 1) * h->n * sizeof(double))) return rc;
    }
    size_t part_need = 0;
    for (auto& s : fwd) part_need = std::max(part_need, (size_t)shf[s.shape].ntiles * ((s.flags & T_READOUT) ? 3 : 0));
    for (auto& s : rev) part_need = std::max(part_need, (size_t)sha[s.shape].ntiles * 2 * s.nr);
    if (int rc = h->partials.reserve((part_need + 4) * sizeof(double))) return rc;
    if (int rc = h->out.reserve((3 + 2 * (size_t)(p + 1)) * sizeof(double))) return rc;
    double* dpart = reinterpret_cast<double*>(h->partials.ptr);
    double* dout = reinterpret_cast<double*>(h->out.ptr);
    CallBlob blob;
    std::vector<size_t> fwd_off, rev_off, fwd_pre, rev_pre, red_off;
    std::vector<int> red_cnt;
    const LayerDev* lf = reinterpret_cast<const LayerDev*>(h->layers_f.ptr);
    const LayerDev* lr = reinterpret_cast<const LayerDev*>(h->layers_r.ptr);
    std::vector<size_t> zred_off;
    std::vector<int> zred_cnt;
    double* dzp = reinterpret_cast<double*>(h->zpart.ptr);
    double* dzo = reinterpret_cast<double*>(h->zout.ptr);
    for (auto& s : fwd) {
        SweepTask t = make_task(h, shf[s.shape], s, 0, s.shape, h->lam, lf, h->tab_f.ptr, p, dpart, objective);
        const Shape& sh = shf[s.shape];
        int variant = 0, pc = 0;
        forward_kernel(h, sh, s, variant, pc);
        if (pc)
            for (int g = 0; g < kMaxLayouts; ++g) t.cprog[g] = I.prog(I.prog_pair[s.shape][g < 2 ? g : 0]);
        t.zpart = dzp;
        t.su2 = su2;
        fwd_off.push_back(blob.add(&t, sizeof t));
        const int64_t pre[2] = {0, shf[s.shape].ntiles};
        fwd_pre.push_back(blob.add(pre, sizeof pre));
        std::vector<ReduceTask> zts;
        if (s.flags & T_ZEXP) {
            SweepLaunch L{kernel_kind(sh), variant, 0, h->dtype, 1, sh.ntiles, nullptr, nullptr, nullptr};
            L.pairc = pc;
            const int64_t g = forward_grid(h, L);
            for (int r = 0; r < s.nr; ++r)
                if (s.r[r].phase_pre && s.r[r].layer > 0)
                    zts.push_back(ReduceTask{dzp, g, kZSlots * kZQ, r * kZQ, h->n,
                                             dzo + (size_t)(s.r[r].layer - 1) * h->n, 0, 1.0});
            if ((s.flags & T_READOUT) && p > 0)
                zts.push_back(ReduceTask{dzp, g, kZSlots * kZQ, kMaxRounds * kZQ, h->n, dzo + (size_t)(p - 1) * h->n, 0, 1.0});
        }
        zred_off.push_back(zts.empty() ? 0 : blob.add(zts.data(), zts.size() * sizeof(ReduceTask)));
        zred_cnt.push_back((int)zts.size());
    }
    for (auto& s : rev) {
        SweepTask t = make_task(h, sha[s.shape], s, 1, s.shape, h->lam, lr, h->tab_r.ptr, p, dpart, objective);
        if (pair_choice(h->dtype, 1, sha[s.shape].kind, sha[s.shape].c, 0))
            for (int g = 0; g < kMaxLayouts; ++g) t.cprog[g] = I.prog(I.prog_pair_adj[s.shape][g]);
        rev_off.push_back(blob.add(&t, sizeof t));
        const int64_t pre[2] = {0, sha[s.shape].ntiles};
        rev_pre.push_back(blob.add(pre, sizeof pre));
        // per round: beta partial -> out[3 + 2 layer], gamma partial -> out[3 + 2 layer + 1]
        std::vector<ReduceTask> rts;
        for (int r = 0; r < s.nr; ++r) {
            const int L = s.r[r].layer;
            rts.push_back(ReduceTask{dpart, sha[s.shape].ntiles, 2 * s.nr, 2 * r, 1, dout + 3 + 2 * L, 1, 1.0});
            if (s.r[r].phase_post)
                rts.push_back(ReduceTask{dpart, sha[s.shape].ntiles, 2 * s.nr, 2 * r + 1, 1, dout + 3 + 2 * L + 1, 1, 1.0});
        }
        red_off.push_back(rts.empty() ? 0 : blob.add(rts.data(), rts.size() * sizeof(ReduceTask)));
        red_cnt.push_back((int)rts.size());
    }
    const ReduceTask rt{dpart, shf[fwd.back().shape].ntiles, 3, 0, 3, dout, 0, 1.0};
    const size_t rd_off = blob.add(&rt, sizeof rt);
    if (int rc = h->up.upload(blob.bytes.data(), blob.bytes.size(), h->st)) return rc;
    const unsigned char* dblob = reinterpret_cast<const unsigned char*>(h->up.dev.ptr);
    int* derr = reinterpret_cast<int*>(h->err.ptr);
    cudaError_t e;
    if (mode_grad) {
        e = cudaMemsetAsync(dout + 3, 0, 2 * (size_t)p * sizeof(double), h->st);
        if (e != cudaSuccess) return cuda_error(e, "zero grads");
    }
    for (size_t i = 0; i < fwd.size(); ++i) {
        const Shape& sh = shf[fwd[i].shape];
        SweepLaunch L{kernel_kind(sh), 0, 0, h->dtype, 1, sh.ntiles,
                      reinterpret_cast<const SweepTask*>(dblob + fwd_off[i]),
                      reinterpret_cast<const int64_t*>(dblob + fwd_pre[i]), derr};
        forward_kernel(h, sh, fwd[i], L.variant, L.pairc);
        L.pq = &I.pair_q[fwd[i].shape];
        L.cluster = h->pair_cluster;
        PairLoad pl;
        if (L.pairc >= 2) {
            pl = make_pair_load(h, sh, h->psi, fwd[i].nr & 1);
            L.load = &pl;
        }
        e = launch_sweep(L, forward_grid(h, L), h->st);
        if (e != cudaSuccess) return cuda_error(e, "sweep launch");
        if (zred_cnt[i]) {
            e = launch_reduce(reinterpret_cast<const ReduceTask*>(dblob + zred_off[i]), zred_cnt[i], h->st);
            if (e != cudaSuccess) return cuda_error(e, "spin expectation reduce");
        }
    }
    e = launch_reduce(reinterpret_cast<const ReduceTask*>(dblob + rd_off), 1, h->st);
    if (e != cudaSuccess) return cuda_error(e, "readout reduce");
    for (size_t i = 0; i < rev.size(); ++i) {
        const Shape& sh = sha[rev[i].shape];
        SweepLaunch L{kernel_kind(sh), 0, 1, h->dtype, 1, sh.ntiles, reinterpret_cast<const SweepTask*>(dblob + rev_off[i]),
                      reinterpret_cast<const int64_t*>(dblob + rev_pre[i]), derr};
        L.pairc = pair_choice(h->dtype, 1, sh.kind, sh.c, 0);
        L.paq = &I.pair_adj_q[rev[i].shape];
        e = launch_sweep(L, grid_for(h, L.pairc ? 3 : L.kind, 1), h->st);
        if (e != cudaSuccess) return cuda_error(e, "adjoint sweep launch");
        if (red_cnt[i]) {
            e = launch_reduce(reinterpret_cast<const ReduceTask*>(dblob + red_off[i]), red_cnt[i], h->st);
            if (e != cudaSuccess) return cuda_error(e, "adjoint reduce");
        }
    }
    return QS_OK;
}

static int run_plain(qs_handle h, int p, bool from_plus) {
    Instance& I = h->inst;
    cudaError_t e;
    if (from_plus) {
        e = launch_plain_init(h->dtype, h->psi, h->nphys, h->st);
        if (e != cudaSuccess) return cuda_error(e, "plain init");
    }
    const LayerDev* lf = reinterpret_cast<const LayerDev*>(h->layers_f.ptr);
    for (int k = 0; k < p; ++k) {
        e = launch_plain_phase(h->dtype, h->psi, h->nphys, I.prog(I.plain_off), I.plain_nf, I.plain_ne,
                               I.plain_const0, lf + k,
                               reinterpret_cast<const unsigned char*>(h->tab_f.ptr) + (size_t)k * I.range * h->elem,
                               I.cost_lo, I.range, h->st);
        if (e != cudaSuccess) return cuda_error(e, "plain phase");
        for (int q = 0; q < h->nphys; ++q) {
            e = launch_plain_rx(h->dtype, h->psi, h->nphys, q, lf + k, h->st);
            if (e != cudaSuccess) return cuda_error(e, "plain rx");
        }
    }
    // readout
    const int64_t nb = plain_readout_blocks(h->nphys);
    if (int rc = h->partials.reserve((size_t)nb * 3 * sizeof(double) + 32)) return rc;
    if (int rc = h->out.reserve(8 * sizeof(double))) return rc;
    double* dpart = reinterpret_cast<double*>(h->partials.ptr);
    e = launch_plain_readout(h->dtype, h->psi, h->nphys, I.prog(I.plain_off), I.plain_nf, I.plain_ne,
                             I.plain_const0, (int)I.cmin, reinterpret_cast<const int*>(h->frame.ptr), dpart, nb,
                             h->st);
    if (e != cudaSuccess) return cuda_error(e, "plain readout");
    ReduceTask rt{dpart, nb, 3, 0, 3, reinterpret_cast<double*>(h->out.ptr), 0, 1.0};
    if (int rc = h->up.upload(&rt, sizeof rt, h->st)) return rc;
    e = launch_reduce(reinterpret_cast<const ReduceTask*>(h->up.dev.ptr), 1, h->st);
    if (e != cudaSuccess) return cuda_error(e, "plain reduce");
    return QS_OK;
}

static int check_angles(int p, const double* gamma, const double* beta) {
    if (p < 0 || p > QS_MAX_LAYERS_PREP) return set_error(QS_EINVAL, "p = %d outside [0, %d]", p, QS_MAX_LAYERS_PREP);
    if (p > 0 && (!gamma || !beta)) return set_error(QS_EINVAL, "gamma or beta is NULL");
    for (int k = 0; k < p; ++k)
        if (!std::isfinite(gamma[k]) || !std::isfinite(beta[k])) return set_error(QS_EINVAL, "non-finite angle at layer %d", k);
    return QS_OK;
}

extern "C" {

int qs_evolve(qs_handle h, int p, const double* gamma, const double* beta, int from_plus) {
    if (int rc = check_handle(h)) return rc;
    if (!h->inst.valid) return set_error(QS_ESTATE, "qs_evolve: call qs_set_ising first");
    if (int rc = check_angles(p, gamma, beta)) return rc;
    const bool plain = h->path == QS_PATH_PLAIN;
    if (int rc = prepare_layers(h, p, gamma, beta, from_plus != 0, false, plain)) return rc;
    int rc = plain ? run_plain(h, p, from_plus != 0) : run_tiled(h, p, from_plus != 0, 0, 0);
    if (rc) return rc;
    if (!plain) {
        cudaError_t e = launch_set_frame(reinterpret_cast<int*>(h->frame.ptr),
                                         reinterpret_cast<const LayerDev*>(h->layers_f.ptr), p, h->st);
        if (e != cudaSuccess) return cuda_error(e, "set frame");
    } else if (from_plus) {
        cudaMemsetAsync(h->frame.ptr, 0, sizeof(int), h->st);
    }
    double bsum = 0;
    for (int k = 0; k < p; ++k) bsum += beta[k];
    h->theta_pad = (from_plus ? 0.0 : h->theta_pad) + (h->nphys - h->n) * bsum;
    h->have_readout = true;
    return QS_OK;
}

int qs_evolve_zexp(qs_handle h, int p, const double* gamma, const double* beta, double* zexp) {
    if (int rc = check_handle(h)) return rc;
    if (!h->inst.valid) return set_error(QS_ESTATE, "qs_evolve_zexp: call qs_set_ising first");
    if (h->path != QS_PATH_TILED) return set_error(QS_EINVAL, "qs_evolve_zexp: needs the tiled path");
    if (int rc = check_angles(p, gamma, beta)) return rc;
    if (p > 0 && !zexp) return set_error(QS_EINVAL, "qs_evolve_zexp: zexp is NULL");
    if (int rc = prepare_layers(h, p, gamma, beta, true, false, false)) return rc;
    if (int rc = run_tiled(h, p, true, 0, 0, true)) return rc;
    cudaError_t e = launch_set_frame(reinterpret_cast<int*>(h->frame.ptr),
                                     reinterpret_cast<const LayerDev*>(h->layers_f.ptr), p, h->st);
    if (e != cudaSuccess) return cuda_error(e, "set frame");
    double bsum = 0;
    for (int k = 0; k < p; ++k) bsum += beta[k];
    h->theta_pad = (h->nphys - h->n) * bsum;
    h->have_readout = true;
    if (p > 0) {
        e = cudaMemcpyAsync(zexp, h->zout.ptr, (size_t)p * h->n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cuda_error(e, "qs_evolve_zexp");
    }
    return check_device_error(h);
}

int qs_evolve_su2(qs_handle h, int p, const double* gamma, const double* u) {
    if (int rc = check_handle(h)) return rc;
    if (!h->inst.valid) return set_error(QS_ESTATE, "qs_evolve_su2: call qs_set_ising first");
    if (h->path != QS_PATH_TILED) return set_error(QS_EINVAL, "qs_evolve_su2: needs the tiled path");
    if (p < 0 || p > QS_MAX_LAYERS_PREP) return set_error(QS_EINVAL, "qs_evolve_su2: p = %d outside [0, %d]", p, QS_MAX_LAYERS_PREP);
    if (p > 0 && (!gamma || !u)) return set_error(QS_EINVAL, "qs_evolve_su2: gamma or u is NULL");
    for (int k = 0; k < p; ++k)
        if (!std::isfinite(gamma[k])) return set_error(QS_EINVAL, "qs_evolve_su2: non-finite gamma at layer %d", k);
    for (size_t i = 0; i < (size_t)p * h->n * 8; ++i)
        if (!std::isfinite(u[i])) return set_error(QS_EINVAL, "qs_evolve_su2: non-finite matrix entry %zu", i);
    // per layer, the n given matrices and the identity on padded idle qubits
    std::vector<double> U((size_t)std::max(p, 1) * h->nphys * 8, 0.0);
    for (int k = 0; k < p; ++k)
        for (int q = 0; q < h->nphys; ++q) {
            double* d = U.data() + ((size_t)k * h->nphys + q) * 8;
            if (q < h->n) std::memcpy(d, u + ((size_t)k * h->n + q) * 8, 8 * sizeof(double));
            else { d[0] = 1.0; d[6] = 1.0; }
        }
    if (int rc = h->up_su2.upload(U.data(), U.size() * sizeof(double), h->st)) return rc;
    std::vector<double> zero((size_t)std::max(p, 1), 0.0);
    if (int rc = prepare_layers(h, p, gamma, zero.data(), true, false, true)) return rc;  // pure phase tables
    if (int rc = run_tiled(h, p, true, 0, 0, false, reinterpret_cast<const double*>(h->up_su2.dev.ptr))) return rc;
    cudaError_t e = cudaMemsetAsync(h->frame.ptr, 0, sizeof(int), h->st);
    if (e != cudaSuccess) return cuda_error(e, "qs_evolve_su2 frame");
    h->theta_pad = 0.0;
    h->have_readout = true;
    return QS_OK;
}

int qs_readout(qs_handle h, double* E, double* P, double* norm) {
    if (int rc = check_handle(h)) return rc;
    if (!h->have_readout) return set_error(QS_ESTATE, "no state evolved yet");
    double r[3];
    cudaError_t e = cudaMemcpyAsync(r, h->out.ptr, sizeof r, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_error(e, "readout");
    if (int rc = check_device_error(h)) return rc;
    const double sc = std::ldexp(1.0, -h->inst.shift);
    if (E) *E = r[0] * sc;
    if (P) *P = r[1];
    if (norm) *norm = r[2];
    return QS_OK;
}

int qs_expect(qs_handle h, double* E) { return qs_readout(h, E, nullptr, nullptr); }

int qs_ground_prob(qs_handle h, double* P, int64_t* argmin, int64_t* cmin, int64_t* ground_count) {
    if (int rc = qs_readout(h, nullptr, P, nullptr)) return rc;
    if (argmin) *argmin = h->inst.argmin;
    if (cmin) *cmin = h->inst.cmin;
    if (ground_count) *ground_count = h->inst.count;
    return QS_OK;
}

int qs_cost_info(qs_handle h, int64_t* cmin, int64_t* cmax, int64_t* argmin, int64_t* ground_count, int* scale_shift) {
    if (int rc = check_handle(h)) return rc;
    if (!h->inst.valid) return set_error(QS_ESTATE, "qs_cost_info: call qs_set_ising first");
    if (cmin) *cmin = h->inst.cmin;
    if (cmax) *cmax = h->inst.cmax;
    if (argmin) *argmin = h->inst.argmin;
    if (ground_count) *ground_count = h->inst.count;
    if (scale_shift) *scale_shift = h->inst.shift;
    return QS_OK;
}

int qs_set_adjoint_buffer(qs_handle h, void* device_buf, size_t buf_bytes) {
    if (int rc = check_handle(h)) return rc;
    const size_t need = ((size_t)1 << h->nphys) * h->elem;
    if (device_buf && (reinterpret_cast<uintptr_t>(device_buf) & 255))
        return set_error(QS_EINVAL, "adjoint buffer must be 256-byte aligned");
    if (device_buf && buf_bytes < need)
        return set_error(QS_ENOMEM, "adjoint buffer holds %zu bytes, %zu needed", buf_bytes, need);
    cudaStreamSynchronize(h->st);
    if (h->own_lam && h->lam) cudaFree(h->lam);
    h->lam = device_buf;
    h->own_lam = false;
    return QS_OK;
}

int qs_grad(qs_handle h, int p, const double* gamma, const double* beta, int objective, double* value,
            double* dgamma, double* dbeta) {
    if (int rc = check_handle(h)) return rc;
    if (!h->inst.valid) return set_error(QS_ESTATE, "qs_grad: call qs_set_ising first");
    if (objective != QS_OBJ_ENERGY && objective != QS_OBJ_GROUND) return set_error(QS_EINVAL, "bad objective");
    if (int rc = check_angles(p, gamma, beta)) return rc;
    if (p > 0 && (!dgamma || !dbeta)) return set_error(QS_EINVAL, "dgamma or dbeta is NULL");
    if (!h->lam) {
        const size_t need = ((size_t)1 << h->nphys) * h->elem;
        cudaError_t e = cudaMalloc(&h->lam, need);
        if (e != cudaSuccess) {
            h->lam = nullptr;
            cudaGetLastError();
            return set_error(QS_ENOMEM, "qs_grad: adjoint buffer cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
        }
        h->own_lam = true;
    }
    if (int rc = prepare_layers(h, p, gamma, beta, true, true, false)) return rc;
    if (int rc = run_tiled(h, p, true, 1, objective)) return rc;
    std::vector<double> r(3 + 2 * (size_t)p);
    cudaError_t e = cudaMemcpyAsync(r.data(), h->out.ptr, r.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_error(e, "qs_grad");
    if (int rc = check_device_error(h)) return rc;
    const double sc = std::ldexp(1.0, -h->inst.shift);
    const double lam_sc = objective == QS_OBJ_ENERGY ? sc : 1.0;
    if (value) *value = objective == QS_OBJ_ENERGY ? r[0] * sc : r[1];
    for (int k = 0; k < p; ++k) {
        dbeta[k] = 2.0 * r[3 + 2 * k] * lam_sc;
        dgamma[k] = 2.0 * r[3 + 2 * k + 1] * sc * lam_sc;
    }
    // the reverse pass un-computed the state: it no longer holds psi_p
    h->have_readout = false;
    cudaMemsetAsync(h->frame.ptr, 0, sizeof(int), h->st);
    return QS_OK;
}

int qs_copy_state(qs_handle h, void* dst_host, size_t bytes) {
    if (int rc = check_handle(h)) return rc;
    const size_t need = ((size_t)1 << h->n) * h->elem;
    if (!dst_host) return set_error(QS_EINVAL, "qs_copy_state: dst is NULL");
    if (bytes != need) return set_error(QS_EINVAL, "qs_copy_state: %zu bytes given, %zu needed", bytes, need);
    const size_t N = (size_t)1 << h->nphys;
    std::vector<unsigned char> full(N * h->elem);
    int frame = 0;
    cudaError_t e = cudaMemcpyAsync(full.data(), h->psi, full.size(), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&frame, h->frame.ptr, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_error(e, "qs_copy_state");
    const size_t fm = frame ? N - 1 : 0;
    // n < nphys: the idle qubits are in |+> times the global phase e^{-i theta}
    const double padscale = std::pow(2.0, 0.5 * (h->nphys - h->n));
    const double cr = std::cos(h->theta_pad) * padscale, ci = std::sin(h->theta_pad) * padscale;
    const size_t Nn = (size_t)1 << h->n;
    for (size_t z = 0; z < Nn; ++z) {
        const size_t src = z ^ fm;
        if (h->dtype == QS_C64) {
            const float* s = reinterpret_cast<const float*>(full.data()) + 2 * src;
            float* d = reinterpret_cast<float*>(dst_host) + 2 * z;
            const double re = s[0], im = s[1];
            d[0] = (float)(re * cr - im * ci);
            d[1] = (float)(re * ci + im * cr);
        } else {
            const double* s = reinterpret_cast<const double*>(full.data()) + 2 * src;
            double* d = reinterpret_cast<double*>(dst_host) + 2 * z;
            d[0] = s[0] * cr - s[1] * ci;
            d[1] = s[0] * ci + s[1] * cr;
        }
    }
    return QS_OK;
}

int qs_state_ptr(qs_handle h, void** device_ptr, int* flip_all) {
    if (int rc = check_handle(h)) return rc;
    if (device_ptr) *device_ptr = h->psi;
    if (flip_all) {
        int f = 0;
        cudaError_t e = cudaMemcpyAsync(&f, h->frame.ptr, sizeof(int), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cuda_error(e, "qs_state_ptr");
        *flip_all = f;
    }
    return QS_OK;
}

int qs_canonicalize(qs_handle h) {
    int f = 0;
    if (int rc = qs_state_ptr(h, nullptr, &f)) return rc;
    if (!f) return QS_OK;
    cudaError_t e = launch_flip_all(h->dtype, h->psi, h->nphys, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->frame.ptr, 0, sizeof(int), h->st);
    return e == cudaSuccess ? QS_OK : cuda_error(e, "qs_canonicalize");
}

int qs_plan_info(qs_handle h, int p, int* tile_shapes, int* sweeps) {
    if (!h) return set_error(QS_EINVAL, "NULL handle");
    if (p < 0) return set_error(QS_EINVAL, "p < 0");
    const auto sh = make_shapes(h->nphys, kernel_cfg(h->dtype, false), page_bit_for(h->dtype), h->rule);
    if (tile_shapes) *tile_shapes = (int)sh.size();
    if (sweeps) *sweeps = (int)plan_forward((int)sh.size(), p, true).size();
    return QS_OK;
}

int qs_plan_sweeps(int n, int dtype, int p, int* tile_shapes, int* sweeps) {
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_plan_sweeps: bad dtype");
    const int nmax = dtype == QS_C64 ? QS_MAX_QUBITS_C64 : QS_MAX_QUBITS_C128;
    if (n < 1 || n > nmax || p < 0) return set_error(QS_EINVAL, "qs_plan_sweeps: bad n or p");
    const int nphys = n < kMinPhysQubits ? kMinPhysQubits : n;
    const auto sh = make_shapes(nphys, kernel_cfg(dtype, false), page_bit_for(dtype));
    if (tile_shapes) *tile_shapes = (int)sh.size();
    if (sweeps) *sweeps = (int)plan_forward((int)sh.size(), p, true).size();
    return QS_OK;
}

int qs_plan_shape(int n, int dtype, int k, int* kind, int* K, int* c, int* g0, int* n1, int* g1) {
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_plan_shape: bad dtype");
    const int nmax = dtype == QS_C64 ? QS_MAX_QUBITS_C64 : QS_MAX_QUBITS_C128;
    if (n < 1 || n > nmax) return set_error(QS_EINVAL, "qs_plan_shape: bad n");
    const int nphys = n < kMinPhysQubits ? kMinPhysQubits : n;
    const auto sh = make_shapes(nphys, kernel_cfg(dtype, false), page_bit_for(dtype));
    if (k < 0 || k >= (int)sh.size()) return set_error(QS_EINVAL, "qs_plan_shape: no shape %d", k);
    const Shape& s = sh[k];
    if (kind) *kind = s.kind;
    if (K) *K = s.K;
    if (c) *c = s.c;
    if (g0) *g0 = s.g0;
    if (n1) *n1 = s.n1;
    if (g1) *g1 = s.g1;
    return QS_OK;
}

int qs_pair_tile_map(int n, int c, int g0, int n1, int g1, int g, int* rank, int* kbit, int* start, int* width,
                     int* box, int* landing) {
    if (!rank || !kbit || !start || !width || !box || !landing)
        return set_error(QS_EINVAL, "qs_pair_tile_map: NULL output");
    const int nt = kPairK - c;
    const bool runs_ok = c >= 0 && n1 >= 0 && n1 <= nt && g0 >= c && g1 >= c && n <= QS_MAX_QUBITS_C64 &&
                         g0 + n1 <= n && g1 + (nt - n1) <= n && (n1 == 0 || g1 >= g0 + n1 || g1 + nt - n1 <= g0);
    if (!runs_ok) return set_error(QS_EINVAL, "qs_pair_tile_map: not a strided shape of %d qubits", n);
    Shape s;
    s.K = kPairK;
    s.c = c;
    s.g0 = g0;
    s.nt = nt;
    s.kind = 1;
    s.n1 = n1;
    s.g1 = g1;
    s.ntiles = (int64_t)1 << (n - kPairK);
    PairTmaDims d;
    if (!pair_tma_dims(s, n, g, d)) return set_error(QS_EINVAL, "qs_pair_tile_map: the shape does not fit a box");
    *rank = d.rank;
    *kbit = d.kbit;
    for (int i = 0; i < 5; ++i) {
        start[i] = i < d.rank ? d.start[i] : 0;
        width[i] = i < d.rank ? d.width[i] : 0;
        box[i] = i < d.rank ? d.box[i] : 0;
    }
    const PairTmaPos tp = pair_tma_pos(c, g);
    for (int tb = 0; tb < kPairK; ++tb) landing[tb] = tp.pos[tb];
    return QS_OK;
}

int qs_aqa_angles(int p, double tau, const double* s, double* gamma, double* beta) {
    if (p < 0 || (p > 0 && (!s || !gamma || !beta)) || !std::isfinite(tau))
        return set_error(QS_EINVAL, "qs_aqa_angles: bad arguments");
    for (int k = 0; k < p; ++k) {
        gamma[k] = tau * s[k];
        beta[k] = -tau * (1.0 - s[k]);
    }
    return QS_OK;
}

int qs_aqa_angles_2nd(int p, double tau, const double* s, double* gamma, double* beta) {
    if (p < 1 || !s || !gamma || !beta || !std::isfinite(tau))
        return set_error(QS_EINVAL, "qs_aqa_angles_2nd: bad arguments");
    for (int k = 0; k < p; ++k) {
        const double A = 1.0 - s[k];
        gamma[k] = tau * s[k];
        beta[k] = (k + 1 < p) ? -tau * ((1.0 - s[k + 1]) + A) / 2.0 : -tau * A / 2.0;
    }
    return QS_OK;
}

int qs_aqa_chain(int p, double tau, const double* s, const double* dgamma, const double* dbeta, double* dtau,
                 double* ds) {
    if (p < 0 || (p > 0 && (!s || !dgamma || !dbeta || !ds)) || !dtau)
        return set_error(QS_EINVAL, "qs_aqa_chain: bad arguments");
    double t = 0;
    for (int k = 0; k < p; ++k) {
        t += s[k] * dgamma[k] - (1.0 - s[k]) * dbeta[k];
        ds[k] = tau * (dgamma[k] + dbeta[k]);
    }
    *dtau = t;
    return QS_OK;
}

int qs_aqa_chain_2nd(int p, double tau, const double* s, const double* dgamma, const double* dbeta, double* dtau,
                     double* ds) {
    if (p < 1 || !s || !dgamma || !dbeta || !ds || !dtau || !std::isfinite(tau))
        return set_error(QS_EINVAL, "qs_aqa_chain_2nd: bad arguments");
    double t = 0;
    for (int k = 0; k < p; ++k) ds[k] = tau * dgamma[k];
    for (int k = 0; k < p; ++k) {
        t += s[k] * dgamma[k];
        const double A = 1.0 - s[k];
        if (k + 1 < p) {
            t -= 0.5 * ((1.0 - s[k + 1]) + A) * dbeta[k];
            ds[k + 1] += 0.5 * tau * dbeta[k];
        } else {
            t -= 0.5 * A * dbeta[k];
        }
        ds[k] += 0.5 * tau * dbeta[k];
    }
    *dtau = t;
    return QS_OK;
}

int qs_qsds_layers(int n, int nsteps, double tau, const double* A, const double* B, const double* hfield,
                   double* gamma, double* u) {
    if (n < 1 || n > QS_MAX_QUBITS_C64 || nsteps < 0 || nsteps + 1 > QS_MAX_LAYERS_PREP || !std::isfinite(tau))
        return set_error(QS_EINVAL, "qs_qsds_layers: bad n, nsteps or tau");
    if ((nsteps > 0 && (!A || !B || !hfield)) || !gamma || !u) return set_error(QS_EINVAL, "qs_qsds_layers: NULL argument");
    using cd = std::complex<double>;
    struct M2 { cd a, b, c, d; };  // [[a, b], [c, d]]
    auto mul = [](const M2& x, const M2& y) {
        return M2{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
    };
    // exp(i theta (ax X + bz Z)) = cos(theta r) + i sin(theta r) (ax X + bz Z) / r
    auto spin = [](double theta, double ax, double bz) {
        const double r = std::sqrt(ax * ax + bz * bz), c = std::cos(theta * r);
        const double sr = r > 0.0 ? std::sin(theta * r) / r : 0.0;
        const cd i(0.0, 1.0);
        return M2{c + i * sr * bz, i * sr * ax, i * sr * ax, c - i * sr * bz};
    };
    const M2 id{1.0, 0.0, 0.0, 1.0};
    auto put = [&](int layer, int q, const M2& m) {
        double* d = u + ((size_t)layer * n + q) * 8;
        const cd e[4] = {m.a, m.b, m.c, m.d};
        for (int k = 0; k < 4; ++k) { d[2 * k] = e[k].real(); d[2 * k + 1] = e[k].imag(); }
    };
    // step l: S_l Z_l S_l with S_l = exp[i tau/2 sum (A_l X - B_l h Z)] and
    // Z_l = exp[-i tau B_l sum J Z Z].  The engine's layer k applies
    // exp(-i gamma_k H_C) (fields included) and then per-qubit matrices, so
    // the fields' part F_l = exp(-i tau B_l h Z) of that phase is undone in
    // the following matrices: Z_l = F_l^{-1} exp(-i tau B_l H_C), and F_l^{-1}
    // commutes with the phase.  Layer 0: gamma = 0, S_0; layer l + 1: gamma =
    // tau B_l, S_{l+1} S_l F_l^{-1} (S_nsteps = 1).
    gamma[0] = 0.0;
    for (int q = 0; q < n; ++q) put(0, q, nsteps > 0 ? spin(0.5 * tau, A[0], -B[0] * hfield[q]) : id);
    for (int l = 0; l < nsteps; ++l) {
        gamma[l + 1] = tau * B[l];
        for (int q = 0; q < n; ++q) {
            const M2 Sl = spin(0.5 * tau, A[l], -B[l] * hfield[q]);
            const M2 Sn = l + 1 < nsteps ? spin(0.5 * tau, A[l + 1], -B[l + 1] * hfield[q]) : id;
            const double th = tau * B[l] * hfield[q];
            const M2 Finv{std::polar(1.0, th), 0.0, 0.0, std::polar(1.0, -th)};  // exp(+i tau B h Z)
            put(l + 1, q, mul(Sn, mul(Sl, Finv)));
        }
    }
    return QS_OK;
}

int qs_launch_count(int64_t* count) {
    if (!count) return set_error(QS_EINVAL, "qs_launch_count: NULL");
    *count = launch_total();
    return QS_OK;
}

const char* qs_last_error(void) { return g_last_error.c_str(); }

const char* qs_version(void) { return "qs-gb300 0.1 (sm_103a)"; }

}  // extern "C"
