// C ABI of include/qs.h: batched instances.
//
// Every instance keeps its own tile shapes and zig-zag sweep list.  A forward
// of the whole batch is one launch of the persistent work-queue kernel
// (qs_queue.cu) over the tiles of every sweep of every instance, ordered wave
// by wave (the w-th sweep of each instance, then the next), with one tile
// counter per instance ordering an instance's sweeps; the adjoint's reverse
// sweeps are a second such launch.  Small states therefore share the GPU
// with large ones, and instances with few layers leave no idle waves.  The
// whole optimiser step (preparation, forward queue, reverse queue,
// reductions, Adam) has static launch parameters, so it can be captured once
// in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qs.h"
#include "qs_api_common.h"

using namespace qs;

namespace {

// Dependency wait limit of the queue kernel (device time).
constexpr uint64_t kQueueWaitNs = 4000000000ull;
// Tiles of one work-queue launch (its item -> task table holds 4 bytes each).
constexpr int64_t kQueueMaxTiles = (int64_t)1 << 26;

// One work-queue launch: its task list, tile prefix and reductions.
struct QueuePlan {
    int ntasks = 0;
    int64_t total = 0;
    size_t task_off = 0, pre_off = 0, red_off = 0, seg_off = 0;  // byte offsets in the uploaded blob
    size_t item_off = 0, dn_off = 0;                             // item -> task table, (dep, need) per task
    int nred = 0, nseg = 0;  // reductions, grouped into segments by output
};

struct Blob {
    std::vector<unsigned char> b;
    size_t add(const void* p, size_t n) {
        size_t off = (b.size() + 63) & ~size_t(63);  // 64-byte aligned records
        b.resize(off + n);
        if (n) std::memcpy(b.data() + off, p, n);
        return off;
    }
};

}  // namespace

struct qs_batch {
    int count = 0, dtype = 0, device = 0;
    cudaStream_t st = nullptr;
    std::vector<int> n, nphys;
    std::vector<Instance> inst;
    std::vector<size_t> st_off;  // element offsets of each state
    DevBuf states, lams, enum_scratch;
    // per-evolve data
    std::vector<int> p;
    std::vector<int64_t> aoff;
    int64_t total = 0;
    std::vector<double> host_angles;  // [gamma_all, beta_all]
    DevBuf angles, grads, adam_m, adam_v, step, err;
    DevBuf layers_f, layers_r, tab_f, tab_r, partials, out, frames;
    std::vector<size_t> lay_off, tab_off;  // per instance: LayerDev index / table element offsets
    Uploader up;
    // plans (device blob in up.dev)
    QueuePlan fwd_q, rev_q;
    DevBuf qctl;  // queue counter (u64) + per-instance tile counters (u32), zeroed per launch
    size_t prep_f_off = 0, prep_r_off = 0;
    bool plan_grad = false, planned = false;
    int grid[2] = {};  // [adjoint]: persistent queue grid
    uint64_t wait_ns = kQueueWaitNs;  // dependency wait limit
    int withhold = -1;  // failure-detection test: the instance whose dependency is withheld
    int ctas_per_sm = 0;       // launch rule: persistent queue CTAs per SM (0 = as many as fit)
    int64_t window_bytes = 0;  // queue order: instance windows of at most this many state bytes (0 = one)
    cudaGraphExec_t graph = nullptr;
    bool have_results = false;
    bool poisoned = false;  // a kernel exited with a tile copy possibly still in flight
    int objective = 0;
};

static int bgrid(qs_batch_handle b, int adjoint) {
    int& g = b->grid[adjoint];
    if (!g) g = queue_grid(adjoint);
    if (b->ctas_per_sm > 0) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        return std::min(g, b->ctas_per_sm * sms);
    }
    return g;
}

// After a synchronisation: report (and clear) a timed-out device wait.
static int batch_check_err(qs_batch_handle b) {
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, b->err.ptr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "error word");
    if (!v) return QS_OK;
    cudaMemset(b->err.ptr, 0, sizeof(int));
    b->have_results = false;
    if (v >= 2) {
        b->poisoned = true;
        return set_error(QS_ETIMEOUT, "a sweep kernel gave up waiting for a tile copy and for its drain; results "
                                      "are invalid and the batch is unusable");
    }
    return set_error(QS_ETIMEOUT, "a sweep kernel gave up waiting for a tile copy; results are invalid");
}

static int check_batch(qs_batch_handle b) {
    if (!b) return set_error(QS_EINVAL, "NULL batch");
    if (b->poisoned)
        return set_error(QS_ESTATE, "the batch is unusable after a tile copy outlived its kernel; destroy it and "
                                    "create a new one");
    return QS_OK;
}

static void drop_graph(qs_batch_handle b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

extern "C" {

int qs_batch_create(qs_batch_handle* out, int count, const int* n, int dtype, void* cuda_stream) {
    if (!out) return set_error(QS_EINVAL, "qs_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || count > (1 << 20) || !n) return set_error(QS_EINVAL, "qs_batch_create: bad count or n");
    if (dtype != QS_C64) return set_error(QS_EINVAL, "qs_batch_create: only QS_C64 batches are supported");
    std::unique_ptr<qs_batch> b(new qs_batch);
    b->count = count;
    b->dtype = dtype;
    b->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > QS_MAX_QUBITS_C64) return set_error(QS_EINVAL, "qs_batch_create: n[%d] = %d", i, n[i]);
        b->n.push_back(n[i]);
        const int np = n[i] < kMinPhysQubits ? kMinPhysQubits : n[i];
        b->nphys.push_back(np);
        b->st_off.push_back(total);
        total += (size_t)1 << np;  // >= 2^13 elements keep every state 256-byte aligned
    }
    if (int rc = b->states.reserve(total * 8)) return rc;
    if (int rc = b->err.reserve(sizeof(int))) return rc;
    e = cudaMemset(b->err.ptr, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "qs_batch_create");
    b->inst.resize(count);
    *out = b.release();
    return QS_OK;
}

int qs_batch_set_ising(qs_batch_handle b, int idx, const double* hfield, int n_edges, const int32_t* edges,
                       const double* J) {
    if (int rc = check_batch(b)) return rc;
    if (idx < 0 || idx >= b->count) return set_error(QS_EINVAL, "qs_batch_set_ising: idx %d out of range", idx);
    cudaSetDevice(b->device);
    Instance tmp;
    // contiguous shape A for every size: the queue kernel serves contiguous
    // and strided tiles
    if (int rc = tmp.set(b->n[idx], b->nphys[idx], b->dtype, hfield, n_edges, edges, J, b->st, b->enum_scratch,
                         ShapeRule{0, -1}))
        return rc;
    b->inst[idx] = std::move(tmp);
    b->planned = false;
    drop_graph(b);
    return QS_OK;
}

}  // extern "C"

// Build the queue plans and the layer / table buffers for the current p[].
static int build_plan(qs_batch_handle b, bool grad, int objective) {
    const int C = b->count;
    // layer and table offsets
    b->lay_off.assign(C, 0);
    b->tab_off.assign(C, 0);
    size_t lay = 0, tab = 0;
    for (int i = 0; i < C; ++i) {
        b->lay_off[i] = lay;
        b->tab_off[i] = tab;
        lay += (size_t)b->p[i] + 1;
        tab += (size_t)std::max(b->p[i], 1) * b->inst[i].range;
    }
    if (int rc = b->layers_f.reserve(lay * sizeof(LayerDev))) return rc;
    if (int rc = b->tab_f.reserve(tab * 8)) return rc;
    if (grad) {
        if (int rc = b->layers_r.reserve(lay * sizeof(LayerDev))) return rc;
        if (int rc = b->tab_r.reserve(tab * 8)) return rc;
    }
    if (int rc = b->frames.reserve((size_t)C * sizeof(int))) return rc;
    if (int rc = b->out.reserve((size_t)C * 3 * sizeof(double))) return rc;
    if (int rc = b->grads.reserve((size_t)std::max<int64_t>(2 * b->total, 1) * sizeof(double))) return rc;
    if (grad && !b->lams.ptr) {
        if (int rc = b->lams.reserve(b->states.cap)) return rc;
    }

    std::vector<std::vector<PlanSweep>> fwd(C), rev(C);
    size_t maxf = 0, maxr = 0;
    for (int i = 0; i < C; ++i) {
        fwd[i] = plan_forward((int)b->inst[i].shapes[0].size(), b->p[i], true);
        if (grad) {
            fwd[i].back().flags |= T_WRITE_LAM;
            rev[i] = plan_reverse(fwd[i], b->inst[i].shapes[1], b->p[i]);
        }
        maxf = std::max(maxf, fwd[i].size());
        maxr = std::max(maxr, rev[i].size());
    }
    double* dout = reinterpret_cast<double*>(b->out.ptr);
    double* dgr = reinterpret_cast<double*>(b->grads.ptr);
    float2* states = reinterpret_cast<float2*>(b->states.ptr);
    float2* lams = reinterpret_cast<float2*>(b->lams.ptr);
    const LayerDev* lf = reinterpret_cast<const LayerDev*>(b->layers_f.ptr);
    const LayerDev* lr = reinterpret_cast<const LayerDev*>(b->layers_r.ptr);
    const float2* tf = reinterpret_cast<const float2*>(b->tab_f.ptr);
    const float2* tr = reinterpret_cast<const float2*>(b->tab_r.ptr);

    Blob blob;
    // partials: one block per task with readout or adjoint sums (the forward
    // queue's reductions run before the reverse queue reuses the buffer)
    auto queue_partials = [&](const std::vector<std::vector<PlanSweep>>& L, int cfgi) {
        size_t need = 0;
        for (int i = 0; i < C; ++i)
            for (const PlanSweep& s : L[i]) {
                const Shape& sh = b->inst[i].shapes[cfgi][s.shape];
                const int np = (s.flags & T_ADJOINT) ? 2 * s.nr : ((s.flags & T_READOUT) ? 3 : 0);
                need += (size_t)sh.ntiles * np;
            }
        return need;
    };
    const size_t part_need = std::max(queue_partials(fwd, 0), grad ? queue_partials(rev, 1) : size_t(0));
    if (int rc = b->partials.reserve((part_need + 4) * sizeof(double))) return rc;
    double* dpart = reinterpret_cast<double*>(b->partials.ptr);
    if (int rc = b->qctl.reserve(64 + (size_t)C * sizeof(unsigned))) return rc;

    // Instance windows: consecutive instances whose states together hold at
    // most window_bytes (at least one each; all instances when 0).  Within a
    // window the queue runs wave by wave, so a window's states can stay in
    // L2 between its sweeps.
    std::vector<std::vector<int>> windows;
    {
        int64_t acc = 0;
        for (int i = 0; i < C; ++i) {
            const int64_t bytes = (int64_t)8 << b->nphys[i];
            if (windows.empty() || (b->window_bytes > 0 && acc + bytes > b->window_bytes)) {
                windows.emplace_back();
                acc = 0;
            }
            windows.back().push_back(i);
            acc += bytes;
        }
    }
    (void)maxf;
    (void)maxr;
    // the task list of one queue, window by window and wave by wave inside a
    // window; task (i, w) needs every tile of instance i's sweeps 0..w-1
    auto build_queue = [&](const std::vector<std::vector<PlanSweep>>& L, int adj, QueuePlan& out) {
        std::vector<SweepTask> tasks;
        std::vector<int64_t> pre{0}, need(C, 0);
        std::vector<ReduceTask> rts;
        int64_t pbase = 0;
        for (const std::vector<int>& win : windows) {
          size_t nw = 0;
          for (int i : win) nw = std::max(nw, L[i].size());
          for (size_t w = 0; w < nw; ++w) {
            for (int i : win) {
                if (w >= L[i].size()) continue;
                const PlanSweep& s = L[i][w];
                const Instance& I = b->inst[i];
                const Shape& sh = I.shapes[adj][s.shape];
                SweepTask t;
                std::memset(&t, 0, sizeof t);
                t.psi = states + b->st_off[i];
                t.lam = lams ? lams + b->st_off[i] : nullptr;
                t.layers = (adj ? lr : lf) + b->lay_off[i];
                t.tab = (adj ? tr : tf) + b->tab_off[i];
                for (int g = 0; g < kMaxLayouts; ++g) t.cprog[g] = I.prog(I.prog_off[adj][s.shape][g]);
                t.tprog = I.prog(I.tprog_off[adj][s.shape]);
                t.ntiles = sh.ntiles;
                t.part_base = 0;
                t.n = b->nphys[i];
                t.c = sh.c;
                t.g0 = sh.g0;
                t.flags = s.flags;
                bool tab = (s.flags & (T_READOUT | T_WRITE_LAM)) != 0;
                for (int r = 0; r < s.nr; ++r) tab = tab || s.r[r].phase_pre || s.r[r].phase_post;
                if (tab) t.flags |= T_TAB;
                t.nrounds = s.nr;
                t.objective = objective;
                t.tab_stride = I.range;
                t.cost_lo = I.cost_lo;
                t.gidx = (int)(I.cmin - I.cost_lo);
                t.end_layer = b->p[i];
                t.amp0 = std::pow(2.0, -0.5 * b->nphys[i]);
                t.np = (s.flags & T_ADJOINT) ? 2 * s.nr : ((s.flags & T_READOUT) ? 3 : 0);
                for (int r = 0; r < s.nr; ++r) t.rounds[r] = s.r[r];
                t.kind = sh.kind;
                t.n1 = sh.n1;
                t.g1 = sh.g1;
                t.dep = i;
                t.need = need[i];
                if (adj == 0 && w == 1 && i == b->withhold) t.need += 1;  // never satisfied: the wait runs out
                need[i] += sh.ntiles;
                // this task's partial block: (part_base + tile) * np indexes it
                const double* tp = dpart + pbase;
                t.partials = dpart + pbase;
                const double sc = std::ldexp(1.0, -I.shift);
                if (s.flags & T_READOUT) {
                    rts.push_back(ReduceTask{tp, sh.ntiles, 3, 0, 1, dout + 3 * i, 0, sc});
                    rts.push_back(ReduceTask{tp, sh.ntiles, 3, 1, 2, dout + 3 * i + 1, 0, 1.0});
                }
                if (s.flags & T_ADJOINT) {
                    const double lam_sc = objective == QS_OBJ_ENERGY ? sc : 1.0;
                    for (int r = 0; r < s.nr; ++r) {
                        const int Ly = s.r[r].layer;
                        double* db = dgr + b->total + b->aoff[i] + Ly;
                        double* dg = dgr + b->aoff[i] + Ly;
                        rts.push_back(ReduceTask{tp, sh.ntiles, 2 * s.nr, 2 * r, 1, db, 1, 2.0 * lam_sc});
                        if (s.r[r].phase_post)
                            rts.push_back(ReduceTask{tp, sh.ntiles, 2 * s.nr, 2 * r + 1, 1, dg, 1, 2.0 * sc * lam_sc});
                    }
                }
                pbase += (int64_t)sh.ntiles * t.np;
                tasks.push_back(t);
                pre.push_back(pre.back() + sh.ntiles);
            }
          }
        }
        out.ntasks = (int)tasks.size();
        out.total = pre.back();
        out.task_off = tasks.empty() ? 0 : blob.add(tasks.data(), tasks.size() * sizeof(SweepTask));
        out.pre_off = blob.add(pre.data(), pre.size() * sizeof(int64_t));
        std::vector<int> item_task((size_t)out.total);
        std::vector<int2> dn(tasks.size());
        for (size_t k = 0; k < tasks.size(); ++k) {
            for (int64_t it = pre[k]; it < pre[k + 1]; ++it) item_task[(size_t)it] = (int)k;
            dn[k] = make_int2(tasks[k].dep, (int)tasks[k].need);
        }
        out.item_off = item_task.empty() ? 0 : blob.add(item_task.data(), item_task.size() * sizeof(int));
        out.dn_off = dn.empty() ? 0 : blob.add(dn.data(), dn.size() * sizeof(int2));
        // every output (an instance's E, P or one angle derivative) gets the
        // sums of several tasks (one per tile shape): group them by output,
        // in plan order, so that one block adds them in a fixed order
        std::stable_sort(rts.begin(), rts.end(),
                         [](const ReduceTask& a, const ReduceTask& b2) { return a.out < b2.out; });
        std::vector<int> seg{0};
        for (size_t k = 1; k < rts.size(); ++k)
            if (rts[k].out != rts[k - 1].out) seg.push_back((int)k);
        seg.push_back((int)rts.size());
        out.nred = (int)rts.size();
        out.nseg = rts.empty() ? 0 : (int)seg.size() - 1;
        out.red_off = rts.empty() ? 0 : blob.add(rts.data(), rts.size() * sizeof(ReduceTask));
        out.seg_off = rts.empty() ? 0 : blob.add(seg.data(), seg.size() * sizeof(int));
    };
    // the item -> task table (4 bytes per tile of every sweep) bounds a queue
    auto queue_tiles = [&](const std::vector<std::vector<PlanSweep>>& L, int cfgi) {
        int64_t t = 0;
        for (int i = 0; i < C; ++i)
            for (const PlanSweep& s : L[i]) t += b->inst[i].shapes[cfgi][s.shape].ntiles;
        return t;
    };
    if (queue_tiles(fwd, 0) > kQueueMaxTiles || (grad && queue_tiles(rev, 1) > kQueueMaxTiles))
        return set_error(QS_EINVAL, "batch too large: more than %lld tiles in one work queue; split the batch",
                         (long long)kQueueMaxTiles);
    build_queue(fwd, 0, b->fwd_q);
    if (grad) build_queue(rev, 1, b->rev_q);
    else b->rev_q = QueuePlan{};

    // preparation tasks (angles live in b->angles: [gamma_all, beta_all])
    const double* da = reinterpret_cast<const double*>(b->angles.ptr);
    std::vector<PrepTask> pf, pr;
    for (int i = 0; i < C; ++i) {
        const Instance& I = b->inst[i];
        PrepTask t{da + b->aoff[i], da + b->total + b->aoff[i], b->p[i], b->nphys[i], I.cost_lo, I.range, I.shift, 0,
                   nullptr, const_cast<LayerDev*>(lf) + b->lay_off[i], const_cast<float2*>(tf) + b->tab_off[i], I.range};
        pf.push_back(t);
        t.reverse = 1;
        t.layers = const_cast<LayerDev*>(lr) + b->lay_off[i];
        t.tab = const_cast<float2*>(tr) + b->tab_off[i];
        pr.push_back(t);
    }
    b->prep_f_off = blob.add(pf.data(), pf.size() * sizeof(PrepTask));
    b->prep_r_off = grad ? blob.add(pr.data(), pr.size() * sizeof(PrepTask)) : 0;
    if (int rc = b->up.upload(blob.b.data(), blob.b.size(), b->st)) return rc;
    b->plan_grad = grad;
    b->objective = objective;
    b->planned = true;
    drop_graph(b);
    return QS_OK;
}

static int run_queue(qs_batch_handle b, const QueuePlan& q, int adjoint) {
    if (q.ntasks == 0) return QS_OK;
    const unsigned char* d = reinterpret_cast<const unsigned char*>(b->up.dev.ptr);
    unsigned char* ctl = reinterpret_cast<unsigned char*>(b->qctl.ptr);
    cudaError_t e = cudaMemsetAsync(ctl, 0, 64 + (size_t)b->count * sizeof(unsigned), b->st);
    if (e != cudaSuccess) return cuda_error(e, "queue counters");
    QueueLaunch Q{adjoint,
                  q.ntasks,
                  q.total,
                  reinterpret_cast<const SweepTask*>(d + q.task_off),
                  reinterpret_cast<const int64_t*>(d + q.pre_off),
                  reinterpret_cast<const int*>(d + q.item_off),
                  reinterpret_cast<const int2*>(d + q.dn_off),
                  reinterpret_cast<unsigned long long*>(ctl),
                  reinterpret_cast<unsigned*>(ctl + 64),
                  reinterpret_cast<int*>(b->err.ptr),
                  b->wait_ns};
    e = launch_queue(Q, bgrid(b, adjoint), b->st);
    if (e != cudaSuccess) return cuda_error(e, "batched queue sweep");
    if (q.nseg) {
        e = launch_reduce_seg(reinterpret_cast<const ReduceTask*>(d + q.red_off),
                              reinterpret_cast<const int*>(d + q.seg_off), q.nseg, b->st);
        if (e != cudaSuccess) return cuda_error(e, "batched reduce");
    }
    return QS_OK;
}

// One evaluation on the device angles: prep, forward queue (+ reverse queue).
static int run_step(qs_batch_handle b, bool grad) {
    const unsigned char* d = reinterpret_cast<const unsigned char*>(b->up.dev.ptr);
    cudaError_t e = launch_prep_batch(b->dtype, reinterpret_cast<const PrepTask*>(d + b->prep_f_off), b->count, b->st);
    if (e != cudaSuccess) return cuda_error(e, "batched prep");
    if (grad) {
        e = launch_prep_batch(b->dtype, reinterpret_cast<const PrepTask*>(d + b->prep_r_off), b->count, b->st);
        if (e != cudaSuccess) return cuda_error(e, "batched prep reverse");
        e = cudaMemsetAsync(b->grads.ptr, 0, (size_t)2 * b->total * sizeof(double), b->st);
        if (e != cudaSuccess) return cuda_error(e, "zero grads");
    }
    if (int rc = run_queue(b, b->fwd_q, 0)) return rc;
    if (grad)
        if (int rc = run_queue(b, b->rev_q, 1)) return rc;
    return QS_OK;
}

static int upload_angles(qs_batch_handle b) {
    const size_t bytes = (size_t)std::max<int64_t>(2 * b->total, 1) * sizeof(double);
    if (b->angles.cap < bytes) {
        cudaStreamSynchronize(b->st);
        if (int rc = b->angles.reserve(bytes)) return rc;
        b->planned = false;
    }
    cudaError_t e = cudaMemcpyAsync(b->angles.ptr, b->host_angles.data(), 2 * b->total * sizeof(double),
                                    cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // pageable source
    return e == cudaSuccess ? QS_OK : cuda_error(e, "angles upload");
}

extern "C" {

int qs_batch_evolve(qs_batch_handle b, const int* p, const int64_t* angle_off, const double* gamma,
                    const double* beta) {
    if (int rc = check_batch(b)) return rc;
    if (!p || !angle_off || !gamma || !beta) return set_error(QS_EINVAL, "qs_batch_evolve: NULL argument");
    cudaSetDevice(b->device);
    for (int i = 0; i < b->count; ++i) {
        if (!b->inst[i].valid) return set_error(QS_ESTATE, "instance %d has no Ising cost", i);
        if (p[i] < 0 || p[i] > QS_MAX_LAYERS_BATCH) return set_error(QS_EINVAL, "p[%d] = %d out of range", i, p[i]);
        if (angle_off[i] < 0) return set_error(QS_EINVAL, "angle_off[%d] < 0", i);
        for (int k = 0; k < p[i]; ++k)
            if (!std::isfinite(gamma[angle_off[i] + k]) || !std::isfinite(beta[angle_off[i] + k]))
                return set_error(QS_EINVAL, "non-finite angle in instance %d", i);
    }
    // compact angle layout [gamma_all, beta_all]
    bool same = (int)b->p.size() == b->count;
    for (int i = 0; same && i < b->count; ++i) same = b->p[i] == p[i];
    if (!same) {
        b->p.assign(p, p + b->count);
        b->aoff.assign(b->count, 0);
        int64_t t = 0;
        for (int i = 0; i < b->count; ++i) { b->aoff[i] = t; t += p[i]; }
        b->total = t;
        b->planned = false;
    }
    b->host_angles.assign(2 * (size_t)b->total, 0.0);
    for (int i = 0; i < b->count; ++i)
        for (int k = 0; k < p[i]; ++k) {
            b->host_angles[b->aoff[i] + k] = gamma[angle_off[i] + k];
            b->host_angles[b->total + b->aoff[i] + k] = beta[angle_off[i] + k];
        }
    if (int rc = upload_angles(b)) return rc;
    if (!b->planned || b->plan_grad)
        if (int rc = build_plan(b, false, 0)) return rc;
    int rc = run_step(b, false);
    if (b->withhold >= 0) {  // one-shot failure-detection test: back to the normal plan and limit
        b->withhold = -1;
        b->wait_ns = kQueueWaitNs;
        b->planned = false;
    }
    if (rc) return rc;
    b->have_results = true;
    return QS_OK;
}

int qs_batch_set_launch_rule(qs_batch_handle b, int ctas_per_sm, int64_t window_bytes) {
    if (int rc = check_batch(b)) return rc;
    if (ctas_per_sm < 0 || ctas_per_sm > 32 || window_bytes < 0)
        return set_error(QS_EINVAL, "qs_batch_set_launch_rule: ctas_per_sm in [0, 32], window_bytes >= 0");
    b->ctas_per_sm = ctas_per_sm;
    if (window_bytes != b->window_bytes) b->planned = false;
    b->window_bytes = window_bytes;
    drop_graph(b);
    return QS_OK;
}

int qs_batch_autotune(qs_batch_handle b, int* ctas_per_sm, int64_t* window_bytes, double* best_ms) {
    if (int rc = check_batch(b)) return rc;
    if ((int)b->p.size() != b->count) return set_error(QS_ESTATE, "qs_batch_autotune: call qs_batch_evolve first");
    cudaSetDevice(b->device);
    const int keep_c = b->ctas_per_sm;
    const int64_t keep_w = b->window_bytes;
    const int per_sm = std::max(1, bgrid(b, 0) / std::max(1, [&] {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        return sms;
    }()));
    std::vector<int> ctas{0};
    if (per_sm > 1) ctas.push_back(per_sm - 1);
    const int64_t windows[3] = {0, (int64_t)256 << 20, (int64_t)64 << 20};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) return cuda_error(ce, "qs_batch_autotune: events");
    int rc = QS_OK;
    double best = 1e300;
    int pick_c = 0;
    int64_t pick_w = 0;
    for (int64_t w : windows) {
        for (int c : ctas) {
            b->ctas_per_sm = c;
            if (w != b->window_bytes) b->planned = false;
            b->window_bytes = w;
            if (!b->planned || b->plan_grad)
                if ((rc = build_plan(b, false, 0))) break;
            double ms = 1e300;
            for (int rep = 0; rep < 3 && !rc; ++rep) {  // one warm-up, the faster of two runs
                cudaEventRecord(e0, b->st);
                rc = run_step(b, false);
                cudaEventRecord(e1, b->st);
                if (!rc && (ce = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_error(ce, "qs_batch_autotune");
                if (!rc) rc = batch_check_err(b);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, (double)t);
            }
            if (rc) break;
            if (ms < best) { best = ms; pick_c = c; pick_w = w; }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->ctas_per_sm = rc ? keep_c : pick_c;
    b->window_bytes = rc ? keep_w : pick_w;
    b->planned = false;
    drop_graph(b);
    if (rc) return rc;
    b->have_results = false;
    if (ctas_per_sm) *ctas_per_sm = pick_c;
    if (window_bytes) *window_bytes = pick_w;
    if (best_ms) *best_ms = best;
    return QS_OK;
}

int qs_batch_test_withhold(qs_batch_handle b, int idx, double wait_limit_s) {
    if (int rc = check_batch(b)) return rc;
    if (idx < 0 || idx >= b->count) return set_error(QS_EINVAL, "qs_batch_test_withhold: bad instance %d", idx);
    if (!(wait_limit_s > 0.0 && wait_limit_s <= 10.0))
        return set_error(QS_EINVAL, "qs_batch_test_withhold: wait limit must lie in (0, 10] s");
    b->withhold = idx;
    b->wait_ns = (uint64_t)(wait_limit_s * 1e9);
    b->planned = false;
    return QS_OK;
}

int qs_batch_results(qs_batch_handle b, double* E, double* P) {
    if (int rc = check_batch(b)) return rc;
    if (!b->have_results) return set_error(QS_ESTATE, "qs_batch_results: nothing evolved yet");
    cudaSetDevice(b->device);
    std::vector<double> r(3 * (size_t)b->count);
    cudaError_t e = cudaMemcpyAsync(r.data(), b->out.ptr, r.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return cuda_error(e, "qs_batch_results");
    if (int rc = batch_check_err(b)) return rc;
    for (int i = 0; i < b->count; ++i) {
        if (E) E[i] = r[3 * i];
        if (P) P[i] = r[3 * i + 1];
    }
    return QS_OK;
}

int qs_batch_grad(qs_batch_handle b, int objective, double* value, double* dgamma, double* dbeta) {
    if (int rc = check_batch(b)) return rc;
    if ((int)b->p.size() != b->count) return set_error(QS_ESTATE, "qs_batch_grad: call qs_batch_evolve first");
    if (objective != QS_OBJ_ENERGY && objective != QS_OBJ_GROUND) return set_error(QS_EINVAL, "bad objective");
    if (b->total > 0 && (!dgamma || !dbeta)) return set_error(QS_EINVAL, "dgamma or dbeta is NULL");
    cudaSetDevice(b->device);
    if (!b->planned || !b->plan_grad || b->objective != objective)
        if (int rc = build_plan(b, true, objective)) return rc;
    if (int rc = run_step(b, true)) return rc;
    std::vector<double> g(2 * (size_t)b->total), r(3 * (size_t)b->count);
    cudaError_t e = cudaMemcpyAsync(g.data(), b->grads.ptr, g.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.data(), b->out.ptr, r.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return cuda_error(e, "qs_batch_grad");
    if (int rc = batch_check_err(b)) return rc;
    for (int i = 0; i < b->count; ++i) {
        if (value) value[i] = objective == QS_OBJ_ENERGY ? r[3 * i] : r[3 * i + 1];
        for (int k = 0; k < b->p[i]; ++k) {
            dgamma[b->aoff[i] + k] = g[b->aoff[i] + k];
            dbeta[b->aoff[i] + k] = g[b->total + b->aoff[i] + k];
        }
    }
    b->have_results = true;
    return QS_OK;
}

int qs_batch_adam(qs_batch_handle b, int steps, double lr, double b1, double b2, double eps, double* gamma_io,
                  double* beta_io, int use_graph) {
    if (int rc = check_batch(b)) return rc;
    if ((int)b->p.size() != b->count) return set_error(QS_ESTATE, "qs_batch_adam: call qs_batch_evolve first");
    if (steps < 0 || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps > 0))
        return set_error(QS_EINVAL, "qs_batch_adam: bad hyper-parameters");
    if (b->total > 0 && (!gamma_io || !beta_io)) return set_error(QS_EINVAL, "qs_batch_adam: NULL angles");
    cudaSetDevice(b->device);
    for (int i = 0; i < b->count; ++i)
        for (int k = 0; k < b->p[i]; ++k) {
            b->host_angles[b->aoff[i] + k] = gamma_io[b->aoff[i] + k];
            b->host_angles[b->total + b->aoff[i] + k] = beta_io[b->aoff[i] + k];
        }
    if (int rc = upload_angles(b)) return rc;
    if (!b->planned || !b->plan_grad || b->objective != QS_OBJ_ENERGY)
        if (int rc = build_plan(b, true, QS_OBJ_ENERGY)) return rc;
    const size_t nb = (size_t)std::max<int64_t>(2 * b->total, 1) * sizeof(double);
    if (int rc = b->adam_m.reserve(nb)) return rc;
    if (int rc = b->adam_v.reserve(nb)) return rc;
    if (int rc = b->step.reserve(sizeof(int))) return rc;
    cudaError_t e = cudaMemsetAsync(b->adam_m.ptr, 0, nb, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->adam_v.ptr, 0, nb, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->step.ptr, 0, sizeof(int), b->st);
    if (e != cudaSuccess) return cuda_error(e, "adam init");
    double* theta = reinterpret_cast<double*>(b->angles.ptr);
    const double* grad = reinterpret_cast<const double*>(b->grads.ptr);
    auto one_step = [&]() -> int {
        if (int rc = run_step(b, true)) return rc;
        cudaError_t e2 = launch_step_inc(reinterpret_cast<int*>(b->step.ptr), b->st);
        if (e2 == cudaSuccess)
            e2 = launch_adam(theta, grad, reinterpret_cast<double*>(b->adam_m.ptr), reinterpret_cast<double*>(b->adam_v.ptr),
                             2 * b->total, reinterpret_cast<const int*>(b->step.ptr), lr, b1, b2, eps, b->st);
        return e2 == cudaSuccess ? QS_OK : cuda_error(e2, "adam");
    };
    if (use_graph && steps > 0) {
        // the graph bakes in lr, b1, b2, eps: capture a fresh one per call
        drop_graph(b);
        cudaGraph_t g = nullptr;
        cudaStream_t cap = b->st;
        bool own = false;
        if (!cap) {  // the legacy stream cannot be captured
            e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_error(e, "capture stream");
            own = true;
            cudaStreamSynchronize(b->st);
        }
        cudaStream_t saved = b->st;
        b->st = cap;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? one_step() : cuda_error(e, "begin capture");
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        b->st = saved;
        if (rc == QS_OK && e2 != cudaSuccess) rc = cuda_error(e2, "end capture");
        if (rc == QS_OK) {
            e = cudaGraphInstantiate(&b->graph, g, 0);
            if (e != cudaSuccess) rc = cuda_error(e, "graph instantiate");
        }
        if (g) cudaGraphDestroy(g);
        for (int s = 0; rc == QS_OK && s < steps; ++s) {
            e = cudaGraphLaunch(b->graph, cap);
            if (e != cudaSuccess) rc = cuda_error(e, "graph launch");
        }
        if (own) {
            cudaStreamSynchronize(cap);
            cudaStreamDestroy(cap);
            drop_graph(b);
        }
        if (rc) return rc;
    } else {
        for (int s = 0; s < steps; ++s)
            if (int rc = one_step()) return rc;
    }
    // final readout at the optimised angles
    if (int rc = run_step(b, false)) return rc;
    std::vector<double> a(2 * (size_t)b->total);
    e = cudaMemcpyAsync(a.data(), b->angles.ptr, a.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return cuda_error(e, "qs_batch_adam");
    if (int rc = batch_check_err(b)) return rc;
    for (int i = 0; i < b->count; ++i)
        for (int k = 0; k < b->p[i]; ++k) {
            gamma_io[b->aoff[i] + k] = a[b->aoff[i] + k];
            beta_io[b->aoff[i] + k] = a[b->total + b->aoff[i] + k];
        }
    b->host_angles = a;
    b->have_results = true;
    return QS_OK;
}

int qs_batch_partition(int count, const int* n, const int* p, int world, int* rank_of, double* load) {
    if (count < 0 || world < 1 || (count > 0 && (!n || !p || !rank_of)))
        return set_error(QS_EINVAL, "qs_batch_partition: bad arguments");
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > QS_MAX_QUBITS_C64 || p[i] < 0)
            return set_error(QS_EINVAL, "qs_batch_partition: instance %d has n = %d, p = %d", i, n[i], p[i]);
        work[i] = std::ldexp((double)std::max(p[i], 1), n[i]);
    }
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<double> acc(world, 0.0);
    for (int i : order) {
        int r = 0;
        for (int q = 1; q < world; ++q)
            if (acc[q] < acc[r]) r = q;
        rank_of[i] = r;
        acc[r] += work[i];
    }
    if (load)
        for (int q = 0; q < world; ++q) load[q] = acc[q];
    return QS_OK;
}

int qs_batch_destroy(qs_batch_handle b) {
    if (!b) return QS_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->st);
    drop_graph(b);
    delete b;
    return QS_OK;
}

}  // extern "C"
