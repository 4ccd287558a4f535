// Internal declarations shared by the host API and the kernels.
// Nothing here is part of the public ABI (include/qs.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

namespace qs {

// ---------------------------------------------------------------------------
// Tiling constants.
//
// A sweep reads every amplitude once and writes it once.  The 2^n index bits
// are split into "tile bits" (held on chip by one CTA) and the rest (which
// tile).  A tile shape is: the c lowest index bits (carried, only there so
// that each tile row is contiguous in HBM) plus a contiguous run of target
// bits [g0, g0 + K - c) whose x-rotations the sweep applies.  The first shape
// (shape A) has c = 0 and targets [0, K_A).
// ---------------------------------------------------------------------------
constexpr int kMinPhysQubits = 13;   // states with n < 13 are padded with idle qubits
constexpr int kMaxRounds = 8;        // rounds (layers) fused into one sweep
constexpr int kMaxShapes = 4;        // tile shapes per plan
constexpr int kMaxLayouts = 3;       // register layouts per tile shape
constexpr int kRunBits = 8;          // run-structured shape A: runs of 2^8 amplitudes
constexpr int kPlanRuleInts = 8;     // ints of a plan rule (QS_PLAN_RULE_INTS)
#define QS_MAX_LAYERS_PREP 1024          // layers per preparation call

// Register-layout parameters per kernel configuration.
struct KernelCfg {
    int K_A;   // tile bits of shape A
    int K_B;   // tile bits of shapes B, C, ...
    int R;     // register bits per thread
    int c_min; // carried low bits of shapes B, C, ... (row = 2^c elements)
};
KernelCfg kernel_cfg(int dtype, bool adjoint);

// Flags of a sweep task.
enum : int {
    T_GEN = 1,        // generate |+> instead of loading (first forward sweep)
    T_READOUT = 2,    // accumulate E, P, norm after the last round
    T_WRITE_LAM = 4,  // write lambda = O psi (adjoint forward pass)
    T_STORE = 8,      // write the tile back (clear only for the last reverse sweep)
    T_ADJOINT = 16,   // two arrays (psi, lambda), gradient accumulation
    T_ZEXP = 32,      // record <Z_q> of the layer ending at each phase point and at the readout
    T_TAB = 64,       // work queue: the tile needs its cost table (a phase or a readout)
    T_SU2 = 128       // general single-spin unitaries per layer and qubit instead of x rotations
};

// Per-layer spin expectations <Z_q> (Sec. III.B.2, Fig. 6): every CTA of a
// T_ZEXP sweep keeps FP64 accumulators in shared memory, one record of kZQ
// qubits per round (the state after the previous layer, seen at the round's
// phase) and one for the readout (slot kMaxRounds), and writes them to
// zpart[blockIdx.x][kZSlots][kZQ] when it exits.
constexpr int kZQ = 36;                  // qubits per record (>= the largest state)
constexpr int kZSlots = kMaxRounds + 1;  // records per CTA

// Kernel variants: FULL has every feature; PHASE (middle sweeps with a layer
// boundary) drops |+> generation, readout and lambda; LEAN (middle sweeps
// without a phase) also drops the phase.  Leaner variants keep the
// instruction footprint of the hot loop small.  ZFULL is FULL with the spin
// expectations of T_ZEXP sweeps; ZPHASE is PHASE with them (the packed-pair
// kernel; sweep_kernel runs ZPHASE sweeps as ZFULL).  SU2 is FULL with
// general per-qubit 2 x 2 unitaries in place of the x rotations.
enum : int { V_FULL = 0, V_PHASE = 1, V_LEAN = 2, V_ZFULL = 3, V_ZPHASE = 4, V_SU2 = 5 };
// Run-structured shape A only (sweep_runs_kernel): the first sweep of an
// evolve (|+> generated, the first layer's phase and rotations; no load)
// and the last one (rotations, then E, P_ground and the norm per tile).
enum : int { V_RUNS_GEN = 6, V_RUNS_READ = 7 };

struct SweepRound {
    int layer;       // index into the per-layer parameter array
    int phase_pre;   // apply the layer's phase before the rotations
    int phase_post;  // apply the layer's (inverse) phase after the rotations
    int r0;          // targets of this layer rotated in earlier sweeps (adjoint scale)
};

// Per-layer device parameters, produced on the device from the angles.
struct LayerDev {
    double w;       // butterfly weight: a' = a + w (-i b), |w| <= 1 (float-exact for complex64)
    double fabs;    // |f| = 1 / sqrt(1 + w^2): magnitude of the per-rotation scalar factor
    double c, s;    // cos(beta), sin(beta) (plain path)
    int frame;      // basis frame (0 / 1 = all bits flipped) when this layer's phase acts
    int var;        // 1: cotangent form (flips the frame)
};

// Header length (int32 words) of a tile program (see build_tile_prog).
constexpr int kTileProgHead = 20;

struct SweepTask {
    int kind;                    // 0 contiguous, 1 strided
    int n1, g1;                  // strided: second target run (see Shape)
    void* psi;
    void* lam;
    const LayerDev* layers;
    const void* tab;             // per-layer phase tables [layer][tab_stride] (Real2)
    const int32_t* cprog[kMaxLayouts];  // layout programs (build_layout_prog) of the kernel's layouts
    const int32_t* tprog;        // tile program of the shape (build_tile_prog)
    double* partials;            // per tile: np doubles
    double* zpart;               // T_ZEXP: per CTA kZSlots * kZQ doubles
    const double* su2;           // T_SU2: per layer and qubit a 2 x 2 unitary (8 doubles, row major)
    int64_t ntiles;
    int64_t part_base;           // first partial slot of this task
    int n, c, g0, flags;
    int nrounds, objective;
    int tab_stride, cost_lo;     // table index = cost - cost_lo
    int gidx;                    // cmin - cost_lo (ground-state table index)
    int end_layer;               // layers[end_layer].frame = frame after the last round
    double amp0;                 // 2^{-n/2} for T_GEN
    int np;                      // doubles per tile in partials
    int dep;                     // work queue: the instance whose tile counter orders this task
    int64_t need;                // work queue: tiles of that instance to complete before any tile of this task
    SweepRound rounds[kMaxRounds];
};

// Intra-register coupling tables Q[m] of the two packed-pair forward layouts
// of one tile shape, passed to the kernel by value (kernel parameters sit in
// the constant bank, so each compile-time Q[g][m] is an instruction operand).
struct PairQ {
    int32_t q[2][64];
};

// The same for the three packed-pair adjoint layouts (2^5 slots each).
struct PairAdjQ {
    int32_t q[3][32];
};

// How a packed-pair forward launch loads its strided tiles.  tma = 0:
// per-thread 16-byte cp.async copies.  tma = 1: two tensor-map copies per
// tile (one launch = one task), the map of its state buffer (rank 3 to 5,
// float elements, no swizzle, dimensions in the landing order of
// pair_tma_pos; L2 promotion l2: 0 none, 1 128 bytes, 2 256 bytes) and, per
// dimension, the first global index bit and the bits it spans, from which
// the kernel forms a tile's coordinates; the pack bit (global bit kbit)
// selects one of the tile's two box copies.
struct PairLoad {
    CUtensorMap map;
    int lo[5], nb[5];
    int rank, kbit;
    int tma, l2;
};

// A sweep over a list of tasks (one tile shape per launch).
struct SweepLaunch {
    int kind;              // tile kind (selects the kernel with dtype / adjoint / variant)
    int variant;           // 0 full, 1 phase, 2 rotations only (sweep_variant)
    int adjoint;
    int dtype;
    int ntasks;
    int64_t total_tiles;
    const SweepTask* tasks;        // device
    const int64_t* tile_prefix;    // device, ntasks + 1
    int* err;                      // device error word (set on a timed-out wait)
    int group = 1;                 // consecutive tiles per CTA turn (a power of 2)
    int pairc = 0;                 // 2 or 3: packed-pair kernel for carried bits c (qs_pair.h)
    const PairQ* pq = nullptr;     // host: Q tables of the shape (packed-pair forward sweeps)
    const PairAdjQ* paq = nullptr; // host: Q tables of the shape (packed-pair adjoint sweeps)
    int cluster = 4;               // strided packed-pair forward: 4-CTA clusters (line sharing) or 1
    const PairLoad* load = nullptr;  // host: strided packed-pair forward tile loads (null: cp.async, default L2)
};

// Cost program: the Ising cost of Eq. (HC) specialised to one register layout.
// Built on the host (see build_cost_prog), evaluated per thread on the device.
//   [0] R  [1] nf  [2] ne  [3] const0  [4..10) regq
//   then nf pairs (i, h), ne pairs (i | j << 8, J),
//   then for b < R: (fb0, cnt, cnt pairs (j, J)), then Q[2^R].
std::vector<int32_t> build_cost_prog(int n, const std::vector<int32_t>& h, const std::vector<int32_t>& ei,
                                     const std::vector<int32_t>& ej, const std::vector<int32_t>& J,
                                     const int* regq, int R);

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All return cudaError_t.
cudaError_t launch_sweep_pair(const SweepLaunch& L, int grid, cudaStream_t st);
cudaError_t launch_sweep_pair_adj(const SweepLaunch& L, int grid, cudaStream_t st);
int sweep_pair_adj_grid();
int sweep_pair_grid(int variant);  // variant as sweep_variant: 1 phase, 2 rotations only
// Packed-pair forward sweep of the run-structured shape A (V_PHASE, V_LEAN).
cudaError_t launch_sweep_runs(const SweepLaunch& L, int grid, cudaStream_t st);
int sweep_runs_grid(int variant);
// Packed-pair kernel choice for a sweep, else 0: the carried-bit count c (2
// or 3) for a strided complex64 sweep (forward: without readout; adjoint:
// every reverse sweep), 1 for a sweep of the run-structured shape A (adjoint:
// every reverse sweep; forward: without |+> generation or readout).
int pair_choice(int dtype, int adjoint, int kind, int c, int variant);
// ---------------------------------------------------------------------------
// Launch accounting (qs_launch_count): every launcher reports its kernels.
cudaError_t note_launch(cudaError_t e, int kernels = 1);
int64_t launch_total();

cudaError_t launch_sweep(const SweepLaunch& L, int grid, cudaStream_t st);

// Persistent work queue over every tile of every task of a batch (complex64,
// kinds 0 and 1): CTAs take tiles in task order from the counter *next; a
// tile of task t starts once done[t.dep] >= t.need (a bounded wait of
// wait_ns, reported through err) and adds one to done[t.dep] when stored.
struct QueueLaunch {
    int adjoint;
    int ntasks;
    int64_t total_tiles;
    const SweepTask* tasks;           // device
    const int64_t* tile_prefix;       // device, ntasks + 1
    const int* item_task;             // device, total_tiles: the task of every item
    const int2* depneed;              // device, ntasks: (dep, need) of every task
    unsigned long long* next;         // device, zeroed before the launch
    unsigned int* done;               // device, one per instance, zeroed before the launch
    int* err;
    uint64_t wait_ns;
};
cudaError_t launch_queue(const QueueLaunch& Q, int grid, cudaStream_t st);
int queue_grid(int adjoint);
int sweep_grid(int dtype, int adjoint, int kind);   // persistent grid size
// Leanest kernel variant that can run a sweep with these flags and rounds.
int sweep_variant(int flags, int nrounds, const SweepRound* rounds);

// Layer preparation: angles -> LayerDev + phase tables (forward or reverse).
cudaError_t launch_prep(int dtype, int p, const double* gamma, const double* beta, int nphys,
                        int cost_lo, int range, int shift, const int* frame0, int reverse,
                        LayerDev* layers, void* tab, int tab_stride, cudaStream_t st);

// Batched variant: one block per instance.
struct PrepTask {
    const double* gamma; const double* beta;
    int p, nphys, cost_lo, range, shift, reverse;
    const int* frame0;
    LayerDev* layers; void* tab; int tab_stride;
};
cudaError_t launch_prep_batch(int dtype, const PrepTask* tasks, int ntasks, cudaStream_t st);

// Reduce per-tile readout partials (E, P, norm) of one task into out[3].
struct ReduceTask {
    const double* partials;  // np doubles per tile
    int64_t ntiles;
    int np, off, count;      // reduce slots [off, off+count) of each tile
    double* out;             // count doubles
    int accumulate;          // add into out instead of overwriting
    double mult;             // out (+)= mult * sum
};
cudaError_t launch_reduce(const ReduceTask* tasks, int ntasks, cudaStream_t st);
// Block b reduces tasks [seg[b], seg[b + 1]) in order (tasks sharing an
// output must sit in one segment).
cudaError_t launch_reduce_seg(const ReduceTask* tasks, const int* seg, int nseg, cudaStream_t st);

// Full-enumeration ground-state search of a cost program with register bits
// 0..5 over 2^n states: writes (cmin, cmax, argmin, count) as int64 into out.
cudaError_t launch_enumerate(const int32_t* cprog, int n, int64_t* scratch, int64_t nscratch, int64_t* out,
                             cudaStream_t st);

// Plain (one launch per gate) kernels.
cudaError_t launch_plain_init(int dtype, void* psi, int nphys, cudaStream_t st);
cudaError_t launch_plain_phase(int dtype, void* psi, int nphys, const int32_t* terms, int nf, int ne, int const0,
                               const LayerDev* layer, const void* tab, int cost_lo, int range, cudaStream_t st);
cudaError_t launch_plain_rx(int dtype, void* psi, int nphys, int q, const LayerDev* layer, cudaStream_t st);
cudaError_t launch_plain_readout(int dtype, const void* psi, int nphys, const int32_t* terms, int nf, int ne,
                                 int const0, int cmin, const int* frame, double* partials, int64_t nblocks,
                                 cudaStream_t st);
int64_t plain_readout_blocks(int nphys);
cudaError_t launch_flip_all(int dtype, void* psi, int nphys, cudaStream_t st);
cudaError_t launch_set_frame(int* frame_dev, const LayerDev* layers, int p, cudaStream_t st);

// Batched Adam on device angles.
cudaError_t launch_adam(double* theta, const double* grad, double* m, double* v, int64_t count, const int* step,
                        double lr, double b1, double b2, double eps, cudaStream_t st);
cudaError_t launch_gather_grad(const double* dsrc, double* ddst, int64_t count, cudaStream_t st);
cudaError_t launch_step_inc(int* step, cudaStream_t st);

}  // namespace qs
