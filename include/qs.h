/*
 * qs.h — C ABI of the GB300 (sm_103a) state-vector engine for the QAOA /
 * approximate-quantum-annealing (AQA) path of arXiv 2104.03293.
 *
 * The engine evolves an n-qubit state under the layered product of
 * Eq. (QAOA_state),
 *
 *     |beta, gamma> = prod_{k=1}^{p} e^{-i beta_k H_D} e^{-i gamma_k H_C} |+>^n,
 *
 * with the mixer H_D = sum_i X_i (Sec. III.A.2) and the diagonal Ising cost
 * H_C = sum_i h_i Z_i + sum_{i<j} J_ij Z_i Z_j (Eq. HC), and reads out
 * <H_C> and the ground-state ("success") probability (Sec. III.B.1 and the
 * success-probability definition of Sec. III.A.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Basis index z: qubit j is bit j of z, q_0 the least significant bit
 *    (Sec. II.A, the rank-N tensor psi_{q_{N-1}...q_0}).  Z|0> = +|0>, so the
 *    spin of qubit i in state z is s_i(z) = 1 - 2 bit_i(z).
 *  - Within a layer the phase e^{-i gamma_k H_C} acts before the mixer
 *    (Eq. QAOA_state; Appendix A writes the factors out).
 *  - State layout in device memory: 2^n contiguous complex amplitudes,
 *    interleaved (re, im): complex64 = 8 bytes (float2), complex128 = 16 bytes
 *    (double2).  A caller-provided buffer must be 256-byte aligned.
 *  - Every entry point returns a status (QS_OK on success).  On failure the
 *    handle is left unchanged unless stated, and qs_last_error() returns a
 *    thread-local, human-readable reason.  No entry point aborts the process.
 *  - Host input arrays are copied before the call returns; the caller keeps
 *    ownership.  Host output arrays are written only on success.
 *  - Work is ordered on the handle's CUDA stream.  qs_evolve is asynchronous;
 *    every call that returns host values synchronises that stream.
 *  - Costs are exact integers: the weights h_i, J_ij must be integer
 *    multiples of 2^-s for some s in 0..3 (half-integers arise in the exact-
 *    cover mapping, Sec. III.A.3).  Internally costs are int32 in units of
 *    2^-s; qs_cost_info reports s.  Other weights give QS_ENOTINT.
 *
 * Thread safety: distinct handles may be used from distinct host threads;
 * one handle must not be used concurrently.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_state* qs_handle;
typedef struct qs_batch* qs_batch_handle;

enum qs_status {
    QS_OK = 0,
    QS_EINVAL = 1,    /* bad argument (size, index, pointer, non-finite angle)    */
    QS_ENOMEM = 2,    /* device allocation failed or caller buffer too small      */
    QS_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error)  */
    QS_ETIMEOUT = 4,  /* a bounded device-side wait gave up (tile load, queue)    */
    QS_ENOTINT = 5,   /* weights are not integer multiples of 2^-s, s <= 3        */
    QS_ESTATE = 6     /* call out of order (e.g. evolve before set_ising)         */
};

enum qs_dtype { QS_C64 = 0, QS_C128 = 1 };
enum qs_objective { QS_OBJ_ENERGY = 0, QS_OBJ_GROUND = 1 };
enum qs_path { QS_PATH_TILED = 0, QS_PATH_PLAIN = 1 };

/* Largest qubit count per dtype on one GPU. */
#define QS_MAX_QUBITS_C64 34
#define QS_MAX_QUBITS_C128 30
/* Largest number of couplings accepted by qs_set_ising. */
#define QS_MAX_EDGES 4096

/* ------------------------------------------------------------------------ */
/* Single state                                                              */
/* ------------------------------------------------------------------------ */

/* Create a handle for an n-qubit state (Sec. II.A: 2^n amplitudes).
 *   n           1..34 (QS_C64) or 1..30 (QS_C128).
 *   dtype       QS_C64 or QS_C128.
 *   cuda_stream cudaStream_t to order all work on; NULL = the legacy default
 *               stream.  The caller keeps it alive for the handle's lifetime.
 *   device_buf  optional caller-owned device buffer for the state (for
 *               example a torch tensor), >= 2^max(n, 13) * element bytes,
 *               256-byte aligned.  NULL: the library allocates and frees it.
 *               States with n < 13 are stored with 13 - n extra idle qubits
 *               (no cost terms, left in |+>), which changes no readout.
 *   buf_bytes   size of device_buf in bytes (ignored when it is NULL).
 * Errors: QS_EINVAL (n, dtype, alignment), QS_ENOMEM (buffer too small or
 * allocation failed), QS_ECUDA. */
int qs_create(qs_handle* out, int n, int dtype, void* cuda_stream, void* device_buf, size_t buf_bytes);

/* Release the handle and everything the library allocated for it.  A
 * caller-provided buffer is not freed.  NULL is accepted. */
int qs_destroy(qs_handle h);

/* Select the kernel path: QS_PATH_TILED (default: multi-qubit HBM sweeps with
 * the phase and readout fused) or QS_PATH_PLAIN (one launch per x-rotation
 * and one per phase: the per-gate 2-component updates of
 * Eq. twocomponentupdates; the reference point for the tiled path). */
int qs_set_path(qs_handle h, int path);

/* Set the Ising cost of Eq. (HC).
 *   hfield   n doubles h_i.
 *   n_edges  0..QS_MAX_EDGES couplings.
 *   edges    2*n_edges int32 pairs (i, j), 0 <= i < j < n, no duplicates.
 *   J        n_edges doubles J_ij.
 * Validates, converts the weights to exact integers (see conventions), and
 * runs the full-enumeration ground-state search (the t_FE search of
 * Table III) on the device: minimum and maximum cost, lowest minimising index
 * and the number of minimisers, all bit-exact.  Errors: QS_EINVAL, QS_ENOTINT
 * (weights not on the 2^-s grid, or the cost range exceeds 2^24 units). */
int qs_set_ising(qs_handle h, const double* hfield, int n_edges, const int32_t* edges, const double* J);

/* Apply p layers of Eq. (QAOA_state).
 *   gamma, beta  p host doubles each (finite).
 *   from_plus    1: start from |+>^n (the ground state of H_I, Eq. HI);
 *                0: continue from the current state.
 * The readout (<H_C>, ground probability, norm) of the final state is fused
 * into the last sweep and cached for qs_expect / qs_ground_prob.  p = 0 with
 * from_plus = 1 prepares |+>^n.  Asynchronous.  Errors: QS_EINVAL,
 * QS_ESTATE (no Ising cost set), QS_ECUDA. */
int qs_evolve(qs_handle h, int p, const double* gamma, const double* beta, int from_plus);

/* Per-layer spin expectations (the magnetisations <sigma^z_i> followed
 * during an annealing run, Sec. III.B.2, Fig. 6): apply p layers of
 * Eq. (QAOA_state) from |+>^n, as qs_evolve with from_plus = 1, and record
 * after every layer k the n values
 *   zexp[k * n + i] = <Z_i> = sum_z |psi_z|^2 (1 - 2 bit_i(z)),  k = 0..p-1,
 * (p * n host doubles, caller-owned).  Each record is accumulated in FP64
 * inside the sweep that applies the next layer's phase (for the last layer,
 * the readout sweep), so the evolve moves no extra state bytes.  The final
 * state and its readout are left as after qs_evolve.  Tiled path only (not
 * QS_PATH_PLAIN).  Synchronises.  Errors: QS_EINVAL, QS_ESTATE, QS_ECUDA,
 * QS_ETIMEOUT. */
int qs_evolve_zexp(qs_handle h, int p, const double* gamma, const double* beta, double* zexp);

/* Layers with general single-spin unitaries in place of the transverse-field
 * mixer (the combined x + z single-spin exponentials of the product formula
 * Eq. (AQA4)): from |+>^n, for k = 0..p-1,
 *   psi <- (prod_i U_{k,i}) exp(-i gamma_k H_C) psi,
 * with H_C the handle's Ising cost (Eq. HC).
 *   gamma  p host doubles;
 *   u      p * n * 8 host doubles: U_{k,i} = [[u00, u01], [u10, u11]] row
 *          major, each entry (re, im), acting on (|0>, |1>) of qubit i.
 * The matrices need not be unitary for the arithmetic, but the readout's
 * meaning assumes they are.  The readout of the final state is cached as
 * after qs_evolve.  Tiled path only; complex64 and complex128; no adjoint.
 * Asynchronous.  Errors: QS_EINVAL, QS_ESTATE, QS_ECUDA. */
int qs_evolve_su2(qs_handle h, int p, const double* gamma, const double* u);

/* The layers of qs_evolve_su2 that reproduce nsteps steps of Eq. (AQA4)
 * with the fields of Eq. (AQA3) (h~^x = A_l, h~^z_i = -B_l h_i, J~^z_ij =
 * -B_l J_ij; A, B nsteps doubles, hfield n doubles): consecutive half steps
 * S_{l+1}(tau/2) S_l(tau/2) are merged into one matrix per qubit, and since
 * the engine's phase exp(-i gamma H_C) includes the fields, their part
 * exp(-i tau B_l h_i Z_i) is undone in the following matrices.  Writes
 * nsteps + 1 layers: gamma (nsteps + 1 doubles) and u ((nsteps + 1) n 8
 * doubles).  Host only.  Errors: QS_EINVAL. */
int qs_qsds_layers(int n, int nsteps, double tau, const double* A, const double* B, const double* hfield,
                   double* gamma, double* u);

/* <H_C> of the current state, accumulated in FP64.  Synchronises. */
int qs_expect(qs_handle h, double* E);

/* Ground-state probability of the current state: total weight on every basis
 * state of minimal cost (all minimisers, ties included).  Also returns the
 * lowest minimising index, the minimal cost in units of 2^-s and the number
 * of minimisers (any output pointer may be NULL).  Synchronises. */
int qs_ground_prob(qs_handle h, double* P, int64_t* argmin, int64_t* cmin, int64_t* ground_count);

/* E, P and sum |psi|^2 of the current state in one call.  Synchronises. */
int qs_readout(qs_handle h, double* E, double* P, double* norm);

/* Exact cost range and ground-state data of the Ising cost in units of 2^-s.
 * Any output pointer may be NULL.  Synchronises. */
int qs_cost_info(qs_handle h, int64_t* cmin, int64_t* cmax, int64_t* argmin, int64_t* ground_count,
                 int* scale_shift);

/* Allocation-free variant of the ground-state enumeration behind
 * qs_set_ising / qs_cost_info.  The paper has no counterpart: it serves
 * callers that cannot allocate device memory.
 *   n, hfield, n_edges, edges, J   as for qs_set_ising (same validation);
 *                                  n at most QS_NOALLOC_MAX_QUBITS.
 *   cuda_stream  cudaStream_t to run on; NULL = the legacy default stream.
 *   outputs      as for qs_cost_info (any may be NULL); written on success.
 * It calls no cudaMalloc, cudaFree or other allocating routine and needs no
 * handle: its scratch (cost program, per-block partials, result words) is a
 * file-scope device array of QS_NOALLOC_SCRATCH_BYTES bytes, whose address
 * is looked up once per device (with that device current) on the first call
 * there; make that first call before any stream capture begins.  Every call
 * in the process shares that array, so calls that overlap on the GPU (from
 * several host threads or streams) race.  Nothing in it has to start at
 * zero: a call writes each word before reading it.  Inputs beyond the limits
 * (or a cost program longer than the scratch holds) give QS_EINVAL with the
 * reason.  Synchronises the stream.  Errors: QS_EINVAL, QS_ENOTINT,
 * QS_ECUDA. */
#define QS_NOALLOC_MAX_QUBITS 40
#define QS_NOALLOC_SCRATCH_BYTES 99584
int qs_enumerate_noalloc(int n, const double* hfield, int n_edges, const int32_t* edges, const double* J,
                         void* cuda_stream, int64_t* cmin, int64_t* cmax, int64_t* argmin, int64_t* ground_count,
                         int* scale_shift);

/* Tile-shape plan of the handle (the sweeps' "tile width and block shape";
 * the paper's gate-by-gate engine has no counterpart).
 *   runs_a  1: shape A is runs of 2^8 amplitudes plus the top four qubits
 *           (complex64, n >= 24); 0: shape A is 2^13 contiguous amplitudes;
 *           -1: the default rule (runs from 33 qubits).
 *   split   index bit from which the strided shapes' qubits are dealt out
 *           evenly; -1: the default (22 with runs, else the 2 MB page bit).
 * Re-plans the current Ising cost (same results up to rounding order).
 * Errors: QS_EINVAL. */
int qs_set_shape_rule(qs_handle h, int runs_a, int split);

/* Plan rule of the handle: QS_PLAN_RULE_INTS ints
 *   [0] runs_a, [1] split   as qs_set_shape_rule;
 *   [2] cmin         carried low bits of the strided shapes: 2 (rows of 32
 *                    bytes, 11 targets per shape) or 3 (64-byte rows, 10
 *                    targets; more shapes); -1 the default (2);
 *   [3] ctas_per_sm  persistent CTAs per SM of the sweep kernels (0: as many
 *                    as fit);
 *   [4] pair_cluster 4: the strided packed-pair sweeps run in 4-CTA
 *                    clusters that fetch shared HBM lines once; 1: without;
 *   [5] pair_tma     1: the strided packed-pair forward sweeps load each
 *                    tile with two tensor-map copies (TMA) issued by one
 *                    thread; 0: with per-thread 16-byte cp.async copies
 *                    (the tensor-map copies fall back to these where a
 *                    shape does not fit a five-dimensional box);
 *   [6] pair_l2      L2 promotion of the tensor-map tile copies: 0 none,
 *                    1 128 bytes, 2 256 bytes;
 *   [7] order        1: the strided shapes in reverse order, so that the
 *                    zig-zag schedule merges the sweeps of another shape
 *                    around the phases (0: the planned order).
 * Every rule gives the same results up to rounding order (the load fields
 * give bit-identical states).  qs_set_plan_rule re-plans the current Ising
 * cost when the shape fields change.  Errors: QS_EINVAL. */
#define QS_PLAN_RULE_INTS 8
int qs_set_plan_rule(qs_handle h, const int* rule);
int qs_get_plan_rule(qs_handle h, int* rule);

/* Autotuner: times p_trial layers (from |+>, fixed angles; one warm-up, the
 * faster of two runs) under candidate plan rules on this GPU and keeps the
 * fastest.  Search, coordinate by coordinate: tile shapes first (contiguous
 * shape A; for complex64 states of 24 qubits and more the run-structured A
 * with split bits 20, 22 and 24; each with cmin 2 and 3), then, for the best
 * shapes, the strided shapes in reverse order, one CTA per SM fewer than
 * fit and (complex64) the strided sweeps without clusters, then
 * (complex64) tensor-map tile copies with no or 256-byte L2 promotion.
 * Reports the measured candidates (up to max_cand rules of
 * QS_PLAN_RULE_INTS ints in cand_rules with their times in cand_ms, the
 * count in ncand) and the kept rule (best_rule, QS_PLAN_RULE_INTS ints) with
 * its time; any output may be NULL when max_cand = 0.  Overwrites the
 * state.  Call after qs_set_ising.  Errors: QS_ESTATE, QS_EINVAL, QS_ECUDA. */
int qs_autotune_ex(qs_handle h, int p_trial, int max_cand, int* ncand, int* cand_rules, double* cand_ms,
                   int* best_rule, double* best_ms);

/* qs_autotune_ex reporting only runs_a, split and the time. */
int qs_autotune(qs_handle h, int p_trial, int* runs_a, int* split, double* best_ms);

/* Gradient of F = <psi_p|O|psi_p> with respect to all 2p angles, where O is
 * H_C (QS_OBJ_ENERGY) or the projector on the minimal-cost states
 * (QS_OBJ_GROUND).  Not in the paper: reverse-mode through the unitary layers,
 * which un-computes psi with the inverse layers (no checkpoints) while it
 * propagates lambda = O psi_p and accumulates, per layer,
 *   dF/dbeta_k  = 2 Im <lambda_k| H_D |psi_k>,
 *   dF/dgamma_k = 2 Im <mu_k| H_C |phi_k>  (mu, phi: after undoing mixer k).
 * Runs from |+>^n.  The reverse sweeps overwrite the state buffer (it ends
 * near |+>^n), so call qs_evolve again to read psi_p.  Needs a second
 * state-sized device buffer: set one with qs_set_adjoint_buffer, or the
 * library allocates it on first use.  value, dgamma, dbeta: host outputs
 * (value may be NULL).  Synchronises. */
int qs_grad(qs_handle h, int p, const double* gamma, const double* beta, int objective,
            double* value, double* dgamma, double* dbeta);

/* Provide the adjoint state buffer used by qs_grad (caller-owned, same size
 * and alignment rules as the state buffer).  NULL releases a library-owned
 * one. */
int qs_set_adjoint_buffer(qs_handle h, void* device_buf, size_t buf_bytes);

/* Copy the state to host memory in the canonical basis order (bytes must be
 * 2^n * element size).  For tests and small n.  Synchronises. */
int qs_copy_state(qs_handle h, void* dst_host, size_t bytes);

/* Device pointer of the state buffer.  The amplitudes stored there are
 * psi_{z XOR F} where F is 0 or 2^n - 1 (*flip_all = 1); qs_canonicalize
 * makes F = 0 in place.  Either output may be NULL. */
int qs_state_ptr(qs_handle h, void** device_ptr, int* flip_all);

/* Bring the stored amplitudes into the canonical basis order in place (one
 * sweep when the stored frame is flipped, nothing otherwise).  Asynchronous. */
int qs_canonicalize(qs_handle h);

/* Sweeps per layer of the current plan (tiled path): the number of
 * distinct tile shapes S and the HBM sweeps that p layers take. */
int qs_plan_info(qs_handle h, int p, int* tile_shapes, int* sweeps);

/* The same without a handle (host only, no GPU needed): an n-qubit state of
 * the given dtype evolved from |+>^n through p layers. */
int qs_plan_sweeps(int n, int dtype, int p, int* tile_shapes, int* sweeps);

/* Tile shape k of the plan for an n-qubit state (host only): shape kind
 * (0 contiguous, 1 strided), tile bits K, carried low bits c, and the two
 * target runs [g0, g0 + n1) and [g1, g1 + K - c - n1).  Returns QS_EINVAL
 * when k is past the last shape. */
int qs_plan_shape(int n, int dtype, int k, int* kind, int* K, int* c, int* g0, int* n1, int* g1);

/* Tensor-map view of the tiles of a strided complex64 shape (K = 13 tile
 * bits, c = 2 or 3 carried bits, target runs [g0, g0 + n1) and [g1, g1 +
 * 13 - c - n1) of an n-qubit state) loaded for a first read into register
 * layout g (0 or 1) of the packed-pair forward sweep (host only; the
 * plan rule's pair_tma).  Outputs: rank (at most 5) dimensions, dimension d
 * covering global index bits [start[d], start[d] + width[d]) of which the
 * box holds the lowest box[d] (dimension 0 starts at bit 0), in the box's
 * shared-memory order; kbit is the global bit of the pack bit, one box
 * copy per value; landing[tb] (13 ints) is the shared-memory position bit
 * of tile bit tb.  Every array has room for 5 (landing: 13) ints.
 * Returns QS_EINVAL for a shape that does not fit such a box. */
int qs_pair_tile_map(int n, int c, int g0, int n1, int g1, int g, int* rank, int* kbit, int* start, int* width,
                     int* box, int* landing);

/* Number of kernels this library has launched in this process so far (all
 * handles and batches).  For accounting in benchmarks. */
int qs_launch_count(int64_t* count);

/* ------------------------------------------------------------------------ */
/* Host-only helpers (no GPU needed)                                         */
/* ------------------------------------------------------------------------ */

/* First-order AQA angles on the linear schedule A(s) = 1 - s, B(s) = s:
 *   gamma_k = tau * s_k,  beta_k = -tau * (1 - s_k).
 * One first-order Trotter step of H(s) = A(s) H_I + B(s) H_C (Eqs. HI, Hofs)
 * per knot; H_I = -H_D makes the driver factor e^{+i tau A H_D}, hence the
 * negative beta (the sign of Eqs. beta_k - gamma_k).  s: p knots in [0, 1]. */
int qs_aqa_angles(int p, double tau, const double* s, double* gamma, double* beta);

/* The paper's second-order map, Eqs. (beta_k)-(gamma_k) with A = 1 - s,
 * B = s:  beta_k = -tau (A(s_{k+1}) + A(s_k)) / 2 (k < p),
 * beta_p = -tau A(s_p) / 2, gamma_k = tau B(s_k). */
int qs_aqa_angles_2nd(int p, double tau, const double* s, double* gamma, double* beta);

/* Chain rule for qs_aqa_angles: from dF/dgamma_k, dF/dbeta_k to
 *   dF/dtau = sum_k [s_k dF/dgamma_k - (1 - s_k) dF/dbeta_k],
 *   dF/ds_k = tau (dF/dgamma_k + dF/dbeta_k). */
int qs_aqa_chain(int p, double tau, const double* s, const double* dgamma, const double* dbeta,
                 double* dtau, double* ds);

/* Chain rule for qs_aqa_angles_2nd (Eqs. beta_k-gamma_k, Appendix A): from
 * dF/dgamma_k, dF/dbeta_k to dF/dtau and dF/ds_k.  With A(s) = 1 - s,
 *   dF/dtau = sum_k s_k dF/dgamma_k + sum_k (beta_k / tau) dF/dbeta_k,
 *   dF/ds_k = tau dF/dgamma_k + tau/2 dF/dbeta_k + tau/2 dF/dbeta_{k-1} (k > 1),
 * since beta_k holds A(s_k) and A(s_{k+1}) with weight tau/2 each (beta_p
 * only A(s_p)).  p >= 1 knots; ds receives p values.  Errors: QS_EINVAL. */
int qs_aqa_chain_2nd(int p, double tau, const double* s, const double* dgamma, const double* dbeta,
                     double* dtau, double* ds);

/* Thread-local text for the last non-OK status on this thread. */
const char* qs_last_error(void);

/* Library version string. */
const char* qs_version(void);

/* ------------------------------------------------------------------------ */
/* Batched instances                                                         */
/* ------------------------------------------------------------------------ */

/* A batch of `count` independent instances of possibly different n
 * (1..QS_MAX_QUBITS_C64, complex64 only), all on one stream.  The forward of
 * the whole batch is one launch of a persistent work-queue kernel over every
 * tile of every sweep of every instance (ordered sweep by sweep, with a tile
 * counter per instance ordering its own sweeps); the adjoint's reverse
 * sweeps are a second launch.  Small states share the GPU with large ones.
 * One queue holds at most 2^26 tiles of 2^13 amplitudes (evolve and grad
 * return QS_EINVAL beyond).  The library allocates every state.  Errors:
 * QS_EINVAL, QS_ENOMEM. */
int qs_batch_create(qs_batch_handle* out, int count, const int* n, int dtype, void* cuda_stream);

/* Ising cost of instance idx (same rules as qs_set_ising). */
int qs_batch_set_ising(qs_batch_handle b, int idx, const double* hfield, int n_edges,
                       const int32_t* edges, const double* J);

/* Evolve every instance from |+> with its own p and angles.
 *   p          count ints (0..QS_MAX_LAYERS_BATCH).
 *   angle_off  count offsets into gamma/beta where instance i's p angles start.
 *   gamma,beta host doubles.  Asynchronous. */
int qs_batch_evolve(qs_batch_handle b, const int* p, const int64_t* angle_off, const double* gamma,
                    const double* beta);

/* E and P_ground per instance after qs_batch_evolve or qs_batch_grad
 * (either pointer may be NULL).  Synchronises. */
int qs_batch_results(qs_batch_handle b, double* E, double* P);

/* Gradients of every instance at its current angles (the last evolve's).
 * value (count), dgamma, dbeta (laid out like the angles).  Synchronises. */
int qs_batch_grad(qs_batch_handle b, int objective, double* value, double* dgamma, double* dbeta);

/* `steps` Adam steps minimising each instance's objective (QS_OBJ_ENERGY)
 * over its 2p angles, entirely on the device: each step is a batched
 * forward + adjoint and an Adam update (bias-corrected; lr, b1, b2, eps).
 * gamma_io, beta_io hold the initial angles (laid out as in
 * qs_batch_evolve's last call) and receive the final ones.  use_graph = 1
 * captures one step in a CUDA graph and replays it.  Afterwards
 * qs_batch_results gives E and P_ground at the final angles.  Synchronises. */
int qs_batch_adam(qs_batch_handle b, int steps, double lr, double b1, double b2, double eps,
                  double* gamma_io, double* beta_io, int use_graph);

/* Launch rule of the batch's work queue: ctas_per_sm persistent CTAs per SM
 * (0: as many as fit); window_bytes > 0 orders the queue in windows of
 * consecutive instances holding at most that many state bytes (wave by wave
 * inside a window, so its states can stay in L2 between sweeps); 0: one
 * window of every instance.  Same results up to rounding order.  Errors:
 * QS_EINVAL. */
int qs_batch_set_launch_rule(qs_batch_handle b, int ctas_per_sm, int64_t window_bytes);

/* Batch autotuner: times the batch's forward at the angles of the last
 * qs_batch_evolve (one warm-up, the faster of two runs) for ctas_per_sm in
 * {as many as fit, one fewer} and window_bytes in {one window, 256 MiB,
 * 64 MiB}, keeps the fastest and reports it (any pointer may be NULL).
 * Overwrites the states; qs_batch_results needs a new evolve.  Errors:
 * QS_ESTATE, QS_ECUDA, QS_ETIMEOUT. */
int qs_batch_autotune(qs_batch_handle b, int* ctas_per_sm, int64_t* window_bytes, double* best_ms);

/* Failure-detection test hook (no counterpart in the paper).  Arms the next
 * qs_batch_evolve to run a work queue in which the second sweep of instance
 * idx waits for one tile more than its first sweep provides, with a
 * dependency wait limit of wait_limit_s seconds (0 < limit <= 10): the wait
 * runs out, the kernel sets its error word and every CTA returns, and the
 * next call that synchronises (qs_batch_results) returns QS_ETIMEOUT with the
 * results invalid.  No copy is left in flight, so the batch stays usable:
 * the next qs_batch_evolve runs the normal plan.  One-shot.  Errors:
 * QS_EINVAL. */
int qs_batch_test_withhold(qs_batch_handle b, int idx, double wait_limit_s);

int qs_batch_destroy(qs_batch_handle b);

/* Partition of a batch over `world` ranks (one GPU each), host only.
 * Instances are independent (no data-path exchange), so the only choice is
 * which rank evolves which: greedy longest-first bin-packing on the work of
 * an instance, max(p_i, 1) 2^{n_i} amplitude-layers (its HBM traffic is
 * proportional to it).  Instances are taken in order of decreasing work
 * (ties: lower index first), each to the rank with the least work so far
 * (ties: lower rank).  Deterministic, so every rank computes the same
 * partition from the same inputs.
 *   count   instances; n, p: count ints each (n in 1..QS_MAX_QUBITS_C64,
 *           p >= 0).
 *   world   ranks, >= 1.
 *   rank_of count ints: the rank of each instance.
 *   load    world doubles (may be NULL): the work given to each rank.
 * Errors: QS_EINVAL. */
int qs_batch_partition(int count, const int* n, const int* p, int world, int* rank_of, double* load);

#define QS_MAX_LAYERS_BATCH 64

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
