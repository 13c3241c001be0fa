/*
 * qs.h -- C ABI of the GB300 state-vector gate engine (libqs.so).
 *
 * What it computes: the data-parallel core of qHiPSTER (Smelyanskiy, Sawaya,
 * Aspuru-Guzik, arXiv:1601.07195): a general single-qubit 2x2 unitary Q on
 * qubit k (Eq. 2) and a controlled-Q gate with control c and target t (Eq. 3),
 * applied in place to a dense state of 2^n complex amplitudes.  Amplitude i
 * holds basis state |i>, qubit k is bit k of i, so the two amplitudes a gate on
 * qubit k mixes are 2^k apart (Section 2).  Runs of gates are fused into one
 * pass over device memory (the gate fusion / cache blocking of Section 4.4,
 * Fig. 5, with a shared-memory tile in place of the last-level cache).
 *
 * Not in the paper, built beside it: complex64 states, FP64 reductions
 * (norm, marginals, probabilities, Pauli-sum expectations), adjoint gradients
 * of rotation angles, batched execution of many small circuits, dense blocks of
 * gates on qubits 0..5 applied as one matrix on the tensor cores (complex64),
 * and page-locked host buffers for state transfers.
 *
 * Conventions for every entry point:
 *   - Pointers are plain host or device pointers; sizes are element counts.
 *     Nothing here takes or returns a framework (PyTorch) object.
 *   - A qs_state is bound to one CUDA device and one stream.  Apply calls are
 *     asynchronous on that stream; calls that return host values (qs_norm,
 *     qs_prob, qs_probs, qs_expect, qs_copy_out, qs_grad) synchronise it.
 *   - Invalid arguments return QS_EINVAL before anything is launched; CUDA
 *     failures return QS_ECUDA; a device-side wait that ran out of time
 *     returns QS_ETIMEOUT.  No call aborts the process.  The message of the
 *     last failure on the calling thread is returned by qs_last_error().
 *   - Matrices are 8 doubles: row-major (q11, q12, q21, q22) as (re, im)
 *     pairs; row = output amplitude, column = input amplitude (Eq. 2).
 *     complex64 states round them to float once on the host.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QS_API __attribute__((visibility("default")))
#else
#define QS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

typedef enum {
    QS_OK = 0,
    QS_EINVAL = 1,    /* bad argument, detected before any launch */
    QS_ENOMEM = 2,    /* device or pinned-host allocation failed */
    QS_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    QS_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    QS_EDTYPE = 5     /* operation not available for this state's dtype */
} qs_status;

/* Gate record kinds.  QS_G_U1: Q on t (Eq. 2).  QS_G_CU: controlled-Q,
 * control c, target t (Eq. 3).  QS_G_SWAP: exchange qubits t and c.
 * QS_G_RX/RY/RZ: exp(-i theta G / 2) on t, G = X/Y/Z, theta = theta[param]. */
enum { QS_G_U1 = 0, QS_G_CU = 1, QS_G_SWAP = 2, QS_G_RX = 3, QS_G_RY = 4, QS_G_RZ = 5 };

/* 80-byte gate record; m is ignored for QS_G_SWAP and the rotation kinds. */
typedef struct {
    int32_t kind;
    int32_t t;      /* target qubit (first qubit of a swap) */
    int32_t c;      /* control qubit (second qubit of a swap); -1 if none */
    int32_t param;  /* angle index for rotations; -1 otherwise */
    double m[8];
} qs_gate;

/* Pauli-sum term: coef * Z_q0, coef * Z_q0 Z_q1, or coef * X_q0. */
enum { QS_P_Z = 0, QS_P_ZZ = 1, QS_P_X = 2 };
typedef struct {
    int32_t kind;
    int32_t q0;
    int32_t q1;     /* second qubit of QS_P_ZZ; -1 otherwise */
    int32_t pad;
    double coef;
} qs_term;

typedef struct qs_state qs_state;
typedef struct qs_plan qs_plan;

/* ---- state lifetime ------------------------------------------------------ */

/* Allocate a device state of 2^n amplitudes (1 <= n <= 36, limited by free
 * device memory) on the current device, bound to `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream), initialised to |0..0>.
 * The state owns its memory; qs_destroy frees it. */
QS_API qs_status qs_create(int n, qs_dtype dt, void* cuda_stream, qs_state** out);

/* Wrap caller-owned device memory of 2^n amplitudes (interleaved re, im;
 * 16-byte aligned for complex128, 8-byte for complex64) without copying.
 * The state belongs to the current device: where the CUDA runtime can
 * classify dev_ptr, it must be device memory of that device (or managed
 * memory), else QS_EINVAL.  The caller keeps the memory alive until after
 * qs_destroy, and does not read or write it from other streams while this
 * library's work on the state's stream is in flight (a plan's passes may hold
 * it in an intermediate form, see qs_plan_execute). */
QS_API qs_status qs_wrap(void* dev_ptr, int n, qs_dtype dt, void* cuda_stream, qs_state** out);

/* Release the handle (and the memory, for qs_create).  NULL is accepted. */
QS_API qs_status qs_destroy(qs_state* s);

/* Rebind the state to another stream of the same device. */
QS_API qs_status qs_set_stream(qs_state* s, void* cuda_stream);

/* Arithmetic of the single-gate calls (qs_apply_*) on a complex128 state:
 * native_f64 = 0 (default) evaluates the 2x2 update in double-float form on
 * the FP32 pipes, 1 uses native FP64 instructions (see QS_PLAN_ARITH_F64). */
QS_API qs_status qs_set_arith(qs_state* s, int native_f64);

/* Kernel form of the single-gate calls whose target t is 0..4 (the partner
 * amplitude 2^t away lies in the same 32-amplitude group; Section 4.1's SIMD
 * analogue).  The lane-exchange kernel has each warp read 32 consecutive
 * amplitudes and exchange partners between lanes with warp shuffles; it
 * covers non-diagonal single-qubit gates and controlled gates whose control
 * is 5 or above.  The pair kernel is the one every other target uses.  Both
 * compute Eq. 2 / Eq. 3 and agree to rounding (bit-exact for X).
 *   QS_LANES_AUTO (default): the measured choice, lane exchange for native
 *     FP64 and for complex64 single-qubit gates, the pair kernel for
 *     double-float complex128 and complex64 controlled gates;
 *   QS_LANES_OFF: the pair kernel;  QS_LANES_ON: the lane exchange.
 * Any other mode, or a NULL state: QS_EINVAL. */
typedef enum { QS_LANES_OFF = 0, QS_LANES_AUTO = 1, QS_LANES_ON = 2 } qs_lane_mode;
QS_API qs_status qs_set_lanes(qs_state* s, int mode);

/* Device address, qubit count and dtype of a state. */
QS_API qs_status qs_info(const qs_state* s, void** dev_ptr, int* n, qs_dtype* dt);

/* Set the state to the basis state |x> (x < 2^n). */
QS_API qs_status qs_init_basis(qs_state* s, uint64_t x);

/* Host <-> device copies of amplitudes [off, off + cnt), in the state's dtype. */
QS_API qs_status qs_copy_out(qs_state* s, uint64_t off, uint64_t cnt, void* host);
QS_API qs_status qs_copy_in(qs_state* s, uint64_t off, uint64_t cnt, const void* host);

/* Page-locked host memory for qs_copy_in / qs_copy_out, at least `bytes`
 * long, zeroed: an anonymous mapping aligned to the transparent huge page size
 * and advised (and, where the fault path found none free, collapsed) into huge
 * pages, then registered with the CUDA runtime.  On the GB300 nodes measured
 * (64 KiB base pages, 512 MiB huge pages), copies of a 17 GB state from a
 * fully huge-page-backed buffer ran at about 210 GB/s every time, while
 * cudaHostAlloc memory slowed to 330-690 ms per copy when each copy followed
 * 0.75 s of kernels on a host whose memory earlier jobs had fragmented.
 * Huge pages are best effort: on fragmented memory part of the buffer may stay
 * on base pages, and copies from that part are slower.
 * Free it with qs_host_free.  QS_ENOMEM or QS_ECUDA if it cannot be had. */
QS_API qs_status qs_host_alloc(size_t bytes, void** out);

/* Release memory from qs_host_alloc (NULL is accepted; any other pointer is
 * QS_EINVAL). */
QS_API qs_status qs_host_free(void* p);

/* ---- single gates (Eq. 2, Eq. 3) ----------------------------------------- */

/* Q on qubit k, 0 <= k < n. */
QS_API qs_status qs_apply_1q(qs_state* s, int k, const double U[8]);

/* Controlled-Q: Q on target t where control bit c is 1; c != t. */
QS_API qs_status qs_apply_ctrl(qs_state* s, int c, int t, const double U[8]);

/* SWAP of qubits a != b (an index permutation; moves amplitudes bit-exactly). */
QS_API qs_status qs_apply_swap(qs_state* s, int a, int b);

/* ---- circuits --------------------------------------------------------------- */

/* Plan flags. */
enum {
    QS_PLAN_DEFAULT = 0,
    QS_PLAN_NO_FUSION = 1,  /* one pass over the state per gate (no tiles) */
    QS_PLAN_GRAPH = 2,      /* capture the launches once and replay a CUDA graph */
    QS_PLAN_ARITH_F64 = 4,  /* complex128: native FP64 instructions for the gate arithmetic.
                               Without it, fused tile passes of complex128 states compute in
                               double-float form on the FP32 pipes (each double carried as an
                               unevaluated float pair of about 48 bits; the state is IEEE
                               double whenever no plan is running, see qs_plan_execute): faster on GPUs whose FP64 rate is a small fraction of
                               FP32, with a per-gate error of order 2^-44 relative to the
                               amplitudes involved instead of 2^-53. */
    QS_PLAN_DRY_RUN = 8,    /* plan on the host only (no device memory); cannot execute */
    QS_PLAN_NO_MERGE = 16,  /* keep every gate separate: no product of adjacent single-qubit
                               gates on the same qubit inside a tile pass */
    QS_PLAN_NO_PHASE_RUNS = 32, /* apply runs of phase gates one by one.  Without it, a run of
                               consecutive gates inside a tile pass that are diagonal with
                               q11 = 1 (T, S, phase, CZ, controlled phase) and all involve one
                               tile qubit j (the controlled-phase chains of the QFT, Section 5)
                               is applied as one update: per tile, a table of phase products
                               over the low and the high half of the tile bits, and two complex
                               products per amplitude whose bit j is 1. */
    QS_PLAN_NO_PRP = 64,    /* complex128 double-float plans: apply every general single-qubit
                               unitary with its full complex 2x2 product.  Without it, inside a
                               tile pass, such a unitary U is applied as
                               U = K diag(1, z) [[1, t], [-t, 1]] diag(1, y)  (|t| <= 1; when
                               |q12| > |q11|, the same form times X): two complex products on
                               the |1> amplitude and one real shear, about 70% of the
                               arithmetic.  The complex scalars K of a pass are multiplied
                               into one other single-qubit update of the pass (a diagonal,
                               anti-diagonal or general one, whose cost does not change), so
                               the pass applies the same product.  Taken only where the form
                               reproduces U to 4e-15 in every entry (unitary U).  Likewise a
                               real single-qubit gate whose four entries share one magnitude
                               (H, HX, XH, ZH, ...), q11 [[1, s1], [r, r s3]] with signs s1,
                               r, s3, is applied as the bracket (two exact sums and no product
                               per component) with q11 left out.  The scalars left out of one
                               pass multiply to at least 2^-24. */
    QS_PLAN_NO_DIAG_RUNS = 256, /* apply runs of phase gates that no phase run covers one by
                               one.  Without it, a run of at least four consecutive gates
                               inside a tile pass that are diagonal with q11 = 1 and whose
                               combined phase separates over the low and the high half of the
                               tile bits (phases on one qubit; controlled phases between a tile
                               qubit and a qubit outside the tile, between two outside qubits,
                               or between two tile qubits of the same half) is applied as one
                               update: per tile, the factor of each tile bit under the tile's
                               outside bits, tables over the two halves, and two complex
                               products per amplitude.  Such runs are the inverse QFT's
                               controlled phases whose target lies outside the tile. */
    QS_PLAN_NO_DENSE = 128  /* complex64 plans: no dense tensor-core passes.  Without it, a run of
                               at least 10 consecutive gates whose qubits all lie in 0..5 is
                               multiplied into one 64 x 64 matrix on the host (FP64) and applied
                               as one pass on the tensor cores (see qs_apply_dense); the rest of
                               the circuit is planned as usual around it.  qs_plan_pass reports
                               such a pass with kind 2 and qs_plan_pass_dense returns its matrix;
                               qs_plan_destroy returns QS_ETIMEOUT if a bounded wait inside one of
                               these passes gave up.  complex128 plans have no dense passes. */
};

/* Build an execution plan for `gates` (copied in) on state s: gate classes,
 * fused tile passes of gates whose mixing qubits fit one tile (Section 4.4,
 * Fig. 5), single-gate passes for the rest.  theta (n_params angles) is read
 * for the rotation kinds; it is copied in too.
 * tile_bits: bits 0-7 = log2 amplitudes per tile, bits 8-15 = how many of the
 * lowest qubits every tile contains (contiguous runs of 2^run amplitudes in
 * device memory); 0 in either field = the tuned value for (dtype, n), see
 * qs_tune_set / qs_autotune, else the built-in default. */
QS_API qs_status qs_plan_create(qs_state* s, const qs_gate* gates, int n_gates, const double* theta, int n_params,
                         int flags, int tile_bits, qs_plan** out);

/* Launch the plan on the state's stream (asynchronous).  For complex128 in
 * double-float arithmetic, consecutive tile passes hand the state to each
 * other as float pairs (hi, lo), the same 16 bytes per amplitude, so while the
 * plan runs the state's memory may hold that form; it holds IEEE complex128
 * again when the plan's last pass has completed.  Work on other streams must
 * not read the state in between. */
QS_API qs_status qs_plan_execute(qs_plan* p);

/* Plan statistics: number of passes over the state, of which tile passes,
 * and the kernel launches one execution makes. */
QS_API qs_status qs_plan_stats(const qs_plan* p, int* n_passes, int* n_tile_passes, int* n_launches);

/* Gate updates one execution applies after fusing adjacent single-qubit gates
 * on the same qubit within a tile pass (into their product, where that is
 * cheaper to apply; exact identities are dropped) and runs of phase gates
 * (one update per run, see QS_PLAN_NO_PHASE_RUNS and QS_PLAN_NO_DIAG_RUNS). */
QS_API qs_status qs_plan_device_ops(const qs_plan* p, int* n_ops);

/* Gate updates of pass i as the kernels apply them (after fusion): counts[3][6]
 * by operation (0 = single-qubit, 1 = controlled, 2 = swap) and class
 * (0 general, 1 real, 2 diagonal, 3 diagonal with q11 = 1, 4 anti-diagonal,
 * 5 permutation).  A fused run of phase gates around one qubit counts as one
 * single-qubit diagonal update (two complex products on half the amplitudes,
 * the same arithmetic); a diagonal run (QS_PLAN_NO_DIAG_RUNS) counts as two
 * (two complex products on every amplitude). */
QS_API qs_status qs_plan_pass_op_counts(const qs_plan* p, int i, int* counts);

/* Of pass i's real gate updates (class 1 above), how many the complex128
 * double-float kernel applies in balanced form: counts[0] single-qubit,
 * counts[1] controlled.  A real gate whose four entries share one magnitude
 * (H and its products with X and Z) updates a pair as q11 (a + s1 b) and
 * q21 (a + s3 b): an exact sum and one product per component.  Zero for
 * other plans. */
QS_API qs_status qs_plan_pass_balanced(const qs_plan* p, int i, int* counts);

/* Single-qubit updates of pass i that the complex128 double-float kernel
 * applies with a scalar left out (QS_PLAN_NO_PRP): counts[0] general ones
 * (class 0 above) in phase-shear-phase form, counts[1] real ones (class 1,
 * not counted by qs_plan_pass_balanced) as a signed sum without q11,
 * counts[2] of counts[0] those whose trailing phase diag(1, z) a later update
 * of the pass on the same qubit took into its matrix (a general, diagonal or
 * anti-diagonal single-qubit update, with only updates that commute with the
 * phase in between), so they skip that product.  Zero for other plans. */
QS_API qs_status qs_plan_pass_prp(const qs_plan* p, int i, int* counts);

/* Per-pass description: for pass i, its kind (0 = single gate, 1 = tile,
 * 2 = dense block on qubits 0..5, see QS_PLAN_NO_DENSE),
 * first gate and gate count in plan order, and the tile's qubit mask. */
QS_API qs_status qs_plan_pass(const qs_plan* p, int i, int* kind, int* n_gates, uint64_t* tile_mask);

/* Circuit positions of pass i's gates in execution order (n_gates ints, see
 * qs_plan_pass).  Within and across passes the planner only moves a gate ahead
 * of gates it commutes with (disjoint qubits, or both diagonal). */
QS_API qs_status qs_plan_pass_gates(const qs_plan* p, int i, int* positions);

/* The 64 x 64 matrix of dense pass i (kind 2): row-major, (re, im) doubles,
 * 8192 doubles into U; the ordered product of the pass's gates on qubits 0..5,
 * formed on the host in FP64.  QS_EINVAL for other passes. */
QS_API qs_status qs_plan_pass_dense(const qs_plan* p, int i, double* U);

/* Per-pass timing with CUDA events recorded on the state's stream around
 * every pass: keep `records` sets of events, used round robin by successive
 * eager executions (0 disables; not for CUDA-graph or dry-run plans). */
QS_API qs_status qs_plan_set_timing(qs_plan* p, int records);

/* Milliseconds of each pass (n_passes floats) of timing record `record`;
 * waits for that record's last event. */
QS_API qs_status qs_plan_pass_times(qs_plan* p, int record, float* ms);

/* Free the plan; waits for the plan's launches on the state's stream first.
 * QS_ETIMEOUT if a bounded wait inside a dense pass gave up (QS_PLAN_NO_DENSE). */
QS_API qs_status qs_plan_destroy(qs_plan* p);

/* ---- tile-shape tuning (the planner's fusion block size) ------------------- */

/* Record the tile shape plans of (dt, n) use when qs_plan_create gets 0:
 * 2^tile_bits amplitudes per tile, the lowest run_bits qubits in every tile.
 * Process-wide, thread-safe. */
QS_API qs_status qs_tune_set(qs_dtype dt, int n, int tile_bits, int run_bits);

/* The tile shape in effect for (dt, n) (tuned or built-in default). */
QS_API qs_status qs_tune_get(qs_dtype dt, int n, int* tile_bits, int* run_bits);

/* Autotuner: time the circuit `gates` on state s (its contents are
 * overwritten) for every tile shape that fits shared memory (tile bits from 9
 * or 10 up to the largest that fits, run bits 3..6), with CUDA events over
 * `reps` executions after one warm-up; record the fastest with qs_tune_set
 * and return it.  Synchronises the state's stream. */
QS_API qs_status qs_autotune(qs_state* s, const qs_gate* gates, int n_gates, const double* theta, int n_params,
                             int reps, int* best_tile_bits, int* best_run_bits, float* best_ms);

/* Plan, execute and destroy in one call. */
QS_API qs_status qs_run(qs_state* s, const qs_gate* gates, int n_gates, const double* theta, int n_params);

/* ---- dense block on the tensor cores (not in the paper) --------------------- */

/* Apply a dense 2^q x 2^q complex matrix U (row-major, U[r][c] as the (re, im)
 * doubles U[2 (r 2^q + c)], U[2 (r 2^q + c) + 1]) to qubits 0..q-1 of a
 * complex64 state: every group of 2^q consecutive amplitudes x (fixed higher
 * bits) becomes U x.  This is the product of a run of gates of Eq. 2 / Eq. 3
 * on those qubits applied as one matrix, where Section 4.4 applies the run
 * gate by gate inside a cached block.  It runs on the tensor cores: the block
 * is widened to 64 x 64 (I (x) U), the state and the matrix are split into
 * three bf16 pieces each, and six piece products accumulate in FP32 (an
 * error of the order of complex64 rounding).  One pass reads and writes the
 * state once.
 *   1 <= q <= 6, n >= 6, complex64 only (QS_EDTYPE for complex128); U need
 *   not be unitary.  The first call allocates a 96 KiB device buffer and a
 *   pinned host buffer kept by the state.  The call synchronises the state's
 *   stream; QS_ETIMEOUT if a bounded wait inside the kernel gave up. */
QS_API qs_status qs_apply_dense(qs_state* s, int q, const double* U);

/* ---- FP64 reductions (not in the paper) ---------------------------------- */

/* *out = sum_i |alpha_i|^2 (squared 2-norm = total probability). */
QS_API qs_status qs_norm(qs_state* s, double* out);

/* Marginal P(qubit k = 1) = sum over i with bit k set of |alpha_i|^2.
 * k >= 0: one value into p1[0]; k = -1: all n marginals into p1[0..n-1];
 * k = -2: the n marginals and then the total sum_i |alpha_i|^2 (the squared
 * norm) into p1[0..n], all from the same single read of the state.
 * For k = -1 / -2 on n >= 12 qubits, |alpha_i|^2 and the sums over each
 * thread's 16 amplitudes of a 4096-amplitude chunk are formed in double-float
 * arithmetic (about 47 significant bits) and the chunk sums accumulate in
 * FP64; a chunk holding a component of magnitude 2^60 or more is summed in
 * FP64 throughout.  Components below 2^-126 contribute nothing (an absolute
 * error below 2^-96 for 2^30 amplitudes). */
QS_API qs_status qs_prob(qs_state* s, int k, double* p1);

/* host_out[i] = |alpha_i|^2 for all 2^n amplitudes (host buffer of 2^n doubles). */
QS_API qs_status qs_probs(qs_state* s, double* host_out);

/* <psi|H|psi> for H = sum_j coef_j P_j with Z, ZZ and X terms. */
QS_API qs_status qs_expect(qs_state* s, const qs_term* terms, int n_terms, double* out);

/* All n marginals without allocating anything (the paper has no counterpart;
 * it exists for callers that cannot allocate device memory).  Some hosts must
 * not call cudaMalloc: an application whose own memory pool already holds the
 * device memory, so a fresh allocation would fail or fragment it; a
 * latency-critical loop that cannot afford the device-wide synchronisation an
 * allocation or free can cause; plugin code whose host forbids it.  This entry
 * point takes a caller-owned state and output and uses, for its partial sums,
 * a static device array of 16384 doubles (128 KiB) that every GPU loading the
 * library keeps until the process exits.
 *   dev_state: 2^n amplitudes of dtype dt in device memory (1 <= n <= 36;
 *              larger n returns QS_EINVAL because the static array is sized
 *              for at most 36 qubits).
 *   dev_out:   device buffer of n + 1 doubles: out[k] = P(qubit k = 1) for
 *              k < n, out[n] = sum_i |alpha_i|^2 (arithmetic as qs_prob, k = -2).
 * Asynchronous on cuda_stream; read dev_out after the stream has finished.
 * Each call whose stream is not capturing looks up the array's device
 * address (cudaGetSymbolAddress) with the current device; a captured call
 * reuses the address of the last such call on the device, so make the first
 * call on a device before any stream capture (QS_EINVAL otherwise).  All calls share the one array and every value
 * they read from it is written earlier in the same call, so nothing needs
 * clearing, but calls whose work overlaps on the GPU (other streams, other
 * threads) race on it and must be serialised by the caller. */
QS_API qs_status qs_marginals_noalloc(const void* dev_state, int n, qs_dtype dt, void* cuda_stream, double* dev_out);

/* ---- adjoint gradients (not in the paper) --------------------------------- */

/* One variational instance: E(theta) = <psi|H|psi>, psi = U_P..U_1 |0..0>. */
typedef struct {
    int32_t n;            /* qubits */
    int32_t n_gates;
    const qs_gate* gates; /* rotation kinds carry the parameter index */
    int32_t n_params;
    const double* theta;
    int32_t n_terms;
    const qs_term* terms;
} qs_instance;

/* A reusable batch: the instances' circuits and observables are copied and
 * planned once, device buffers are allocated once, and the first execution
 * captures every launch (and the upload of the gate matrices for the current
 * angles) into a CUDA graph that later executions replay.
 *   - Instances small enough to hold phi and lambda in one CTA's shared
 *     memory (n <= 12 for complex128, n <= 13 for complex64 on GB300) run in
 *     one persistent kernel, one CTA per instance taken from a work counter.
 *   - Larger instances with identical circuit structure (gate kinds, qubits,
 *     parameter indices, observable terms) form a group that runs as batched
 *     tile passes: forward passes, lambda = H psi, the energy, then reverse
 *     tile passes holding phi and lambda together.
 * flags: 1 = launch directly instead of capturing a graph.
 * The caller's stream must not be capturing; NULL gives the batch its own
 * non-blocking stream.  Angles passed at creation are used until an
 * execution passes new ones. */
typedef struct qs_batch qs_batch;
QS_API qs_status qs_batch_create(const qs_instance* batch, int n_inst, qs_dtype dt, void* cuda_stream, int flags,
                                 qs_batch** out);

/* Run the batch.  theta_all: the instances' angles concatenated in instance
 * order (sum of n_params doubles), or NULL for the last angles used.
 * energies: n_inst host doubles; grads: concatenated host gradients.
 * Synchronises the batch's stream. */
QS_API qs_status qs_batch_execute(qs_batch* b, const double* theta_all, double* energies, double* grads);

/* How the batch runs: instances in the persistent small-instance kernel,
 * number of structure groups, and kernel launches per execution. */
QS_API qs_status qs_batch_stats(const qs_batch* b, int* n_small, int* n_groups, int* n_launches);

QS_API qs_status qs_batch_destroy(qs_batch* b);

/* One-shot form of qs_batch_create / qs_batch_execute / qs_batch_destroy
 * (without graph capture).
 * Energies and gradients dE/dtheta of a batch of instances by one adjoint
 * reverse sweep each (Jones & Gacon, arXiv:2009.02823).  energies[i] gets
 * instance i's energy; grads gets the instances' gradients concatenated in
 * order (sum of n_params doubles).  Both are host buffers.  dt selects the
 * state precision; all reductions are FP64. */
QS_API qs_status qs_grad(const qs_instance* batch, int n_inst, qs_dtype dt, void* cuda_stream,
                  double* energies, double* grads);

/* ---- diagnostics ------------------------------------------------------------- */

/* Message of the last failure on the calling thread ("" if none). */
QS_API const char* qs_last_error(void);

/* Library version string. */
QS_API const char* qs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
