// qs_internal.h -- structures shared by the host code (C ABI, planner) and the
// kernels of libqs.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qs.h"

namespace qs {

// Gate classes, decided on the host from the exact matrix entries.
enum GateClass : int {
    GC_GENERAL = 0,   // any 2x2
    GC_REAL = 1,      // every imaginary part is zero (H, RY)
    GC_DIAG = 2,      // q12 = q21 = 0 (RZ)
    GC_DIAG1 = 3,     // q12 = q21 = 0 and q11 = 1 exactly (T, phase): only |1> amplitudes change
    GC_ANTIDIAG = 4,  // q11 = q22 = 0
    GC_PERM = 5,      // exactly [[0,1],[1,0]] (X): a move
    // internal to double-float tile records (counted as GC_REAL): a real gate
    // whose four entries have one magnitude (H and its products with X and Z);
    // the record holds q11 and q21 and the signs s1 = q12/q11, s3 = q22/q21
    GC_REAL_BAL = 6,
    // internal to double-float tile records (counted as GC_GENERAL): a
    // single-qubit unitary written as  U = K diag(1, z) [[1, t], [-t, 1]] diag(1, y)
    // (GC_PRP) or, when |q12| > |q11|, as that form times X (GC_PRP_X: the pair
    // is swapped first).  The record holds y (doubles 0, 1), the real t
    // (double 2, 0 <= t <= 1) and z (doubles 4, 5); the complex scalar K is
    // left out and multiplied into another update of the same pass (plan.cu).
    GC_PRP = 7,
    GC_PRP_X = 8,
    // internal to double-float tile records (counted as GC_REAL): a balanced
    // real gate whose four entries share one magnitude, applied without its
    // scalar q11 (multiplied into another update of the pass, like K above):
    // a' = a + s1 b, b' = r (a + s3 b) with s1 = c[2], s3 = c[10], r = q21/q11 = c[8]
    GC_REAL_BAL1 = 9,
    // GC_PRP / GC_PRP_X with z = 1: the trailing phase diag(1, z) was moved into
    // a later op of the pass (plan.cu), so the record skips that product
    GC_PRP_NZ = 10,
    GC_PRP_X_NZ = 11
};

// Operation kinds after lowering the gate records.  OP_PRUN and OP_PDATA occur
// only in tile-pass records: a fused run of phase gates around one qubit (a
// header record followed by cls payload records of kind OP_PDATA).
enum OpKind : int { OP_1Q = 0, OP_CU = 1, OP_SWAP = 2, OP_PRUN = 3, OP_PDATA = 4, OP_DRUN = 5 };

// A lowered gate (host side, FP64 matrix).
struct Op {
    int kind;      // OpKind
    int cls;       // GateClass (unused for OP_SWAP)
    int t;         // target (first swap qubit)
    int c;         // control (second swap qubit), -1 if none
    double m[8];
};

inline bool op_is_diagonal(const Op& o) {
    return o.kind != OP_SWAP && (o.cls == GC_DIAG || o.cls == GC_DIAG1);
}

// A gate inside a tile pass, in tile coordinates (device side).
template <class R>
struct TileOp {
    int32_t kind;  // OpKind
    int32_t cls;   // GateClass
    int32_t tb;    // target tile bit, -1 if the target lies outside the tile (diagonal only)
    int32_t tq;    // target qubit
    int32_t cb;    // control (or second swap qubit) tile bit, -1 if outside / none
    int32_t cq;    // control (or second swap qubit) qubit, -1 if none
    int32_t pad0, pad1;
    R m[8];
};

// A tile-pass gate for complex128 states evaluated in double-float arithmetic:
// c[2j], c[2j+1] = (hi, lo) floats of matrix double j (q11r, q11i, ..., q22i).
struct TileOpDF {
    int32_t kind, cls, tb, tq, cb, cq, pad0, pad1;
    float c[16];
};

constexpr int kMaxTileBits = 14;

// Fused phase runs (plan.cu builds them, tile_ops.cuh / tile_df_ops.cuh apply
// them).  A run is a sequence of gates diagonal with q11 = 1 (phase gates on
// qubit j, controlled phases between j and other qubits k) that all involve
// the pivot qubit j, a tile bit jb.  The run multiplies each amplitude whose
// bit j is 1 by   C * T_lo[e & (2^lob - 1)] * T_hi[e >> lob]   where e is the
// tile index, T_lo / T_hi are products of the per-tile-bit factors psi_k over
// the set bits of the low / high part of e, and C is the product of the phase
// gates on j alone and of the factors of qubits outside the tile that are 1 in
// the tile's base index.  Records:
//   header  kind OP_PRUN, cls = payload records, tb = jb, tq = j,
//           cb = number of outside factors, cq = lob; factor slot 0 = the
//           phase gates on j alone (product)
//   payload ceil(b / 4) records of dense per-tile-bit factors psi_0..psi_{b-1}
//           (identity where no gate couples j with that bit), then
//           ceil(cb / 4) records of outside factors whose qubits are in the
//           int fields tb, tq, cb, cq (factor slots 0..3)
// A factor slot f of a record holds one complex number: m[2f], m[2f+1]
// (native records) or c[4f..4f+3] = re.hi, re.lo, im.hi, im.lo (double-float).
//
// Diagonal runs (kind OP_DRUN): a sequence of gates diagonal with q11 = 1 whose
// combined phase separates over the low and the high half of the tile index
// (phases on one qubit; controlled phases between a tile bit and an outside
// qubit, between two outside qubits, or between two tile bits of one half).
// The run multiplies every amplitude by  T_lo[e & (2^lob - 1)] * T_hi[e >> lob]
// where, for the tile with base index `base`,
//   psi_k   = product of the "bit" terms (k, y) with y none or bit y of base set,
//   C       = product of the "scalar" terms whose outside qubits are all set in base,
//   T_lo[i] = C * product of psi_k over the set bits k of i, times the "pair"
//             terms (x, y) of the low half with both bits set in i;
//   T_hi[u] = the same over the high half.
// Records:
//   header  kind OP_DRUN, cls = payload records, tb = number of terms, cq = lob
//   payload ceil(terms / 4) records; term f of a record: its int field
//           (tb, tq, cb, cq for f = 0..3) = type << 16 | x << 8 | y, factor slot f
//           type 0 bit: x = tile bit, y = outside qubit of the condition or 255
//           type 1 pair: x, y = tile bits of one half
//           type 2 scalar: x = outside qubit, y = second outside qubit or 255
inline int prun_lo_bits(int b) { return b / 2; }
// shared-memory entries (16 bytes each) for T_lo, T_hi, C and the per-bit factors
inline size_t prun_table_entries(int b) {
    return ((size_t)1 << prun_lo_bits(b)) + ((size_t)1 << (b - prun_lo_bits(b))) + 1 + (size_t)b;
}
constexpr int kDrunBit = 0, kDrunPair = 1, kDrunScalar = 2, kDrunNone = 255;

// Kernel argument describing one tile pass (by value).
struct TilePass {
    uint64_t nontile_mask;     // qubits that are NOT tile bits
    int32_t b;                 // tile bits (2^b amplitudes per tile)
    int32_t b0;                // tile bits 0..b0-1 are qubits 0..b0-1 (contiguous runs)
    int32_t hi_q[kMaxTileBits];// qubit of tile bit b0 + j
    int32_t op0;               // first op in the plan's TileOp array
    int32_t nops;
    uint64_t inst_stride;      // batched launches: amplitudes between instances (blockIdx.y)
    int32_t ops_stride;        // batched launches: op records between instances
    int32_t io;                // double-float passes: kIoPairsIn / kIoPairsOut (state held as float pairs)
};

// Double-float tile passes of one plan may hand the state to each other as
// float pairs (hi, lo) instead of rounded doubles: 16 bytes per amplitude
// either way, so no extra HBM traffic, and the split at load and the join at
// store happen once per run of such passes instead of once per pass.
constexpr int kIoPairsIn = 1;   // the pass reads float pairs (no split)
constexpr int kIoPairsOut = 2;  // the pass writes float pairs (no join)
constexpr int kIoDiscard = 4;   // reverse adjoint passes: the states are not read again, no store
constexpr int kIoDiagRuns = 8;  // the pass holds diagonal runs: launched with the kernel variant that applies them

// One pass of a plan, before its ops are converted to device records.
struct PassDesc {
    std::vector<int> members;  // op indices in execution order
    bool tile = false;         // false: a single op, run by the strided kernels
    uint64_t mask = 0;         // tile qubits (tile pass) or the op's qubits
    TilePass tp;               // tile passes: everything but op0 / nops / strides
    int bit_of[64];            // qubit -> tile bit, -1 if not a tile bit
};

// Greedy pass building (plan.cu): gates join a pass while their mixing qubits
// fit b tile bits, pulled ahead only over gates they commute with.  Passes of
// fewer than min_tile_members gates become single-op passes.
qs_status plan_passes(int n, const std::vector<Op>& ops, int b, int b0, bool fuse, int min_tile_members,
                      std::vector<PassDesc>& out);

// Diagonal runs (plan.cu) for other record builders: the length of the run
// worth fusing that starts at ops[i] of a pass (0: none), and its records.
size_t diag_run_length(const std::vector<Op>& ops, size_t i, const int* bit_of, int b, qs_dtype dt);
void diag_run_records(const std::vector<Op>& ops, size_t i0, size_t i1, const int* bit_of, int b,
                      std::vector<TileOpDF>& out);
void diag_run_records(const std::vector<Op>& ops, size_t i0, size_t i1, const int* bit_of, int b,
                      std::vector<TileOp<float>>& out);

}  // namespace qs

// Internal state handle.
struct qs_state {
    int n;
    qs_dtype dt;
    void* data;          // device amplitudes
    bool owned;
    cudaStream_t stream;
    int device;
    double* d_partials;  // reduction scratch: per-block FP64 partial sums
    size_t partials_cap; // doubles
    double* h_result;    // pinned host staging for reduction results
    size_t h_result_cap;
    bool arith_f64;      // complex128 single-gate kernels: native FP64 instead of double-float
    int lane_mode;       // single gates on targets 0..4: 0 measured choice, -1 pair kernel, 1 lane exchange
    void* d_dense;       // dense tensor-core block: operand image (bf16 pieces) + error flag
    void* h_dense;       // pinned host staging of that operand image
};

namespace qs {

// Error reporting (thread-local message).
void set_error(const std::string& msg);
qs_status fail(qs_status st, const std::string& msg);
qs_status cuda_fail(cudaError_t e, const char* what);
#define QS_CUDA_TRY(expr)                                        \
    do {                                                         \
        cudaError_t qs_e_ = (expr);                              \
        if (qs_e_ != cudaSuccess) return ::qs::cuda_fail(qs_e_, #expr); \
    } while (0)

inline size_t amp_bytes(qs_dtype dt) { return dt == QS_C128 ? 16 : 8; }

// Device properties cached per device.
int sm_count();
size_t smem_optin();

// Host-side classification and lowering of gate records.
int classify(const double m[8]);
qs_status lower_gates(const qs_gate* g, int ng, const double* theta, int np, int n, std::vector<Op>& out);

// Single-gate launchers (gates.cu).
qs_status launch_op(qs_state* s, const Op& op, bool arith_f64);

// Tile pass launcher (tile.cu); complex128 without arith_f64 goes to the
// double-float kernel (tile_df.cu), whose op array holds TileOpDF records.
// count > 1 runs `count` instances side by side (grid.y), strides in `pass`.
qs_status launch_tile_pass(qs_state* s, const void* d_ops, const TilePass& pass, bool arith_f64, unsigned count = 1);
cudaError_t launch_tile_df(qs_state* s, const void* d_ops, const TilePass& pass, unsigned count);
// Double-float pass whose op records (host copies, pass.op0 indexes h_ops) travel
// in the kernel's parameter block; at most tile_df_param_ops() ops.
cudaError_t launch_tile_df_params(qs_state* s, const TileOpDF* h_ops, const TilePass& pass);
int tile_df_param_ops();
// Native-arithmetic pass (TileOp<float> for complex64, TileOp<double> with f64)
// whose op records travel in the kernel's parameter block; at most
// tile_param_ops(f64) ops.
qs_status launch_tile_pass_params(qs_state* s, const void* h_ops, const TilePass& pass, bool f64);
int tile_param_ops(bool f64);
void split_to_floats(double x, float& hi, float& lo);
size_t tile_smem_bytes(qs_dtype dt, int b);
// dynamic shared memory of a tile pass: the tile, the phase-run tables, the
// offsets of the 2^(b - b0) contiguous runs
inline size_t tile_pass_smem(qs_dtype dt, int b, int b0) {
    return tile_smem_bytes(dt, b) + 16 * prun_table_entries(b) + ((size_t)8 << (b - b0));
}

// Dense 64 x 64 block on qubits 0..5 of a complex64 state, tensor cores (dense_tc.cu).
void dense_tc_operand(const double* U, uint16_t* out);
size_t dense_tc_operand_bytes();
cudaError_t launch_dense_tc(qs_state* s, const void* d_w, int* d_err, int max_ctas);
cudaError_t dense_tc_prepare();

// Reductions (reduce.cu).
qs_status ensure_scratch(qs_state* s, size_t partial_doubles, size_t result_doubles);

}  // namespace qs
