// plan.cu -- the circuit planner and executor.
//
// Section 4.4 groups consecutive gates on qubits below l_c and applies the
// group block by block while the block stays in the last-level cache.  Here a
// pass is a set of gates applied tile by tile in shared memory (tile.cu).  The
// planner builds passes greedily in gate order:
//   * qubits 0..b0-1 are always tile bits (contiguous global-memory runs);
//   * a gate joins the pass if its mixing qubits (target; both qubits of a
//     swap; none for a diagonal gate) fit in the b tile bits;
//   * a later gate may be pulled into the pass ahead of gates left behind when
//     it commutes with each of them: disjoint qubits, or both diagonal;
//   * a pass holding a single gate runs as a strided single-gate kernel
//     (gates.cu), which moves only the amplitudes the gate changes;
//   * after the greedy scan, a local search exchanges one tile qubit for one
//     left out while that admits more gates into the pass.
// The order of the gates within a pass and among the gates left behind is the
// circuit order, so the plan computes the same ordered product (up to
// rounding) as applying the gates one at a time.  Within a pass, adjacent
// same-qubit gates are multiplied into one matrix and runs of phase gates
// around one qubit become one table update; consecutive double-float passes
// hand the state over as float pairs (qs_internal.h).  For double-float
// passes the planner also rewrites single-qubit matrices into cheaper forms
// that leave a scalar out (phase-shear-phase for general unitaries, H-like
// gates without q11), moves those scalars into one other update of the pass
// and trailing phases into later updates on the same qubit: each rewrite
// changes matrices only, so the pass still applies the same product.
#include <algorithm>
#include <cmath>
#include <utility>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>

#include "device.cuh"
#include "../../include/qs_records.h"

namespace qs {
namespace {

constexpr int kWindow = 512;     // gates scanned ahead when filling a pass
constexpr int kSearchRounds = 4; // local-search rounds over the tile set of a pass

struct PlanPass {
    int kind;        // 0 = single gate, 1 = tile pass, 2 = dense block on qubits 0..5 (tensor cores)
    int dense = -1;  // dense pass: index of its operand image in the plan's dense buffer
    std::vector<double> U;  // dense pass: its 64 x 64 matrix (FP64, row-major (re, im))
    Op op;           // single gate
    TilePass tp;     // tile pass
    uint64_t mask;   // tile qubits (tile pass) or the gate's qubits
    int n_gates;
    bool moves_only; // every gate is a permutation (X, CNOT, SWAP): exact moves of 16-byte values
    std::vector<int> members;  // circuit positions of the pass's gates, in execution order
    int op_counts[3][6];       // ops the kernel applies, by kind (1q, controlled, swap) and class
    int balanced[2];           // of the real ones: balanced (H-like) single-qubit / controlled records
    int forms[3];              // single-qubit records that leave a scalar out: phase-shear-phase, balanced
                               // real; and of the first, those whose trailing phase a later op took
};

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

// Tile shape per (dtype, n): built-in defaults, overridden by qs_tune_set
// (the autotuner's choices).
std::mutex g_tune_mu;
std::map<std::pair<int, int>, std::pair<int, int>> g_tune;

void default_tile(qs_dtype dt, int n, int& b, int& b0) {
    if (dt == QS_C128) { b = 12; b0 = 4; }
    else { b = 12; b0 = 4; }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({(int)dt, n});
    if (it != g_tune.end()) { b = it->second.first; b0 = it->second.second; }
}

}  // namespace
}  // namespace qs

struct qs_plan {
    qs_state* s = nullptr;
    int flags = 0;
    std::vector<qs::PlanPass> passes;
    void* d_ops = nullptr;
    void* d_ops_f64 = nullptr;  // complex128 double-float plans: TileOp<double> copy for moves-only passes
    std::vector<qs::TileOpDF> h_ops_df;  // host copy of double-float records (passed as kernel parameters)
    std::vector<unsigned char> h_ops;     // host copy of native records (TileOp<float> or TileOp<double>)
    std::vector<qs::TileOp<double>> h_ops_f64;  // host copy of the moves-only records of double-float plans
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // optional per-pass timing: `records` sets of (passes + 1) events, used round robin
    std::vector<cudaEvent_t> events;
    int records = 0;
    int next_record = 0;
    int device_ops = 0;  // gate updates the kernels apply per execution (after fusion)
    // dense passes (complex64): operand images, uploaded once, then an error flag
    std::vector<uint16_t> h_dense;
    void* d_dense = nullptr;
    int n_dense = 0;
};

namespace qs {
namespace {

template <class OpT>
void fill_common(OpT& t, const Op& o, const int* bit_of) {
    t.kind = o.kind;
    t.cls = o.cls;
    t.tq = o.t;
    t.tb = bit_of[o.t];
    t.cq = o.c;
    t.cb = o.c >= 0 ? bit_of[o.c] : -1;
}

template <class OpT> OpT to_tile_op(const Op& o, const int* bit_of);

template <> TileOp<double> to_tile_op<TileOp<double>>(const Op& o, const int* bit_of) {
    TileOp<double> t{};
    fill_common(t, o, bit_of);
    for (int j = 0; j < 8; ++j) t.m[j] = o.m[j];
    return t;
}
template <> TileOp<float> to_tile_op<TileOp<float>>(const Op& o, const int* bit_of) {
    TileOp<float> t{};
    fill_common(t, o, bit_of);
    for (int j = 0; j < 8; ++j) t.m[j] = (float)o.m[j];
    return t;
}
template <> TileOpDF to_tile_op<TileOpDF>(const Op& o, const int* bit_of) {
    TileOpDF t{};
    fill_common(t, o, bit_of);
    for (int j = 0; j < 8; ++j) split_to_floats(o.m[j], t.c[2 * j], t.c[2 * j + 1]);
    // a real gate whose entries share one magnitude (H, HX, XH, ZH, ...):
    // a' = q11 (a + s1 b), b' = q21 (a + s3 b) with s1 = q12/q11, s3 = q22/q21 = +-1
    if (o.kind != OP_SWAP && o.cls == GC_REAL && o.m[0] != 0.0 && o.m[4] != 0.0 &&
        std::fabs(o.m[0]) == std::fabs(o.m[2]) && std::fabs(o.m[4]) == std::fabs(o.m[6])) {
        t.cls = GC_REAL_BAL;
        t.c[2] = (o.m[2] == o.m[0]) ? 1.0f : -1.0f;
        t.c[10] = (o.m[6] == o.m[4]) ? 1.0f : -1.0f;
    }
    return t;
}

// acc *= (r + i I)
void cmul_acc(double* acc, double r, double i) {
    const double ar = acc[0], ai = acc[1];
    acc[0] = ar * r - ai * i;
    acc[1] = ar * i + ai * r;
}

// ---- general single-qubit unitaries in phase-shear-phase form ------------------
// For a unitary V with |v11| >= |v12| (else V = U X, the columns swapped):
//   V = K diag(1, z) [[1, t], [-t, 1]] diag(1, y),
//   K = v11,  t = |v21| / |v11|,  z = -(v21 / v11) / t,  y = (v22 / v11) / z,
// which reproduces v11, v21 and v22 to rounding and gives v12 = K t y, equal to
// the given v12 up to the departure of V from unitarity.  The double-float
// kernel then applies two complex products to the |1> amplitude and a shear
// (one product and one sum per component) instead of the full 2x2 product.
struct PrpForm {
    bool swap;
    double K[2], t, y[2], z[2];
};

constexpr double kPrpTol = 4e-15;          // largest entry error of the form accepted
constexpr double kPrpMinScale = 0x1p-24;   // smallest product of left-out scalars K in one pass

void cdiv(double ar, double ai, double br, double bi, double& r, double& i) {
    const double d = br * br + bi * bi;
    r = (ar * br + ai * bi) / d;
    i = (ai * br - ar * bi) / d;
}

// unit_z: take z = 1 exactly (an op whose trailing phase a later op has taken)
bool prp_form(const Op& o, PrpForm& f, bool unit_z = false) {
    if (o.kind != OP_1Q || o.cls != GC_GENERAL) return false;
    const double* m = o.m;
    f.swap = std::hypot(m[2], m[3]) > std::hypot(m[0], m[1]);
    double v[8];
    const int col[2] = {f.swap ? 1 : 0, f.swap ? 0 : 1};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            v[2 * (2 * r + c)] = m[2 * (2 * r + col[c])];
            v[2 * (2 * r + c) + 1] = m[2 * (2 * r + col[c]) + 1];
        }
    const double a11 = std::hypot(v[0], v[1]), a21 = std::hypot(v[4], v[5]);
    if (!(a11 >= 0.5 && a11 <= 1.0 + 1e-12 && a21 > 0.0)) return false;
    f.K[0] = v[0];
    f.K[1] = v[1];
    f.t = a21 / a11;
    if (!(f.t <= 1.0 + 1e-12)) return false;
    double q[2];
    cdiv(v[4], v[5], v[0], v[1], q[0], q[1]);
    f.z[0] = unit_z ? 1.0 : -q[0] / f.t;
    f.z[1] = unit_z ? 0.0 : -q[1] / f.t;
    cdiv(v[6], v[7], v[0], v[1], q[0], q[1]);
    cdiv(q[0], q[1], f.z[0], f.z[1], f.y[0], f.y[1]);
    // the entries the form gives, against V
    auto cm = [](const double* a, const double* b, double* out) {
        const double r = a[0] * b[0] - a[1] * b[1], i = a[0] * b[1] + a[1] * b[0];
        out[0] = r;
        out[1] = i;
    };
    double e12[2], e21[2], e22[2], zy[2];
    cm(f.K, f.y, e12);
    e12[0] *= f.t;
    e12[1] *= f.t;
    cm(f.K, f.z, e21);
    e21[0] *= -f.t;
    e21[1] *= -f.t;
    cm(f.z, f.y, zy);
    cm(f.K, zy, e22);
    double err = 0.0;
    for (int j = 0; j < 2; ++j) {
        err = std::max(err, std::fabs(e12[j] - v[2 + j]));
        err = std::max(err, std::fabs(e21[j] - v[4 + j]));
        err = std::max(err, std::fabs(e22[j] - v[6 + j]));
    }
    return err <= kPrpTol;  // false for NaN
}

TileOpDF prp_record(const Op& o, const PrpForm& f, const int* bit_of) {
    TileOpDF r{};
    fill_common(r, o, bit_of);
    const bool unit_z = f.z[0] == 1.0 && f.z[1] == 0.0;
    r.cls = f.swap ? (unit_z ? GC_PRP_X_NZ : GC_PRP_X) : (unit_z ? GC_PRP_NZ : GC_PRP);
    split_to_floats(f.y[0], r.c[0], r.c[1]);
    split_to_floats(f.y[1], r.c[2], r.c[3]);
    split_to_floats(f.t, r.c[4], r.c[5]);
    split_to_floats(f.z[0], r.c[8], r.c[9]);
    split_to_floats(f.z[1], r.c[10], r.c[11]);
    return r;
}

// The trailing factor diag(1, z) of a phase-shear-phase op on qubit q can move
// into the next op of the pass that involves q when every op in between
// commutes with it (controlled ops with q as control, diagonal controlled ops)
// and that op takes it into its matrix at no cost: a general, diagonal or
// anti-diagonal single-qubit op on q (U diag(1, z) keeps its class).  Returns
// that op's index, or -1.
int phase_taker(const std::vector<Op>& ops, size_t i) {
    const int q = ops[i].t;
    for (size_t j = i + 1; j < ops.size(); ++j) {
        const Op& o = ops[j];
        if (o.t != q && o.c != q) continue;
        if (o.kind == OP_1Q)
            return (o.cls == GC_GENERAL || o.cls == GC_DIAG || o.cls == GC_DIAG1 || o.cls == GC_ANTIDIAG) ? (int)j
                                                                                                          : -1;
        if (o.kind == OP_CU && (o.c == q || o.cls == GC_DIAG || o.cls == GC_DIAG1)) continue;
        return -1;
    }
    return -1;
}

// m := diag(1, conj(z)) m (row 2) or m := m diag(1, z) (column 2)
void scale_row2(double* m, const double* z) {
    cmul_acc(&m[4], z[0], -z[1]);
    cmul_acc(&m[6], z[0], -z[1]);
}
void scale_col2(double* m, const double* z) {
    cmul_acc(&m[2], z[0], z[1]);
    cmul_acc(&m[6], z[0], z[1]);
}

// A balanced real single-qubit gate whose four entries share one magnitude
// (H, HX, XH, ZH, ...) = q11 [[1, s1], [r, r s3]] with s1, r, s3 = +-1: the
// record applies the bracket, the scalar q11 is left out like K above.
bool bal1_form(const Op& o) {
    const double a = std::fabs(o.m[0]);
    return o.kind == OP_1Q && o.cls == GC_REAL && a != 0.0 && std::fabs(o.m[2]) == a && std::fabs(o.m[4]) == a &&
           std::fabs(o.m[6]) == a;
}

TileOpDF bal1_record(const Op& o, const int* bit_of) {
    TileOpDF r{};
    fill_common(r, o, bit_of);
    r.cls = GC_REAL_BAL1;
    r.c[2] = (o.m[2] == o.m[0]) ? 1.0f : -1.0f;   // s1 = q12 / q11
    r.c[10] = (o.m[6] == o.m[4]) ? 1.0f : -1.0f;  // s3 = q22 / q21
    r.c[8] = (o.m[4] == o.m[0]) ? 1.0f : -1.0f;   // r = q21 / q11
    return r;
}

// Forms of the single-qubit ops of one pass (after fusion) that leave a
// scalar out: 1 = phase-shear-phase (scalar K), 2 = balanced real without q11;
// 0 = as given.  Returns the op (keeper) that takes the product of the
// scalars left out: a diagonal, anti-diagonal or general update whose class
// and cost a complex scale leaves unchanged; else the last phase-shear-phase
// candidate, which then stays general; else (real scalars only) the last
// balanced candidate, which keeps its scalar times the product.  Candidates
// whose scalar would bring the product below kPrpMinScale keep their own, so
// the amplitudes inside the pass grow by less than 2^24.  -1: no form taken.
//
// With pass_phase, a phase-shear-phase op whose trailing phase another op can
// take (phase_taker) hands it over first: ops[i] becomes diag(1, conj(z)) U_i,
// whose form has z = 1, and ops[j] becomes U_j diag(1, z), so the product of
// the pass is unchanged whatever form each op takes afterwards.
int choose_forms(std::vector<Op>& ops, bool balanced, bool pass_phase, std::vector<PrpForm>& forms,
                 std::vector<char>& form, double* Kpass) {
    forms.assign(ops.size(), PrpForm{});
    form.assign(ops.size(), 0);
    Kpass[0] = 1.0;
    Kpass[1] = 0.0;
    int keeper = -1, last_prp = -1, last_bal = -1;
    for (size_t i = 0; i < ops.size(); ++i) {
        if (prp_form(ops[i], forms[i])) {
            form[i] = 1;
            last_prp = (int)i;
            const int j = pass_phase ? phase_taker(ops, i) : -1;
            if (j >= 0) {
                const Op keep_i = ops[i], keep_j = ops[(size_t)j];
                const double z[2] = {forms[i].z[0], forms[i].z[1]};
                scale_row2(ops[i].m, z);
                scale_col2(ops[(size_t)j].m, z);
                PrpForm f;
                if (prp_form(ops[i], f, true)) {
                    forms[i] = f;
                } else {  // the form with z = 1 misses the tolerance: keep both as they were
                    ops[i] = keep_i;
                    ops[(size_t)j] = keep_j;
                }
            }
        } else if (balanced && bal1_form(ops[i])) {
            form[i] = 2;
            last_bal = (int)i;
        }
    }
    if (last_prp < 0 && last_bal < 0) return -1;
    for (size_t i = 0; i < ops.size() && keeper < 0; ++i) {
        const Op& o = ops[i];
        if (o.kind == OP_1Q && !form[i] && (o.cls == GC_DIAG || o.cls == GC_ANTIDIAG || o.cls == GC_GENERAL))
            keeper = (int)i;
    }
    if (keeper < 0) {
        keeper = last_prp >= 0 ? last_prp : last_bal;
        form[keeper] = 0;
    }
    double mag = 1.0;
    int used = 0;
    for (size_t i = 0; i < ops.size(); ++i) {
        if (!form[i]) continue;
        const double kr = form[i] == 1 ? forms[i].K[0] : ops[i].m[0], ki = form[i] == 1 ? forms[i].K[1] : 0.0;
        const double k = std::hypot(kr, ki);
        if (mag * k < kPrpMinScale) {
            form[i] = 0;
            continue;
        }
        mag *= k;
        cmul_acc(Kpass, kr, ki);
        ++used;
    }
    return used > 0 ? keeper : -1;
}

template <class OpT>
qs_status upload_ops(const std::vector<OpT>& v, void** dst) {
    if (v.empty()) return QS_OK;
    const size_t bytes = v.size() * sizeof(OpT);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); *dst = nullptr; return fail(QS_ENOMEM, "plan: cudaMalloc of tile ops failed"); }
    QS_CUDA_TRY(cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice));
    return QS_OK;
}

// ---- matrix fusion of single-qubit gates inside a pass ---------------------------
// Two single-qubit gates on the same qubit with nothing on that qubit between
// them (in the pass's execution order) are replaced by their product when the
// product's class is cheaper to apply than the two classes plus one op's
// fixed overhead (index math, op read, barrier).  Costs are instructions per
// amplitude pair of the tile kernels: double-float for complex128, FP32 for
// complex64.  A product that is exactly the identity is dropped.
int class_cost(int cls, qs_dtype dt) {
    static const int df[] = {200, 92, 92, 50, 92, 16};   // general, real, diag, diag1, antidiag, perm
    static const int f32[] = {48, 32, 32, 20, 32, 16};
    return dt == QS_C128 ? df[cls] : f32[cls];
}

void matmul2(const double* B, const double* A, double* M) {  // M = B A (A applied first)
    auto mul = [](double ar, double ai, double br, double bi, double& r, double& i) { r = ar * br - ai * bi; i = ar * bi + ai * br; };
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double x1r, x1i, x2r, x2i;
            mul(B[2 * (2 * r + 0)], B[2 * (2 * r + 0) + 1], A[2 * (2 * 0 + c)], A[2 * (2 * 0 + c) + 1], x1r, x1i);
            mul(B[2 * (2 * r + 1)], B[2 * (2 * r + 1) + 1], A[2 * (2 * 1 + c)], A[2 * (2 * 1 + c) + 1], x2r, x2i);
            M[2 * (2 * r + c)] = x1r + x2r;
            M[2 * (2 * r + c) + 1] = x1i + x2i;
        }
}

bool is_identity(const double* m) {
    return m[0] == 1.0 && m[1] == 0.0 && m[2] == 0.0 && m[3] == 0.0 && m[4] == 0.0 && m[5] == 0.0 && m[6] == 1.0 &&
           m[7] == 0.0;
}

std::vector<Op> fuse_single_qubit(const std::vector<Op>& ops, const std::vector<int>& members, qs_dtype dt,
                                  bool enable) {
    std::vector<Op> out;
    std::vector<char> dead;
    int pending[64];
    for (int q = 0; q < 64; ++q) pending[q] = -1;
    const int overhead = 12;
    for (int j : members) {
        const Op& o = ops[j];
        if (enable && o.kind == OP_1Q && pending[o.t] >= 0) {
            Op& a = out[pending[o.t]];
            Op m = a;
            matmul2(o.m, a.m, m.m);
            m.cls = classify(m.m);
            if (is_identity(m.m)) {
                dead[pending[o.t]] = 1;
                pending[o.t] = -1;
                continue;
            }
            if (class_cost(m.cls, dt) <= class_cost(a.cls, dt) + class_cost(o.cls, dt) + overhead) {
                a = m;
                continue;
            }
        }
        if (o.kind == OP_1Q) {
            pending[o.t] = (int)out.size();
        } else {
            pending[o.t] = -1;
            if (o.c >= 0) pending[o.c] = -1;
        }
        out.push_back(o);
        dead.push_back(0);
    }
    std::vector<Op> live;
    for (size_t i = 0; i < out.size(); ++i)
        if (!dead[i]) live.push_back(out[i]);
    return live;
}

// ---- fused runs of phase gates (record layout in qs_internal.h) -----------------
// A maximal sequence of consecutive ops of the pass (after matrix fusion) that
// are diagonal with q11 = 1 and all involve one tile qubit j.  Its product
// changes only amplitudes with bit j = 1, by a factor that is a product of
// one factor per other qubit: the kernel builds two tables over the low and
// high halves of the tile index and applies two complex products per changed
// amplitude instead of one product per gate.  Fused when the gates' cost
// (class_cost units) is above the run's own.
bool phase_gate(const Op& o) { return (o.kind == OP_1Q || o.kind == OP_CU) && o.cls == GC_DIAG1; }

int phase_gate_cost(const Op& o, qs_dtype dt) {
    const int c = class_cost(GC_DIAG1, dt);
    return (o.kind == OP_1Q ? c : c / 2) + 12;
}
int phase_run_cost(qs_dtype dt) { return 2 * class_cost(GC_DIAG1, dt) + 5 * 12; }

void set_slot(TileOpDF& r, int f, const double* v) {
    split_to_floats(v[0], r.c[4 * f], r.c[4 * f + 1]);
    split_to_floats(v[1], r.c[4 * f + 2], r.c[4 * f + 3]);
}
template <class R> void set_slot(TileOp<R>& r, int f, const double* v) {
    r.m[2 * f] = (R)v[0];
    r.m[2 * f + 1] = (R)v[1];
}
template <class OpT> void set_slot_qubit(OpT& r, int f, int q) {
    if (f == 0) r.tb = q;
    else if (f == 1) r.tq = q;
    else if (f == 2) r.cb = q;
    else r.cq = q;
}

// Records of the run ops[i0, i1) around pivot qubit j (tile bit bit_of[j]).
template <class OpT>
void emit_phase_run(const std::vector<Op>& ops, size_t i0, size_t i1, int j, const int* bit_of, int b,
                    std::vector<OpT>& out) {
    double c0[2] = {1.0, 0.0};
    std::vector<double> psi(2 * (size_t)b, 0.0);
    for (int k = 0; k < b; ++k) psi[2 * k] = 1.0;
    std::map<int, std::pair<double, double>> outside;  // qubit -> factor
    for (size_t i = i0; i < i1; ++i) {
        const Op& o = ops[i];
        const double fr = o.m[6], fi = o.m[7];  // q22: the phase applied when every qubit of the gate is 1
        const int k = o.kind == OP_1Q ? -1 : (o.t == j ? o.c : o.t);
        if (k < 0) {
            cmul_acc(c0, fr, fi);
        } else if (bit_of[k] >= 0) {
            cmul_acc(&psi[2 * bit_of[k]], fr, fi);
        } else {
            auto it = outside.emplace(k, std::make_pair(1.0, 0.0)).first;
            double acc[2] = {it->second.first, it->second.second};
            cmul_acc(acc, fr, fi);
            it->second = {acc[0], acc[1]};
        }
    }
    const int tile_rec = (b + 3) / 4, out_rec = ((int)outside.size() + 3) / 4;
    OpT h{};
    h.kind = OP_PRUN;
    h.cls = tile_rec + out_rec;
    h.tb = bit_of[j];
    h.tq = j;
    h.cb = (int)outside.size();
    h.cq = prun_lo_bits(b);
    set_slot(h, 0, c0);
    out.push_back(h);
    for (int r = 0; r < tile_rec; ++r) {
        OpT d{};
        d.kind = OP_PDATA;
        const double one[2] = {1.0, 0.0};
        for (int f = 0; f < 4; ++f) set_slot(d, f, 4 * r + f < b ? &psi[2 * (4 * r + f)] : one);
        out.push_back(d);
    }
    auto it = outside.begin();
    for (int r = 0; r < out_rec; ++r) {
        OpT d{};
        d.kind = OP_PDATA;
        d.tb = d.tq = d.cb = d.cq = 0;
        const double one[2] = {1.0, 0.0};
        for (int f = 0; f < 4; ++f) {
            if (it != outside.end()) {
                const double v[2] = {it->second.first, it->second.second};
                set_slot(d, f, v);
                set_slot_qubit(d, f, it->first);
                ++it;
            } else {
                set_slot(d, f, one);
            }
        }
        out.push_back(d);
    }
}

// ---- diagonal runs (record layout in qs_internal.h) --------------------------------
// A phase gate that can join a diagonal run of a pass with tile bits bit_of:
// its phase separates over the two halves of the tile index unless it couples
// a tile bit of the low half (< lob) with one of the high half.
bool drun_gate(const Op& o, const int* bit_of, int lob) {
    if (!phase_gate(o)) return false;
    if (o.kind == OP_1Q) return true;
    const int bt = bit_of[o.t], bc = bit_of[o.c];
    return !(bt >= 0 && bc >= 0 && ((bt < lob) != (bc < lob)));
}
// two complex products on every amplitude (twice a phase gate's half-tile
// product) and the per-tile tables
int diag_run_cost(qs_dtype dt) { return 4 * class_cost(GC_DIAG1, dt) + 8 * 12; }

// Length of the diagonal run starting at ops[i] (0: none worth fusing).
size_t find_diag_run(const std::vector<Op>& ops, size_t i, const int* bit_of, int b, qs_dtype dt) {
    const int lob = prun_lo_bits(b);
    size_t k = i;
    int cost = 0;
    while (k < ops.size() && drun_gate(ops[k], bit_of, lob)) {
        cost += phase_gate_cost(ops[k], dt);
        ++k;
    }
    return (k - i >= 4 && cost > diag_run_cost(dt)) ? k - i : 0;
}

// Records of the diagonal run ops[i0, i1): its gates as bit, pair and scalar
// terms, equal terms multiplied together.
template <class OpT>
void emit_diag_run(const std::vector<Op>& ops, size_t i0, size_t i1, const int* bit_of, int b,
                   std::vector<OpT>& out) {
    std::map<int, std::pair<double, double>> terms;  // type << 16 | x << 8 | y -> factor
    auto add = [&](int type, int x, int y, double fr, double fi) {
        auto it = terms.emplace(type << 16 | x << 8 | y, std::make_pair(1.0, 0.0)).first;
        double acc[2] = {it->second.first, it->second.second};
        cmul_acc(acc, fr, fi);
        it->second = {acc[0], acc[1]};
    };
    for (size_t i = i0; i < i1; ++i) {
        const Op& o = ops[i];
        const double fr = o.m[6], fi = o.m[7];  // q22: the phase where every qubit of the gate is 1
        if (o.kind == OP_1Q) {
            if (bit_of[o.t] >= 0) add(kDrunBit, bit_of[o.t], kDrunNone, fr, fi);
            else add(kDrunScalar, o.t, kDrunNone, fr, fi);
            continue;
        }
        const int bt = bit_of[o.t], bc = bit_of[o.c];
        if (bt >= 0 && bc >= 0) add(kDrunPair, std::min(bt, bc), std::max(bt, bc), fr, fi);
        else if (bt >= 0) add(kDrunBit, bt, o.c, fr, fi);
        else if (bc >= 0) add(kDrunBit, bc, o.t, fr, fi);
        else add(kDrunScalar, std::min(o.t, o.c), std::max(o.t, o.c), fr, fi);
    }
    const int n_terms = (int)terms.size(), n_rec = (n_terms + 3) / 4;
    const double one[2] = {1.0, 0.0};
    OpT h{};
    h.kind = OP_DRUN;
    h.cls = n_rec;
    h.tb = n_terms;
    h.tq = -1;
    h.cb = -1;
    h.cq = prun_lo_bits(b);
    set_slot(h, 0, one);
    out.push_back(h);
    auto it = terms.begin();
    for (int r = 0; r < n_rec; ++r) {
        OpT dr{};
        dr.kind = OP_PDATA;
        for (int f = 0; f < 4; ++f) {
            if (it != terms.end()) {
                const double v[2] = {it->second.first, it->second.second};
                set_slot(dr, f, v);
                set_slot_qubit(dr, f, it->first);
                ++it;
            } else {
                set_slot(dr, f, one);
                set_slot_qubit(dr, f, kDrunScalar << 16 | kDrunNone << 8 | kDrunNone);  // not read
            }
        }
        out.push_back(dr);
    }
}

// Length of the longest run starting at ops[i] and its pivot (-1: none worth fusing).
size_t find_phase_run(const std::vector<Op>& ops, size_t i, const int* bit_of, qs_dtype dt, int& pivot) {
    pivot = -1;
    if (!phase_gate(ops[i])) return 0;
    size_t best = 0;
    const int cand[2] = {ops[i].t, ops[i].c};
    for (int q : cand) {
        if (q < 0 || bit_of[q] < 0) continue;
        size_t k = i;
        int cost = 0;
        while (k < ops.size() && phase_gate(ops[k]) && (ops[k].t == q || ops[k].c == q)) {
            cost += phase_gate_cost(ops[k], dt);
            ++k;
        }
        if (k - i > best && cost > phase_run_cost(dt)) {
            best = k - i;
            pivot = q;
        }
    }
    return best;
}

// ---- dense blocks on qubits 0..5 (complex64 plans, unless QS_PLAN_NO_DENSE) -----
// A run of at least kDenseMinOps consecutive gates (circuit order) whose qubits
// all lie in 0..5 is multiplied into one 64 x 64 matrix on the host (FP64) and
// applied by the tensor-core block kernel (dense_tc.cu) as its own pass.  At
// n = 30 (complex64) one such pass takes 2.6 ms, about one HBM round trip, while
// each update of these gates costs the SIMT tile kernel about 0.25 ms inside a
// pass it shares with other gates, so shorter runs stay in tile passes.
constexpr int kDenseQubits = 6;
constexpr size_t kDenseMinOps = 10;

std::vector<std::pair<size_t, size_t>> dense_runs(const std::vector<Op>& ops) {
    std::vector<std::pair<size_t, size_t>> runs;
    size_t i = 0;
    while (i < ops.size()) {
        size_t j = i;
        while (j < ops.size() && ops[j].t < kDenseQubits && ops[j].c < kDenseQubits) ++j;
        if (j - i >= kDenseMinOps) runs.push_back({i, j});
        i = j > i ? j : i + 1;
    }
    return runs;
}

// U = product of ops[a..b) (last op leftmost) on qubits 0..5, row-major (re, im):
// every op applied to every column, as Eq. 2 / Eq. 3 apply it to a state.
void dense_product(const std::vector<Op>& ops, size_t a, size_t b, std::vector<double>& U) {
    const int D = 1 << kDenseQubits;
    U.assign(2 * D * D, 0.0);
    for (int i = 0; i < D; ++i) U[2 * (i * D + i)] = 1.0;
    for (size_t j = a; j < b; ++j) {
        const Op& o = ops[j];
        for (int col = 0; col < D; ++col) {
            double* u = &U[0];
            auto re = [&](int r) -> double& { return u[2 * (r * D + col)]; };
            auto im = [&](int r) -> double& { return u[2 * (r * D + col) + 1]; };
            if (o.kind == OP_SWAP) {
                for (int r = 0; r < D; ++r) {
                    if (((r >> o.t) & 1) || !((r >> o.c) & 1)) continue;
                    const int r2 = r ^ (1 << o.t) ^ (1 << o.c);
                    std::swap(re(r), re(r2));
                    std::swap(im(r), im(r2));
                }
                continue;
            }
            const double* m = o.m;
            for (int r = 0; r < D; ++r) {
                if ((r >> o.t) & 1) continue;
                if (o.kind == OP_CU && !((r >> o.c) & 1)) continue;
                const int r1 = r | (1 << o.t);
                const double ar = re(r), ai = im(r), br = re(r1), bi = im(r1);
                re(r) = m[0] * ar - m[1] * ai + m[2] * br - m[3] * bi;
                im(r) = m[0] * ai + m[1] * ar + m[2] * bi + m[3] * br;
                re(r1) = m[4] * ar - m[5] * ai + m[6] * br - m[7] * bi;
                im(r1) = m[4] * ai + m[5] * ar + m[6] * bi + m[7] * br;
            }
        }
    }
}

template <class OpT>
qs_status build(qs_plan* p, const std::vector<Op>& all_ops, int b, int b0, bool fuse, bool upload,
                const std::vector<std::pair<size_t, size_t>>& dense) {
    std::vector<OpT> tops;
    std::vector<TileOp<double>> t64;  // parallel records for moves-only passes of double-float plans
    const bool df = std::is_same<OpT, TileOpDF>::value;
    // segments of ordinary passes between the dense runs
    size_t seg0 = 0;
    for (size_t di = 0; di <= dense.size(); ++di) {
    const size_t seg1 = di < dense.size() ? dense[di].first : all_ops.size();
    std::vector<Op> seg_ops;
    if (!dense.empty()) seg_ops.assign(all_ops.begin() + seg0, all_ops.begin() + seg1);
    const std::vector<Op>& ops = dense.empty() ? all_ops : seg_ops;
    std::vector<PassDesc> descs;
    if (!ops.empty())
        if (qs_status st = plan_passes(p->s->n, ops, b, b0, fuse, 2, descs)) return st;
    for (const PassDesc& d : descs) {
        PlanPass pp{};
        pp.n_gates = (int)d.members.size();
        pp.members = d.members;
        for (int& m : pp.members) m += (int)seg0;  // circuit positions
        pp.mask = d.mask;
        if (!d.tile) {
            pp.kind = 0;
            pp.op = ops[d.members[0]];
            pp.op_counts[pp.op.kind][pp.op.cls] += 1;
            p->device_ops += 1;
            p->passes.push_back(pp);
            continue;
        }
        pp.kind = 1;
        pp.tp = d.tp;
        pp.tp.op0 = (int)tops.size();
        std::vector<Op> fused = fuse_single_qubit(ops, d.members, p->s->dt, !(p->flags & QS_PLAN_NO_MERGE));
        pp.moves_only = true;
        const bool runs = !(p->flags & QS_PLAN_NO_PHASE_RUNS);
        const bool druns = !(p->flags & QS_PLAN_NO_DIAG_RUNS);
        std::vector<PrpForm> forms;
        std::vector<char> form;
        double Kpass[2] = {1.0, 0.0};
        const int keeper =
            (df && !(p->flags & QS_PLAN_NO_PRP)) ? choose_forms(fused, true, true, forms, form, Kpass) : -1;
        if (keeper < 0) form.assign(fused.size(), 0);
        for (size_t i = 0; i < fused.size();) {
            int pivot = -1;
            const size_t len = runs ? find_phase_run(fused, i, d.bit_of, p->s->dt, pivot) : 0;
            const size_t dlen = druns ? find_diag_run(fused, i, d.bit_of, d.tp.b, p->s->dt) : 0;
            if (dlen > len) {
                const size_t before = tops.size();
                emit_diag_run(fused, i, i + dlen, d.bit_of, d.tp.b, tops);
                if (df) t64.resize(t64.size() + (tops.size() - before), TileOp<double>{});
                // two complex products on every amplitude: the arithmetic of two diagonal gates
                pp.op_counts[OP_1Q][GC_DIAG] += 2;
                pp.tp.io |= kIoDiagRuns;
                pp.moves_only = false;
                p->device_ops += 1;
                i += dlen;
                continue;
            }
            if (len > 0) {
                const size_t before = tops.size();
                emit_phase_run(fused, i, i + len, pivot, d.bit_of, d.tp.b, tops);
                if (df) t64.resize(t64.size() + (tops.size() - before), TileOp<double>{});
                // two complex products on half the tile: the arithmetic of one single-qubit diagonal gate
                pp.op_counts[OP_1Q][GC_DIAG] += 1;
                pp.moves_only = false;
                p->device_ops += 1;
                i += len;
                continue;
            }
            const size_t at = i++;
            Op o = fused[at];
            pp.op_counts[o.kind][o.cls] += 1;
            if constexpr (std::is_same<OpT, TileOpDF>::value) {
                if (form[at]) {
                    tops.push_back(form[at] == 1 ? prp_record(o, forms[at], d.bit_of) : bal1_record(o, d.bit_of));
                    t64.push_back(to_tile_op<TileOp<double>>(o, d.bit_of));
                    pp.forms[form[at] - 1] += 1;
                    if (tops.back().cls == GC_PRP_NZ || tops.back().cls == GC_PRP_X_NZ) pp.forms[2] += 1;
                    pp.moves_only = false;
                    p->device_ops += 1;
                    continue;
                }
                if ((int)at == keeper)  // the pass's scalars K, multiplied into every entry
                    for (int j = 0; j < 4; ++j) cmul_acc(&o.m[2 * j], Kpass[0], Kpass[1]);
            }
            tops.push_back(to_tile_op<OpT>(o, d.bit_of));
            if (tops.back().cls == GC_REAL_BAL) pp.balanced[o.kind == OP_CU ? 1 : 0] += 1;
            if (df) t64.push_back(to_tile_op<TileOp<double>>(o, d.bit_of));
            if (!(o.kind == OP_SWAP || o.cls == GC_PERM)) pp.moves_only = false;
            p->device_ops += 1;
        }
        pp.tp.nops = (int)tops.size() - pp.tp.op0;
        p->passes.push_back(pp);
    }
    if (di < dense.size()) {  // the dense run after this segment
        PlanPass pp{};
        pp.kind = 2;
        pp.dense = p->n_dense++;
        pp.mask = (1ull << kDenseQubits) - 1ull;
        pp.n_gates = (int)(dense[di].second - dense[di].first);
        for (size_t j = dense[di].first; j < dense[di].second; ++j) pp.members.push_back((int)j);
        pp.moves_only = false;
        dense_product(all_ops, dense[di].first, dense[di].second, pp.U);
        const size_t per = dense_tc_operand_bytes() / sizeof(uint16_t);
        p->h_dense.resize(p->h_dense.size() + per);
        dense_tc_operand(pp.U.data(), p->h_dense.data() + p->h_dense.size() - per);
        p->device_ops += 1;
        p->passes.push_back(pp);
        seg0 = dense[di].second;
    }
    }
    if (upload && p->n_dense > 0) {
        const size_t bytes = p->h_dense.size() * sizeof(uint16_t);
        cudaError_t e = cudaMalloc(&p->d_dense, bytes + 256);
        if (e != cudaSuccess) { cudaGetLastError(); p->d_dense = nullptr; return fail(QS_ENOMEM, "plan: dense operands"); }
        QS_CUDA_TRY(cudaMemcpy(p->d_dense, p->h_dense.data(), bytes, cudaMemcpyHostToDevice));
        QS_CUDA_TRY(cudaMemset((char*)p->d_dense + bytes, 0, sizeof(int)));
        QS_CUDA_TRY(dense_tc_prepare());
    }
    if (df) {
        // Consecutive tile passes hand the state to each other as float pairs: in
        // each run of tile passes, the first double-float pass splits the doubles
        // it loads and the last one joins what it stores.  Moves-only passes in
        // between move 16-byte values whatever they hold; single-gate passes
        // need doubles and end a run.
        size_t i = 0;
        while (i < p->passes.size()) {
            if (p->passes[i].kind != 1) { ++i; continue; }
            size_t j = i;
            std::vector<size_t> dfp;
            for (; j < p->passes.size() && p->passes[j].kind == 1; ++j)
                if (!p->passes[j].moves_only) dfp.push_back(j);
            for (size_t k = 0; k < dfp.size(); ++k) {
                int io = 0;
                if (k > 0) io |= kIoPairsIn;
                if (k + 1 < dfp.size()) io |= kIoPairsOut;
                p->passes[dfp[k]].tp.io = (p->passes[dfp[k]].tp.io & kIoDiagRuns) | io;
            }
            i = j;
        }
    }
    if (upload) {
        if (qs_status st = upload_ops(tops, &p->d_ops)) return st;
        if (qs_status st = upload_ops(t64, &p->d_ops_f64)) return st;
    }
    if (df) {
        p->h_ops_df.assign(reinterpret_cast<const TileOpDF*>(tops.data()),
                           reinterpret_cast<const TileOpDF*>(tops.data()) + tops.size());
        p->h_ops_f64 = t64;
    } else {
        const unsigned char* b = reinterpret_cast<const unsigned char*>(tops.data());
        p->h_ops.assign(b, b + tops.size() * sizeof(OpT));
    }
    return QS_OK;
}

qs_status launch_all(qs_plan* p, cudaEvent_t* ev) {
    const bool f64 = (p->flags & QS_PLAN_ARITH_F64) != 0;
    for (size_t i = 0; i < p->passes.size(); ++i) {
        const PlanPass& pp = p->passes[i];
        if (ev) QS_CUDA_TRY(cudaEventRecord(ev[i], p->s->stream));
        qs_status st;
        if (pp.kind == 0) st = launch_op(p->s, pp.op, f64);
        else if (pp.kind == 2) {
            const size_t per = dense_tc_operand_bytes();
            int* d_err = reinterpret_cast<int*>((char*)p->d_dense + per * (size_t)p->n_dense);
            cudaError_t e = launch_dense_tc(p->s, (const char*)p->d_dense + per * (size_t)pp.dense, d_err, 0);
            st = e == cudaSuccess ? QS_OK : cuda_fail(e, "dense block kernel launch");
        } else if (!p->h_ops_df.empty()) {  // complex128 in double-float
            if (pp.moves_only) {
                st = pp.tp.nops <= tile_param_ops(true)
                         ? launch_tile_pass_params(p->s, p->h_ops_f64.data(), pp.tp, true)
                         : launch_tile_pass(p->s, p->d_ops_f64, pp.tp, true);
            } else if (pp.tp.nops <= tile_df_param_ops()) {
                cudaError_t e = launch_tile_df_params(p->s, p->h_ops_df.data(), pp.tp);
                st = e == cudaSuccess ? QS_OK : cuda_fail(e, "tile kernel launch");
            } else {
                st = launch_tile_pass(p->s, p->d_ops, pp.tp, false);
            }
        } else {  // native FP32 (complex64) or FP64 (QS_PLAN_ARITH_F64) records
            const bool dbl = p->s->dt == QS_C128;
            st = pp.tp.nops <= tile_param_ops(dbl) ? launch_tile_pass_params(p->s, p->h_ops.data(), pp.tp, dbl)
                                                    : launch_tile_pass(p->s, p->d_ops, pp.tp, f64);
        }
        if (st != QS_OK) return st;
    }
    if (ev) QS_CUDA_TRY(cudaEventRecord(ev[p->passes.size()], p->s->stream));
    return QS_OK;
}

}  // namespace

size_t diag_run_length(const std::vector<Op>& ops, size_t i, const int* bit_of, int b, qs_dtype dt) {
    return find_diag_run(ops, i, bit_of, b, dt);
}
void diag_run_records(const std::vector<Op>& ops, size_t i0, size_t i1, const int* bit_of, int b,
                      std::vector<TileOpDF>& out) {
    emit_diag_run(ops, i0, i1, bit_of, b, out);
}
void diag_run_records(const std::vector<Op>& ops, size_t i0, size_t i1, const int* bit_of, int b,
                      std::vector<TileOp<float>>& out) {
    emit_diag_run(ops, i0, i1, bit_of, b, out);
}

qs_status plan_passes(int n, const std::vector<Op>& ops, int b, int b0, bool fuse, int min_tile_members,
                      std::vector<PassDesc>& out) {
    b = std::min(b, n);
    b0 = std::min(b0, b);
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    std::vector<char> taken(ops.size(), 0);
    size_t first = 0;
    out.clear();
    while (first < ops.size()) {
        std::vector<int> mem;
        uint64_t T = (1ull << b0) - 1ull;
        if (!fuse) {
            mem.push_back((int)first);
            taken[first] = 1;
        } else {
            const Op& f = ops[first];
            const uint64_t fneed = f.kind == OP_SWAP ? ((1ull << f.t) | (1ull << f.c))
                                                     : (op_is_diagonal(f) ? 0ull : (1ull << f.t));
            if (popc(T | fneed) > b) {  // the next gate cannot share a tile: it runs alone
                mem.push_back((int)first);
                taken[first] = 1;
                T |= fneed;
            }
        }
        if (fuse && mem.empty()) {
            // One greedy scan from tile set T0: gates join while their mixing
            // qubits fit b tile bits, pulled ahead only over gates they commute with.
            auto scan = [&](uint64_t T0, std::vector<int>& m) -> uint64_t {
                uint64_t Ts = T0, blocked_all = 0, blocked_nd = 0;
                int scanned = 0;
                m.clear();
                for (size_t j = first; j < ops.size() && scanned < kWindow; ++j) {
                    if (taken[j]) continue;
                    ++scanned;
                    const Op& o = ops[j];
                    const uint64_t sup = (1ull << o.t) | (o.c >= 0 ? (1ull << o.c) : 0ull);
                    const bool diag = op_is_diagonal(o);
                    const bool movable = diag ? !(sup & blocked_nd) : !(sup & blocked_all);
                    if (movable) {
                        const uint64_t need = o.kind == OP_SWAP ? sup : (diag ? 0ull : (1ull << o.t));
                        if (popc(Ts | need) <= b) {
                            Ts |= need;
                            m.push_back((int)j);
                            continue;
                        }
                    }
                    blocked_all |= sup;
                    if (!diag) blocked_nd |= sup;
                    if ((blocked_nd & all) == all) break;
                }
                return Ts;
            };
            T = scan(T, mem);
            // Local search over tile sets: exchanging one chosen qubit for one
            // left out can let more gates into the pass (the greedy takes
            // qubits in first-come order).  Each round keeps the best exchange;
            // fewer passes mean fewer HBM round trips for the same gates.
            const uint64_t low = (1ull << b0) - 1ull;
            std::vector<int> cand_mem;
            for (int round = 0; round < kSearchRounds && n > b; ++round) {
                const uint64_t base_T = T;
                uint64_t best_T = T;
                std::vector<int> best_mem;
                for (int q_out = b0; q_out < n; ++q_out) {
                    if (!((base_T >> q_out) & 1ull)) continue;
                    for (int q_in = b0; q_in < n; ++q_in) {
                        if ((base_T >> q_in) & 1ull) continue;
                        const uint64_t Tc = ((base_T & ~(1ull << q_out)) | (1ull << q_in)) | low;
                        const uint64_t Tr = scan(Tc, cand_mem);
                        if (cand_mem.size() > std::max(mem.size(), best_mem.size())) {
                            best_mem.swap(cand_mem);
                            best_T = Tr;
                        }
                    }
                }
                if (best_mem.empty()) break;
                mem.swap(best_mem);
                T = best_T;
            }
            for (int j : mem) taken[j] = 1;
        }
        if (mem.empty()) return fail(QS_EINVAL, "planner made no progress");  // unreachable: the first gate always fits
        while (first < ops.size() && taken[first]) ++first;

        PassDesc d;
        d.members = mem;
        for (int q = 0; q < 64; ++q) d.bit_of[q] = -1;
        std::memset(&d.tp, 0, sizeof(d.tp));
        const bool tile = (int)mem.size() >= min_tile_members && popc(T) <= b;
        if (!tile) {
            d.tile = false;
            const Op& o = ops[mem[0]];
            d.mask = (1ull << o.t) | (o.c >= 0 ? (1ull << o.c) : 0ull);
            out.push_back(d);
            continue;
        }
        // pad the tile to b bits with the lowest unused qubits (longer contiguous runs)
        for (int q = 0; q < n && popc(T) < b; ++q) T |= (1ull << q);
        int run = 0;
        while (run < n && ((T >> run) & 1ull)) ++run;
        d.tile = true;
        d.mask = T;
        TilePass& tp = d.tp;
        tp.b = b;
        tp.b0 = run < b ? run : b;
        tp.nontile_mask = all & ~T;
        int nh = 0;
        for (int q = 0; q < n; ++q) {
            if (!((T >> q) & 1ull)) continue;
            if (q < tp.b0) d.bit_of[q] = q;
            else { d.bit_of[q] = tp.b0 + nh; tp.hi_q[nh++] = q; }
        }
        out.push_back(d);
    }
    return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_plan_create(qs_state* s, const qs_gate* gates, int n_gates, const double* theta, int n_params,
                         int flags, int tile_bits, qs_plan** out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!s || !s->data) return fail(QS_EINVAL, "state handle is NULL");
    if (n_params < 0) return fail(QS_EINVAL, "n_params < 0");
    std::vector<Op> ops;
    if (qs_status st = lower_gates(gates, n_gates, theta, n_params, s->n, ops)) return st;
    int b, b0;
    default_tile(s->dt, s->n, b, b0);
    const int req_b = tile_bits & 0xFF, req_b0 = (tile_bits >> 8) & 0xFF;
    if (tile_bits < 0 || req_b > kMaxTileBits || req_b0 > kMaxTileBits) return fail(QS_EINVAL, "bad tile_bits");
    if (req_b > 0) b = req_b;
    if (req_b0 > 0) b0 = req_b0;
    if (b0 > b) b0 = b;
    if (!(flags & QS_PLAN_DRY_RUN) &&  // a host-only plan is not bound by this device's shared memory
        tile_pass_smem(s->dt, std::min(b, s->n), std::min(b0, s->n)) > smem_optin())
        return fail(QS_EINVAL, "tile shape too large for shared memory");
    qs_plan* p = new (std::nothrow) qs_plan();
    if (!p) return fail(QS_ENOMEM, "host allocation failed");
    p->s = s;
    p->flags = flags;
    const bool fuse = !(flags & QS_PLAN_NO_FUSION);
    const bool upload = !(flags & QS_PLAN_DRY_RUN);
    std::vector<std::pair<size_t, size_t>> dense;
    if (s->dt == QS_C64 && !(flags & QS_PLAN_NO_DENSE) && s->n >= kDenseQubits && fuse) dense = dense_runs(ops);
    qs_status st;
    if (s->dt == QS_C64) st = build<TileOp<float>>(p, ops, b, b0, fuse, upload, dense);
    else if (flags & QS_PLAN_ARITH_F64) st = build<TileOp<double>>(p, ops, b, b0, fuse, upload, dense);
    else st = build<TileOpDF>(p, ops, b, b0, fuse, upload, dense);
    if (st != QS_OK) {
        qs_plan_destroy(p);
        return st;
    }
    *out = p;
    return QS_OK;
}

qs_status qs_plan_execute(qs_plan* p) {
    if (!p || !p->s) return fail(QS_EINVAL, "plan is NULL");
    if (p->flags & QS_PLAN_DRY_RUN) return fail(QS_EINVAL, "a dry-run plan cannot be executed");
    const bool graph = (p->flags & QS_PLAN_GRAPH) && p->s->stream != nullptr;
    if (!graph) {
        cudaEvent_t* ev = nullptr;
        if (p->records > 0) {
            ev = &p->events[(size_t)p->next_record * (p->passes.size() + 1)];
            p->next_record = (p->next_record + 1) % p->records;
        }
        return launch_all(p, ev);
    }
    if (!p->gexec) {
        QS_CUDA_TRY(cudaStreamBeginCapture(p->s->stream, cudaStreamCaptureModeThreadLocal));
        qs_status st = launch_all(p, nullptr);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->s->stream, &g);
        if (st != QS_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        p->graph = g;
        QS_CUDA_TRY(cudaGraphInstantiate(&p->gexec, g, 0));
    }
    QS_CUDA_TRY(cudaGraphLaunch(p->gexec, p->s->stream));
    return QS_OK;
}

qs_status qs_plan_pass_op_counts(const qs_plan* p, int i, int* counts) {
    if (!p || !counts) return fail(QS_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    std::memcpy(counts, p->passes[i].op_counts, sizeof(p->passes[i].op_counts));
    return QS_OK;
}

qs_status qs_plan_pass_balanced(const qs_plan* p, int i, int* counts) {
    if (!p || !counts) return fail(QS_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    counts[0] = p->passes[i].balanced[0];
    counts[1] = p->passes[i].balanced[1];
    return QS_OK;
}

qs_status qs_plan_pass_prp(const qs_plan* p, int i, int* counts) {
    if (!p || !counts) return fail(QS_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    counts[0] = p->passes[i].forms[0];
    counts[1] = p->passes[i].forms[1];
    counts[2] = p->passes[i].forms[2];
    return QS_OK;
}

qs_status qs_plan_device_ops(const qs_plan* p, int* n_ops) {
    if (!p || !n_ops) return fail(QS_EINVAL, "NULL argument");
    *n_ops = p->device_ops;
    return QS_OK;
}

qs_status qs_plan_stats(const qs_plan* p, int* n_passes, int* n_tile_passes, int* n_launches) {
    if (!p) return fail(QS_EINVAL, "plan is NULL");
    int tiles = 0;
    for (const PlanPass& pp : p->passes) tiles += pp.kind == 1;
    if (n_passes) *n_passes = (int)p->passes.size();
    if (n_tile_passes) *n_tile_passes = tiles;
    if (n_launches) *n_launches = (int)p->passes.size();
    return QS_OK;
}

qs_status qs_plan_pass(const qs_plan* p, int i, int* kind, int* n_gates, uint64_t* tile_mask) {
    if (!p) return fail(QS_EINVAL, "plan is NULL");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    const PlanPass& pp = p->passes[i];
    if (kind) *kind = pp.kind;
    if (n_gates) *n_gates = pp.n_gates;
    if (tile_mask) *tile_mask = pp.mask;
    return QS_OK;
}

qs_status qs_plan_pass_dense(const qs_plan* p, int i, double* U) {
    if (!p || !U) return fail(QS_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    if (p->passes[i].kind != 2) return fail(QS_EINVAL, "pass is not a dense block");
    std::memcpy(U, p->passes[i].U.data(), p->passes[i].U.size() * sizeof(double));
    return QS_OK;
}

qs_status qs_plan_pass_records(const qs_plan* p, int i, void* out, int cap, int* n, int* tile_qubits, int* b,
                               int* format) {
    static_assert(sizeof(qs::TileOpDF) == 96 && sizeof(qs::TileOp<float>) == 64 &&
                      sizeof(qs::TileOp<double>) == 96,
                  "record layouts of qs_records.h");
    if (!p || !n) return fail(QS_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    const PlanPass& pp = p->passes[i];
    const bool df = !p->h_ops_df.empty();
    const size_t rec = df ? sizeof(qs::TileOpDF)
                          : (p->s->dt == QS_C64 ? sizeof(qs::TileOp<float>) : sizeof(qs::TileOp<double>));
    const unsigned char* base = df ? reinterpret_cast<const unsigned char*>(p->h_ops_df.data()) : p->h_ops.data();
    const bool has = pp.kind == 1 && (df || !p->h_ops.empty());
    *n = has ? pp.tp.nops : 0;
    if (b) *b = has ? pp.tp.b : 0;
    if (format) *format = df ? 1 : (p->s->dt == QS_C64 ? 2 : 3);
    if (!has) return QS_OK;
    if (tile_qubits) {
        for (int k = 0; k < pp.tp.b0; ++k) tile_qubits[k] = k;
        for (int k = pp.tp.b0; k < pp.tp.b; ++k) tile_qubits[k] = pp.tp.hi_q[k - pp.tp.b0];
    }
    if (out) {
        if (cap < pp.tp.nops) return fail(QS_EINVAL, "record buffer too small");
        std::memcpy(out, base + rec * (size_t)pp.tp.op0, rec * (size_t)pp.tp.nops);
    }
    return QS_OK;
}

qs_status qs_plan_pass_gates(const qs_plan* p, int i, int* positions) {
    if (!p || !positions) return fail(QS_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)p->passes.size()) return fail(QS_EINVAL, "pass index out of range");
    const PlanPass& pp = p->passes[i];
    for (size_t j = 0; j < pp.members.size(); ++j) positions[j] = pp.members[j];
    return QS_OK;
}

qs_status qs_plan_set_timing(qs_plan* p, int records) {
    if (!p) return fail(QS_EINVAL, "plan is NULL");
    if (records < 0 || records > 4096) return fail(QS_EINVAL, "records must be in [0, 4096]");
    if (p->flags & (QS_PLAN_DRY_RUN | QS_PLAN_GRAPH)) return fail(QS_EINVAL, "timing needs an eager, executable plan");
    if (!p->events.empty()) cudaStreamSynchronize(p->s->stream);
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    p->events.clear();
    p->records = 0;
    p->next_record = 0;
    const size_t count = (size_t)records * (p->passes.size() + 1);
    p->events.resize(count);
    for (size_t i = 0; i < count; ++i) {
        cudaError_t e = cudaEventCreate(&p->events[i]);
        if (e != cudaSuccess) { p->events.resize(i); return cuda_fail(e, "cudaEventCreate"); }
    }
    p->records = records;
    return QS_OK;
}

qs_status qs_plan_pass_times(qs_plan* p, int record, float* ms) {
    if (!p || !ms) return fail(QS_EINVAL, "NULL argument");
    if (record < 0 || record >= p->records) return fail(QS_EINVAL, "record out of range");
    cudaEvent_t* ev = &p->events[(size_t)record * (p->passes.size() + 1)];
    QS_CUDA_TRY(cudaEventSynchronize(ev[p->passes.size()]));
    for (size_t i = 0; i < p->passes.size(); ++i) QS_CUDA_TRY(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
    return QS_OK;
}

qs_status qs_plan_destroy(qs_plan* p) {
    if (!p) return QS_OK;
    if (p->s && p->s->stream && !(p->flags & QS_PLAN_DRY_RUN)) cudaStreamSynchronize(p->s->stream);
    int timed_out = 0;
    if (p->d_dense) {  // did a bounded wait of a dense pass give up?
        const size_t bytes = p->h_dense.size() * sizeof(uint16_t);
        if (cudaMemcpy(&timed_out, (char*)p->d_dense + bytes, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            timed_out = 0;
        }
        cudaFree(p->d_dense);
    }
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_ops) cudaFree(p->d_ops);
    if (p->d_ops_f64) cudaFree(p->d_ops_f64);
    delete p;
    if (timed_out) return fail(QS_ETIMEOUT, "dense block: a bounded wait inside the kernel gave up");
    return QS_OK;
}

qs_status qs_tune_set(qs_dtype dt, int n, int tile_bits, int run_bits) {
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EDTYPE, "unknown dtype");
    if (n < 1 || n > 40 || tile_bits < 1 || tile_bits > kMaxTileBits || run_bits < 0 || run_bits > tile_bits)
        return fail(QS_EINVAL, "bad tuning entry");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{(int)dt, n}] = {tile_bits, run_bits};
    return QS_OK;
}

qs_status qs_tune_get(qs_dtype dt, int n, int* tile_bits, int* run_bits) {
    if (!tile_bits || !run_bits) return fail(QS_EINVAL, "NULL argument");
    int b, b0;
    default_tile(dt, n, b, b0);
    *tile_bits = b;
    *run_bits = b0;
    return QS_OK;
}

qs_status qs_autotune(qs_state* s, const qs_gate* gates, int n_gates, const double* theta, int n_params, int reps,
                      int* best_tile_bits, int* best_run_bits, float* best_ms) {
    if (!s || !s->data) return fail(QS_EINVAL, "state handle is NULL");
    if (reps < 1 || reps > 100) return fail(QS_EINVAL, "reps must be in [1, 100]");
    const int bmin = s->dt == QS_C128 ? 9 : 10;
    float best = 1e30f;
    int bb = 0, bb0 = 0;
    cudaEvent_t e0, e1;
    QS_CUDA_TRY(cudaEventCreate(&e0));
    QS_CUDA_TRY(cudaEventCreate(&e1));
    qs_status out = QS_OK;
    for (int b = std::min(bmin, s->n); b <= std::min(kMaxTileBits, s->n) && out == QS_OK; ++b) {
        for (int b0 = 3; b0 <= 6 && b0 <= b - 2; ++b0) {
            if (tile_pass_smem(s->dt, b, b0) > smem_optin()) continue;
            qs_plan* p = nullptr;
            out = qs_plan_create(s, gates, n_gates, theta, n_params, QS_PLAN_DEFAULT, b | (b0 << 8), &p);
            if (out != QS_OK) break;
            out = qs_plan_execute(p);  // warm-up
            float ms = 0.0f;
            if (out == QS_OK && cudaEventRecord(e0, s->stream) == cudaSuccess) {
                for (int r = 0; r < reps && out == QS_OK; ++r) out = qs_plan_execute(p);
                cudaEventRecord(e1, s->stream);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
            }
            qs_plan_destroy(p);
            if (out == QS_OK && ms < best) { best = ms; bb = b; bb0 = b0; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out != QS_OK) return out;
    if (bb == 0) return fail(QS_EINVAL, "no tile shape fits this state");
    qs_tune_set(s->dt, s->n, bb, bb0);
    if (best_tile_bits) *best_tile_bits = bb;
    if (best_run_bits) *best_run_bits = bb0;
    if (best_ms) *best_ms = best;
    return QS_OK;
}

qs_status qs_run(qs_state* s, const qs_gate* gates, int n_gates, const double* theta, int n_params) {
    qs_plan* p = nullptr;
    if (qs_status st = qs_plan_create(s, gates, n_gates, theta, n_params, QS_PLAN_DEFAULT, 0, &p)) return st;
    qs_status st = qs_plan_execute(p);
    // the plan's op table must outlive the launches that read it
    cudaError_t e = cudaStreamSynchronize(s->stream);
    qs_plan_destroy(p);
    if (st != QS_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "qs_run synchronize");
    return QS_OK;
}

}  // extern "C"
