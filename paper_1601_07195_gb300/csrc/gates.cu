// gates.cu -- one gate = one pass over the state (Eq. 2, Eq. 3, and SWAP).
//
// The pair loop of Fig. 3 is flattened: work item p in [0, 2^(n-1)) maps to the
// pair (i0, i0 + 2^k) with i0 = p with a zero bit inserted at k, so the GPU
// needs no choice between the outer and inner loop (Section 4.2).  Consecutive
// threads take consecutive p: for k >= 1 (complex128) every 32-byte sector a
// warp touches is fully used, and each thread issues 128-bit loads.
// Controlled gates (Eq. 3) enumerate the 2^(n-2) pairs whose control bit is 1
// by inserting two zero bits and setting bit c, so the amplitudes with control
// bit 0 are never read (a controlled gate moves half the state, Table 2 case 3).
// Diagonal gates with q11 = 1 (T, controlled phase) read and write only the
// amplitudes they change.
#include "device.cuh"
#include "df.cuh"
#include "tile_df_ops.cuh"

namespace qs {

namespace {

constexpr int kThreads = 512;
constexpr int kUnroll = 2;

// MODE 0: single-qubit gate on t.  MODE 1: controlled on (c, t).  MODE 2: swap(t, c).
template <class R, int CLS, int MODE>
__global__ void __launch_bounds__(kThreads) k_strided(typename Amp<R>::T* __restrict__ psi, uint64_t n_items,
                                                      int t, int c, Mat2<R> mat) {
    using T = typename Amp<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const int lo = min(t, c), hi = max(t, c);
    for (uint64_t p0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; p0 < n_items; p0 += stride * kUnroll) {
        uint64_t i0[kUnroll], i1[kUnroll];
        T a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t p = p0 + u * stride;
            if (MODE == 0) {
                i0[u] = insert_zero(p, t);
                i1[u] = i0[u] | (1ull << t);
            } else if (MODE == 1) {
                i0[u] = insert_two_zeros(p, lo, hi) | (1ull << c);
                i1[u] = i0[u] | (1ull << t);
            } else {
                const uint64_t i = insert_two_zeros(p, lo, hi);
                i0[u] = i | (1ull << t);
                i1[u] = i | (1ull << c);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (p0 + u * stride < n_items) {
                if (CLS != GC_DIAG1) a[u] = psi[i0[u]];
                b[u] = psi[i1[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (p0 + u * stride < n_items) {
                pair_update<CLS>(mat.v, a[u], b[u]);
                if (CLS != GC_DIAG1) psi[i0[u]] = a[u];
                psi[i1[u]] = b[u];
            }
        }
    }
}

// complex128 with the 2x2 update in double-float form on the FP32 pipes: each
// amplitude is split into float pairs on load and rounded back on store.
template <int CLS, int MODE>
__global__ void __launch_bounds__(kThreads) k_strided_df(double2* __restrict__ psi, uint64_t n_items, int t, int c,
                                                         Mat2<float> hi, Mat2<float> lo) {
    float cc[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) { cc[2 * j] = hi.v[j]; cc[2 * j + 1] = lo.v[j]; }
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const int lo_q = min(t, c), hi_q = max(t, c);
    for (uint64_t p0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; p0 < n_items; p0 += stride * kUnroll) {
        uint64_t i0[kUnroll], i1[kUnroll];
        double2 a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t p = p0 + u * stride;
            if (MODE == 0) {
                i0[u] = insert_zero(p, t);
                i1[u] = i0[u] | (1ull << t);
            } else {
                i0[u] = insert_two_zeros(p, lo_q, hi_q) | (1ull << c);
                i1[u] = i0[u] | (1ull << t);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (p0 + u * stride < n_items) {
                if (CLS != GC_DIAG1) a[u] = psi[i0[u]];
                b[u] = psi[i1[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (p0 + u * stride < n_items) {
                float4 fa = CLS != GC_DIAG1 ? df_load_lean(a[u]) : make_float4(0, 0, 0, 0), fb = df_load_lean(b[u]);
                df_pair_update<CLS>(cc, fa, fb);
                if (CLS != GC_DIAG1) psi[i0[u]] = df_store_lean(fa);
                psi[i1[u]] = df_store_lean(fb);
            }
        }
    }
}

template <int CLS, int MODE>
cudaError_t launch_df(qs_state* s, uint64_t items, int t, int c, const double* m) {
    Mat2<float> hi, lo;
    for (int j = 0; j < 8; ++j) split_to_floats(m[j], hi.v[j], lo.v[j]);
    uint64_t want = (items + (uint64_t)kThreads * kUnroll - 1) / ((uint64_t)kThreads * kUnroll);
    uint64_t cap = (uint64_t)sm_count() * 16;
    unsigned blocks = (unsigned)(want < cap ? (want ? want : 1) : cap);
    k_strided_df<CLS, MODE><<<blocks, kThreads, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), items, t, c, hi, lo);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch_df(qs_state* s, int cls, uint64_t items, int t, int c, const double* m) {
    switch (cls) {
    case GC_GENERAL: return launch_df<GC_GENERAL, MODE>(s, items, t, c, m);
    case GC_REAL: return launch_df<GC_REAL, MODE>(s, items, t, c, m);
    case GC_DIAG: return launch_df<GC_DIAG, MODE>(s, items, t, c, m);
    case GC_DIAG1: return launch_df<GC_DIAG1, MODE>(s, items, t, c, m);
    default: return launch_df<GC_ANTIDIAG, MODE>(s, items, t, c, m);
    }
}

template <class R, int CLS, int MODE>
cudaError_t launch(qs_state* s, uint64_t items, int t, int c, const double* m) {
    Mat2<R> mat;
    for (int j = 0; j < 8; ++j) mat.v[j] = (R)m[j];
    uint64_t want = (items + (uint64_t)kThreads * kUnroll - 1) / ((uint64_t)kThreads * kUnroll);
    uint64_t cap = (uint64_t)sm_count() * 16;
    unsigned blocks = (unsigned)(want < cap ? (want ? want : 1) : cap);
    k_strided<R, CLS, MODE><<<blocks, kThreads, 0, s->stream>>>(
        reinterpret_cast<typename Amp<R>::T*>(s->data), items, t, c, mat);
    return cudaGetLastError();
}

template <class R, int MODE>
cudaError_t dispatch_cls(qs_state* s, int cls, uint64_t items, int t, int c, const double* m) {
    switch (cls) {
    case GC_GENERAL: return launch<R, GC_GENERAL, MODE>(s, items, t, c, m);
    case GC_REAL: return launch<R, GC_REAL, MODE>(s, items, t, c, m);
    case GC_DIAG: return launch<R, GC_DIAG, MODE>(s, items, t, c, m);
    case GC_DIAG1: return launch<R, GC_DIAG1, MODE>(s, items, t, c, m);
    case GC_ANTIDIAG: return launch<R, GC_ANTIDIAG, MODE>(s, items, t, c, m);
    default: return launch<R, GC_PERM, MODE>(s, items, t, c, m);
    }
}

template <class R>
cudaError_t dispatch(qs_state* s, const Op& op) {
    const uint64_t N = 1ull << s->n;
    if (op.kind == OP_1Q) return dispatch_cls<R, 0>(s, op.cls, N >> 1, op.t, op.t, op.m);
    if (op.kind == OP_CU) return dispatch_cls<R, 1>(s, op.cls, N >> 2, op.t, op.c, op.m);
    return launch<R, GC_PERM, 2>(s, N >> 2, op.t, op.c, op.m);
}

}  // namespace

qs_status launch_op(qs_state* s, const Op& op, bool arith_f64) {
    cudaError_t e;
    const uint64_t N = 1ull << s->n;
    if (s->dt == QS_C128 && !arith_f64 && op.kind != OP_SWAP && op.cls != GC_PERM) {
        // complex128 arithmetic in double-float; permutations stay exact moves of doubles
        e = op.kind == OP_1Q ? dispatch_df<0>(s, op.cls, N >> 1, op.t, op.t, op.m)
                             : dispatch_df<1>(s, op.cls, N >> 2, op.t, op.c, op.m);
    } else {
        e = (s->dt == QS_C128) ? dispatch<double>(s, op) : dispatch<float>(s, op);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gate kernel launch");
    return QS_OK;
}

}  // namespace qs
