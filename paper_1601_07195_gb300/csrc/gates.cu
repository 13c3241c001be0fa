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
// amplitudes they change.  Targets 0..4 of non-diagonal gates exchange the
// partner between the lanes of a warp instead (k_lanes below).
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
    const uint64_t hm_lo = ~0ull << lo, hm_hi = ~0ull << hi;  // zero-bit insertion as p + (p & hm)
    for (uint64_t p0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; p0 < n_items; p0 += stride * kUnroll) {
        uint64_t i0[kUnroll], i1[kUnroll];
        T a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t p = p0 + u * stride;
            if (MODE == 0) {
                i0[u] = insert_zero_hm(p, hm_lo);  // lo = t here
                i1[u] = i0[u] | (1ull << t);
            } else if (MODE == 1) {
                i0[u] = insert_zero_hm(insert_zero_hm(p, hm_lo), hm_hi) | (1ull << c);
                i1[u] = i0[u] | (1ull << t);
            } else {
                const uint64_t i = insert_zero_hm(insert_zero_hm(p, hm_lo), hm_hi);
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
    const uint64_t hm_lo = ~0ull << lo_q, hm_hi = ~0ull << hi_q;  // zero-bit insertion as p + (p & hm)
    for (uint64_t p0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; p0 < n_items; p0 += stride * kUnroll) {
        uint64_t i0[kUnroll], i1[kUnroll];
        double2 a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t p = p0 + u * stride;
            if (MODE == 0) {
                i0[u] = insert_zero_hm(p, hm_lo);  // lo_q = t here
                i1[u] = i0[u] | (1ull << t);
            } else {
                i0[u] = insert_zero_hm(insert_zero_hm(p, hm_lo), hm_hi) | (1ull << c);
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

// ---- targets 0..4: the partner in another lane (the GPU form of the SIMD lanes of Section 4.1)
//
// A warp reads 32 consecutive amplitudes, one per lane (fully used sectors, no
// pair indexing).  For target t < 5 the partner of lane l is lane l ^ 2^t,
// fetched with __shfl_xor_sync, and each lane computes and writes only its own
// amplitude with the row of Eq. 2 its bit t selects:
//   bit t of l = 0 (self = alpha_{..0_t..}):  self' = q11 self + q12 partner
//   bit t of l = 1 (self = alpha_{..1_t..}):  self' = q22 self + q21 partner
// The row is fixed per lane, so it is selected once.  Controlled gates with a
// control c >= 5 (a bit above the lanes) visit only the 32-amplitude groups
// whose bit c is 1; a control among the lanes stays with the pair kernel, which
// reads only the amplitudes whose control bit is 1.  Diagonal classes need no
// partner and stay with the pair kernel too.
constexpr int kLaneUnroll = 4;  // 32-amplitude groups per warp in flight

template <class T>
__device__ __forceinline__ T shfl_xor_amp(T v, unsigned m) {
    T o;
    o.x = __shfl_xor_sync(0xffffffffu, v.x, m);
    o.y = __shfl_xor_sync(0xffffffffu, v.y, m);
    return o;
}
__device__ __forceinline__ float4 shfl_xor_amp(float4 v, unsigned m) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                       __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}

// Group g (MODE 0: g < 2^(n-5); MODE 1: g < 2^(n-6)) as the index of its first
// amplitude: MODE 1 inserts bit c - 5 of the group number, set to 1.
template <int MODE>
__device__ __forceinline__ uint64_t lane_group_base(uint64_t g, int c) {
    if (MODE == 0) return g << 5;
    return (insert_zero(g, c - 5) | (1ull << (c - 5))) << 5;
}

template <class R, int CLS, int MODE>
__global__ void __launch_bounds__(kThreads) k_lanes(typename Amp<R>::T* __restrict__ psi, uint64_t n_groups, int t,
                                                    int c, Mat2<R> mat) {
    using T = typename Amp<R>::T;
    const unsigned lane = threadIdx.x & 31u, xm = 1u << t;
    const uint64_t warp = ((uint64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint64_t warps = ((uint64_t)gridDim.x * kThreads) >> 5;
    const bool one = (lane >> t) & 1u;
    const R sr = one ? mat.v[6] : mat.v[0], si = one ? mat.v[7] : mat.v[1];  // on self
    const R pr = one ? mat.v[4] : mat.v[2], pi = one ? mat.v[5] : mat.v[3];  // on the partner
    for (uint64_t g0 = warp; g0 < n_groups; g0 += warps * kLaneUnroll) {
        uint64_t idx[kLaneUnroll];
        T v[kLaneUnroll];
#pragma unroll
        for (int u = 0; u < kLaneUnroll; ++u) {
            const uint64_t g = g0 + u * warps;  // uniform over the warp
            idx[u] = lane_group_base<MODE>(g, c) + lane;
            if (g < n_groups) v[u] = psi[idx[u]];
        }
#pragma unroll
        for (int u = 0; u < kLaneUnroll; ++u) {
            if (g0 + u * warps < n_groups) {
                const T w = shfl_xor_amp(v[u], xm);
                T o;
                if constexpr (CLS == GC_GENERAL) o = cmul2(sr, si, v[u], pr, pi, w);
                else if constexpr (CLS == GC_REAL) o = rmul2(sr, v[u], pr, w);
                else if constexpr (CLS == GC_ANTIDIAG) o = cmul(pr, pi, w);
                else o = w;  // GC_PERM: a move, bit-exact
                psi[idx[u]] = o;
            }
        }
    }
}

// complex128 in double-float form: the lane's row as DF constants
// (self re, self im, partner re, partner im), then the update of df.cuh
template <int CLS, int MODE>
__global__ void __launch_bounds__(kThreads) k_lanes_df(double2* __restrict__ psi, uint64_t n_groups, int t, int c,
                                                       Mat2<float> hi, Mat2<float> lo) {
    const unsigned lane = threadIdx.x & 31u, xm = 1u << t;
    const uint64_t warp = ((uint64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint64_t warps = ((uint64_t)gridDim.x * kThreads) >> 5;
    const bool one = (lane >> t) & 1u;
    float cc[8];
    cc[0] = one ? hi.v[6] : hi.v[0]; cc[1] = one ? lo.v[6] : lo.v[0];
    cc[2] = one ? hi.v[7] : hi.v[1]; cc[3] = one ? lo.v[7] : lo.v[1];
    cc[4] = one ? hi.v[4] : hi.v[2]; cc[5] = one ? lo.v[4] : lo.v[2];
    cc[6] = one ? hi.v[5] : hi.v[3]; cc[7] = one ? lo.v[5] : lo.v[3];
    for (uint64_t g0 = warp; g0 < n_groups; g0 += warps * kLaneUnroll) {
        uint64_t idx[kLaneUnroll];
        double2 v[kLaneUnroll];
#pragma unroll
        for (int u = 0; u < kLaneUnroll; ++u) {
            const uint64_t g = g0 + u * warps;
            idx[u] = lane_group_base<MODE>(g, c) + lane;
            if (g < n_groups) v[u] = psi[idx[u]];
        }
#pragma unroll
        for (int u = 0; u < kLaneUnroll; ++u) {
            if (g0 + u * warps < n_groups) {
                const float4 a = df_load_lean(v[u]);
                const float4 w = shfl_xor_amp(a, xm);
                float4 o;
                if constexpr (CLS == GC_GENERAL) o = df_cmul2(cc, 0, 1, a, 2, 3, w);
                else if constexpr (CLS == GC_REAL) o = df_rmul2(cc, 0, a, 2, w);
                else o = df_cmul(cc, 2, 3, w);  // GC_ANTIDIAG
                psi[idx[u]] = df_store_lean(o);
            }
        }
    }
}

unsigned lane_blocks(uint64_t n_groups) {
    const uint64_t warps_per_block = kThreads / 32;
    const uint64_t want = (n_groups + warps_per_block * kLaneUnroll - 1) / (warps_per_block * kLaneUnroll);
    const uint64_t cap = (uint64_t)sm_count() * 16;
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

template <class R, int CLS, int MODE>
cudaError_t launch_lanes(qs_state* s, uint64_t groups, int t, int c, const double* m) {
    Mat2<R> mat;
    for (int j = 0; j < 8; ++j) mat.v[j] = (R)m[j];
    k_lanes<R, CLS, MODE><<<lane_blocks(groups), kThreads, 0, s->stream>>>(
        reinterpret_cast<typename Amp<R>::T*>(s->data), groups, t, c, mat);
    return cudaGetLastError();
}

template <int CLS, int MODE>
cudaError_t launch_lanes_df(qs_state* s, uint64_t groups, int t, int c, const double* m) {
    Mat2<float> hi, lo;
    for (int j = 0; j < 8; ++j) split_to_floats(m[j], hi.v[j], lo.v[j]);
    k_lanes_df<CLS, MODE><<<lane_blocks(groups), kThreads, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), groups,
                                                                          t, c, hi, lo);
    return cudaGetLastError();
}

// The lane kernels of one precision, by class (GENERAL, REAL, ANTIDIAG, PERM).
template <class R, int MODE>
cudaError_t dispatch_lanes(qs_state* s, int cls, uint64_t groups, int t, int c, const double* m, bool df) {
    if (df && cls != GC_PERM) {
        switch (cls) {
        case GC_GENERAL: return launch_lanes_df<GC_GENERAL, MODE>(s, groups, t, c, m);
        case GC_REAL: return launch_lanes_df<GC_REAL, MODE>(s, groups, t, c, m);
        default: return launch_lanes_df<GC_ANTIDIAG, MODE>(s, groups, t, c, m);
        }
    }
    switch (cls) {
    case GC_GENERAL: return launch_lanes<R, GC_GENERAL, MODE>(s, groups, t, c, m);
    case GC_REAL: return launch_lanes<R, GC_REAL, MODE>(s, groups, t, c, m);
    case GC_ANTIDIAG: return launch_lanes<R, GC_ANTIDIAG, MODE>(s, groups, t, c, m);
    default: return launch_lanes<R, GC_PERM, MODE>(s, groups, t, c, m);
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

// Whether a gate takes the lane-exchange kernel.  The measured choice
// (lane_mode 0; n = 30, GB/s for targets 0..4, lanes vs pair kernel):
//   native FP64:  single-qubit 2,333 vs 2,099-2,106, controlled 2,343-2,347 vs 2,096-2,103: lanes
//   complex64:    single-qubit 6,607-6,612 vs 6,543-6,645 (a tie): lanes;
//                 controlled 6,077-6,137 vs 6,507-6,613: pair kernel
//   double-float: single-qubit 5,849-5,862 vs 6,284-6,397, controlled 5,291-5,330 vs
//                 6,129-6,248: pair kernel (its four extra shuffles per amplitude cost
//                 issue slots in a kernel bound by the integer pipe)
bool lane_op(const qs_state* s, const Op& op, bool arith_f64) {
    if (s->lane_mode < 0 || s->n < 5 || op.t >= 5) return false;
    if (op.cls == GC_DIAG || op.cls == GC_DIAG1) return false;
    if (!(op.kind == OP_1Q || (op.kind == OP_CU && op.c >= 5))) return false;
    if (s->lane_mode > 0) return true;
    if (s->dt == QS_C128) return arith_f64;
    return op.kind == OP_1Q;
}

qs_status launch_op(qs_state* s, const Op& op, bool arith_f64) {
    cudaError_t e;
    const uint64_t N = 1ull << s->n;
    if (lane_op(s, op, arith_f64)) {
        const bool df = s->dt == QS_C128 && !arith_f64;
        if (op.kind == OP_1Q) {
            e = s->dt == QS_C128 ? dispatch_lanes<double, 0>(s, op.cls, N >> 5, op.t, op.t, op.m, df)
                                 : dispatch_lanes<float, 0>(s, op.cls, N >> 5, op.t, op.t, op.m, false);
        } else {
            e = s->dt == QS_C128 ? dispatch_lanes<double, 1>(s, op.cls, N >> 6, op.t, op.c, op.m, df)
                                 : dispatch_lanes<float, 1>(s, op.cls, N >> 6, op.t, op.c, op.m, false);
        }
        if (e != cudaSuccess) return cuda_fail(e, "gate kernel launch");
        return QS_OK;
    }
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
