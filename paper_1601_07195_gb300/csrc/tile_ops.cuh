// tile_ops.cuh -- in-shared-memory gate updates on a tile of 2^b amplitudes
// (tile bits, not qubits): Eq. 2 pairs for single-qubit gates, Eq. 3 pairs
// with a control tile bit, per-tile factors for diagonal gates whose target is
// not a tile bit, and swaps.  Every branch depends only on the op and on the
// tile's fixed non-tile bits (`base`), so it is uniform over the CTA.
// THREADS is the CTA size that strides the loops.
#pragma once

#include "device.cuh"

namespace qs {

// Two pairs per step (p and p + THREADS), both loaded before either is
// updated, so the two updates are independent instruction chains.
template <class R, int CLS, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void tile_1q(typename Amp<R>::T* sm, uint32_t N, int tb, const R* m) {
    using T = typename Amp<R>::T;
    const uint32_t half = N >> 1;
    for (uint32_t p = threadIdx.x; p < half; p += 2 * THREADS) {
        const uint32_t q = p + THREADS;
        const bool two = q < half;
        const uint32_t i0 = insert_zero32(p, tb), i1 = i0 | (1u << tb);
        const uint32_t j0 = insert_zero32(two ? q : p, tb), j1 = j0 | (1u << tb);
        T a, b, x, y;
        if (CLS != GC_DIAG1) { a = sm[L::at(i0)]; x = sm[L::at(j0)]; }
        b = sm[L::at(i1)];
        y = sm[L::at(j1)];
        pair_update<CLS>(m, a, b);
        pair_update<CLS>(m, x, y);
        if (CLS != GC_DIAG1) sm[L::at(i0)] = a;
        sm[L::at(i1)] = b;
        if (two) {
            if (CLS != GC_DIAG1) sm[L::at(j0)] = x;
            sm[L::at(j1)] = y;
        }
    }
}

template <class R, int CLS, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void tile_cu(typename Amp<R>::T* sm, uint32_t N, int cb, int tb, const R* m) {
    using T = typename Amp<R>::T;
    const int lo = min(cb, tb), hi = max(cb, tb);
    const uint32_t quarter = N >> 2;
    for (uint32_t p = threadIdx.x; p < quarter; p += 2 * THREADS) {
        const uint32_t q = p + THREADS;
        const bool two = q < quarter;
        const uint32_t i0 = insert_two_zeros32(p, lo, hi) | (1u << cb), i1 = i0 | (1u << tb);
        const uint32_t j0 = insert_two_zeros32(two ? q : p, lo, hi) | (1u << cb), j1 = j0 | (1u << tb);
        T a, b, x, y;
        if (CLS != GC_DIAG1) { a = sm[L::at(i0)]; x = sm[L::at(j0)]; }
        b = sm[L::at(i1)];
        y = sm[L::at(j1)];
        pair_update<CLS>(m, a, b);
        pair_update<CLS>(m, x, y);
        if (CLS != GC_DIAG1) sm[L::at(i0)] = a;
        sm[L::at(i1)] = b;
        if (two) {
            if (CLS != GC_DIAG1) sm[L::at(j0)] = x;
            sm[L::at(j1)] = y;
        }
    }
}

// Fixed-size tiles (2^B amplitudes): one per-thread base index per op plus
// offsets uniform over the CTA (insert_zero is additive over the disjoint bits
// of t < THREADS and m * THREADS), fully unrolled.
#ifndef QS_TILE_ILP
#define QS_TILE_ILP 2
#endif
// independent pairs loaded before any is computed, per step of the fixed paths
constexpr int kTileIlp = QS_TILE_ILP;

// Unroll depth of the step loops of the fixed-size paths (each step applies
// STEP independent pairs).  Full unrolling removes the loop's integer work but
// multiplies the code of every gate class; compile with -DQS_TILE_STEP_UNROLL=n to bound it.
#ifndef QS_TILE_STEP_UNROLL
#define QS_TILE_STEP_UNROLL 64  // complex64 n = 30 step: 291 ms fully unrolled, 297 at 2, 302 at 1
#endif

template <class R, int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void tile_1q_fixed(typename Amp<R>::T* sm, int tb, const R* m) {
    using T = typename Amp<R>::T;
    static_assert(THREADS % 32 == 0, "step offsets must leave bits 0..4 alone");
    constexpr int PAIRS = (1 << (B - 1)) / THREADS;
    constexpr int STEP = (PAIRS % kTileIlp == 0) ? kTileIlp : 2;
    const uint32_t e0 = insert_zero32(threadIdx.x, tb), hm = ~0u << tb;
    T* s0 = sm + L::at(e0);
    T* s1 = sm + L::at(e0 | (1u << tb));
QS_UNROLL(QS_TILE_STEP_UNROLL)
    for (int k = 0; k < PAIRS; k += STEP) {
        uint32_t d[STEP];
        T a[STEP], b[STEP];
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            d[u] = insert_zero32_hm((uint32_t)((k + u) * THREADS), hm);
            if (CLS != GC_DIAG1) a[u] = s0[d[u]];
            b[u] = s1[d[u]];
        }
#pragma unroll
        for (int u = 0; u < STEP; ++u) pair_update<CLS>(m, a[u], b[u]);
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            if (CLS != GC_DIAG1) s0[d[u]] = a[u];
            s1[d[u]] = b[u];
        }
    }
}

template <class R, int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void tile_cu_fixed(typename Amp<R>::T* sm, int cb, int tb, const R* m) {
    using T = typename Amp<R>::T;
    static_assert(THREADS % 32 == 0, "step offsets must leave bits 0..4 alone");
    constexpr int ITEMS = (1 << (B - 2)) / THREADS;
    constexpr int STEP = (ITEMS % kTileIlp == 0) ? kTileIlp : 2;
    const int lo = min(cb, tb), hi = max(cb, tb);
    const uint32_t e0 = insert_two_zeros32(threadIdx.x, lo, hi) | (1u << cb);
    const uint32_t hlo = ~0u << lo, hhi = ~0u << hi;
    T* s0 = sm + L::at(e0);
    T* s1 = sm + L::at(e0 | (1u << tb));
QS_UNROLL(QS_TILE_STEP_UNROLL)
    for (int k = 0; k < ITEMS; k += STEP) {
        uint32_t d[STEP];
        T a[STEP], b[STEP];
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            d[u] = insert_zero32_hm(insert_zero32_hm((uint32_t)((k + u) * THREADS), hlo), hhi);
            if (CLS != GC_DIAG1) a[u] = s0[d[u]];
            b[u] = s1[d[u]];
        }
#pragma unroll
        for (int u = 0; u < STEP; ++u) pair_update<CLS>(m, a[u], b[u]);
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            if (CLS != GC_DIAG1) s0[d[u]] = a[u];
            s1[d[u]] = b[u];
        }
    }
}

template <class R, int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void tile_1q_any(typename Amp<R>::T* sm, uint32_t N, int tb, const R* m) {
    if constexpr (B > 0 && (1 << (B - 1)) / THREADS >= 2) tile_1q_fixed<R, CLS, THREADS, B, L>(sm, tb, m);
    else tile_1q<R, CLS, THREADS, L>(sm, N, tb, m);
}
template <class R, int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void tile_cu_any(typename Amp<R>::T* sm, uint32_t N, int cb, int tb, const R* m) {
    if constexpr (B > 0 && (1 << (B - 2)) / THREADS >= 2) tile_cu_fixed<R, CLS, THREADS, B, L>(sm, cb, tb, m);
    else tile_cu<R, CLS, THREADS, L>(sm, N, cb, tb, m);
}

// Multiply the tile (or, with cb >= 0, the half whose tile bit cb is 1) by f.
template <class R, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void tile_scale(typename Amp<R>::T* sm, uint32_t N, R fr, R fi, int cb) {
    if (cb < 0) {
        for (uint32_t e = threadIdx.x; e < N; e += THREADS) sm[L::at(e)] = cmul(fr, fi, sm[L::at(e)]);
    } else {
        for (uint32_t p = threadIdx.x; p < (N >> 1); p += THREADS) {
            const uint32_t e = L::at(insert_zero32(p, cb) | (1u << cb));
            sm[e] = cmul(fr, fi, sm[e]);
        }
    }
}

template <class R, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void tile_swap(typename Amp<R>::T* sm, uint32_t N, int ab, int bb) {
    using T = typename Amp<R>::T;
    const int lo = min(ab, bb), hi = max(ab, bb);
    for (uint32_t p = threadIdx.x; p < (N >> 2); p += THREADS) {
        const uint32_t i = insert_two_zeros32(p, lo, hi);
        const uint32_t ia = L::at(i | (1u << ab)), ib = L::at(i | (1u << bb));
        const T x = sm[ia];
        sm[ia] = sm[ib];
        sm[ib] = x;
    }
}

// B > 0: the tile has exactly 2^B amplitudes (fixed-size paths); B = 0: any size.
template <class R, int THREADS, int B = 0, class L = FlatLayout>
__device__ __forceinline__ void tile_pairs(typename Amp<R>::T* sm, uint32_t N, int cls, int cb, int tb, const R* m) {
    if (cb < 0) {
        switch (cls) {
        case GC_GENERAL: tile_1q_any<R, GC_GENERAL, THREADS, B, L>(sm, N, tb, m); break;
        case GC_REAL: tile_1q_any<R, GC_REAL, THREADS, B, L>(sm, N, tb, m); break;
        case GC_DIAG: tile_1q_any<R, GC_DIAG, THREADS, B, L>(sm, N, tb, m); break;
        case GC_DIAG1: tile_1q_any<R, GC_DIAG1, THREADS, B, L>(sm, N, tb, m); break;
        case GC_ANTIDIAG: tile_1q_any<R, GC_ANTIDIAG, THREADS, B, L>(sm, N, tb, m); break;
        default: tile_1q_any<R, GC_PERM, THREADS, B, L>(sm, N, tb, m); break;
        }
    } else {
        switch (cls) {
        case GC_GENERAL: tile_cu_any<R, GC_GENERAL, THREADS, B, L>(sm, N, cb, tb, m); break;
        case GC_REAL: tile_cu_any<R, GC_REAL, THREADS, B, L>(sm, N, cb, tb, m); break;
        case GC_DIAG: tile_cu_any<R, GC_DIAG, THREADS, B, L>(sm, N, cb, tb, m); break;
        case GC_DIAG1: tile_cu_any<R, GC_DIAG1, THREADS, B, L>(sm, N, cb, tb, m); break;
        case GC_ANTIDIAG: tile_cu_any<R, GC_ANTIDIAG, THREADS, B, L>(sm, N, cb, tb, m); break;
        default: tile_cu_any<R, GC_PERM, THREADS, B, L>(sm, N, cb, tb, m); break;
        }
    }
}

// Apply one op to the tile whose non-tile qubits are fixed by `base`.  Every
// branch depends only on the op and on base, so it is uniform over the CTA.
// Returns false when the op leaves this tile unchanged (no barrier needed).
// ---- fused phase runs (record layout in qs_internal.h) ------------------------
template <class T, class R>
__device__ __forceinline__ T slot_value(const TileOp<R>& r, int f) {
    T v;
    v.x = r.m[2 * f];
    v.y = r.m[2 * f + 1];
    return v;
}
template <class R>
__device__ __forceinline__ int slot_qubit(const TileOp<R>& r, int f) {
    return f == 0 ? r.tb : f == 1 ? r.tq : f == 2 ? r.cb : r.cq;
}
template <class T>
__device__ __forceinline__ T cmul_v(T q, T a) {
    return cmul(q.x, q.y, a);
}

// The run whose header is record g; steps and barriers as in df_phase_run
// (tile_df_ops.cuh): tables T_lo and T_hi and the per-tile constant C, then
// T_lo *= C, then every amplitude with bit jb = 1 times T_lo * T_hi.  The
// tables live in `tab`, 16 bytes per entry whatever the amplitude type.
template <class R, int THREADS, int B, class L, class OpAt>
__device__ __forceinline__ void phase_run(typename Amp<R>::T* sm, void* tab_raw, uint32_t N, int b,
                                          const TileOp<R>& h, OpAt op_at, int g, uint64_t base) {
    using T = typename Amp<R>::T;
    const int jb = h.tb, n_out = h.cb, lob = h.cq, hib = b - lob;
    const int tile_rec = (b + 3) >> 2;
    const uint32_t nlo = 1u << lob, nhi = 1u << hib;
    T* tlo = reinterpret_cast<T*>(tab_raw);
    T* thi = tlo + nlo;
    T* tc = tlo + nlo + nhi;
    const uint32_t t = threadIdx.x;
    T one;
    one.x = (R)1;
    one.y = (R)0;
    if (t < nlo) {
        T v = one;
        for (int k = 0; k < lob; ++k)
            if ((t >> k) & 1u) v = cmul_v(slot_value<T>(op_at(g + 1 + (k >> 2)), k & 3), v);
        tlo[t] = v;
    } else if (t < nlo + nhi) {
        const uint32_t u = t - nlo;
        T v = one;
        for (int k = 0; k < hib; ++k)
            if ((u >> k) & 1u) v = cmul_v(slot_value<T>(op_at(g + 1 + ((lob + k) >> 2)), (lob + k) & 3), v);
        thi[u] = v;
    }
    if (t >= THREADS - 32) {
        const int lane = (int)(t & 31u);
        T v = one;
        for (int i = lane; i < n_out; i += 32) {
            const TileOp<R>& r = op_at(g + 1 + tile_rec + (i >> 2));
            if ((base >> slot_qubit(r, i & 3)) & 1ull) v = cmul_v(slot_value<T>(r, i & 3), v);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            T o;
            o.x = __shfl_xor_sync(0xffffffffu, v.x, off);
            o.y = __shfl_xor_sync(0xffffffffu, v.y, off);
            v = cmul_v(o, v);
        }
        if (lane == 0) *tc = cmul_v(slot_value<T>(h, 0), v);
    }
    __syncthreads();
    if (t < nlo) tlo[t] = cmul_v(*tc, tlo[t]);
    __syncthreads();
    const uint32_t lmask = nlo - 1u;
    if constexpr (B > 0 && (1 << (B - 1)) / THREADS >= 1) {
        constexpr int ITEMS = (1 << (B - 1)) / THREADS;
        const uint32_t e0 = insert_zero32(t, jb) | (1u << jb), s0 = L::at(e0), hm = ~0u << jb;
#pragma unroll
        for (int m = 0; m < ITEMS; ++m) {
            const uint32_t d = insert_zero32_hm((uint32_t)(m * THREADS), hm);
            const uint32_t e = e0 + d;  // tables by tile index, the amplitude by its SMEM place
            sm[s0 + d] = cmul_v(cmul_v(tlo[e & lmask], thi[e >> lob]), sm[s0 + d]);
        }
    } else {
        for (uint32_t p = t; p < (N >> 1); p += THREADS) {
            const uint32_t e = insert_zero32(p, jb) | (1u << jb), se = L::at(e);
            sm[se] = cmul_v(cmul_v(tlo[e & lmask], thi[e >> lob]), sm[se]);
        }
    }
}

// Applies the diagonal run whose header is record g; steps and barriers as in
// df_diag_run (tile_df_ops.cuh): per-bit factors psi_k and the per-tile C, then
// T_lo (times C) and T_hi with the pair terms of each half, then every
// amplitude times T_lo * T_hi.  The tables live in `tab`, 16 bytes per entry.
template <class R, int THREADS, int B, class L, class OpAt>
__device__ __forceinline__ void diag_run(typename Amp<R>::T* sm, void* tab_raw, uint32_t N, int b,
                                         const TileOp<R>& h, OpAt op_at, int g, uint64_t base) {
    using T = typename Amp<R>::T;
    const int n_terms = h.tb, lob = h.cq, hib = b - lob;
    const uint32_t nlo = 1u << lob, nhi = 1u << hib;
    T* tlo = reinterpret_cast<T*>(tab_raw);
    T* thi = tlo + nlo;
    T* tc = tlo + nlo + nhi;
    T* psi = tc + 1;
    const uint32_t t = threadIdx.x;
    T one;
    one.x = (R)1;
    one.y = (R)0;
    auto term = [&](int i, int& type, int& x, int& y) -> T {
        const TileOp<R>& r = op_at(g + 1 + (i >> 2));
        const int f = i & 3;
        const int code = slot_qubit(r, f);
        type = code >> 16;
        x = (code >> 8) & 255;
        y = code & 255;
        return slot_value<T>(r, f);
    };
    auto holds = [&](int q) { return q == kDrunNone || ((base >> q) & 1ull) != 0; };
    if ((int)t < b) {
        T v = one;
        for (int i = 0; i < n_terms; ++i) {
            int type, x, y;
            const T f = term(i, type, x, y);
            if (type == kDrunBit && x == (int)t && holds(y)) v = cmul_v(f, v);
        }
        psi[t] = v;
    } else if (t == THREADS - 1) {
        T v = one;
        for (int i = 0; i < n_terms; ++i) {
            int type, x, y;
            const T f = term(i, type, x, y);
            if (type == kDrunScalar && holds(x) && holds(y)) v = cmul_v(f, v);
        }
        *tc = v;
    }
    __syncthreads();
    if (t < nlo + nhi) {
        const bool low = t < nlo;
        const uint32_t u = low ? t : t - nlo;
        const int k0 = low ? 0 : lob, nb = low ? lob : hib;
        T v = low ? *tc : one;
        for (int k = 0; k < nb; ++k)
            if ((u >> k) & 1u) v = cmul_v(psi[k0 + k], v);
        for (int i = 0; i < n_terms; ++i) {
            int type, x, y;
            const T f = term(i, type, x, y);
            if (type == kDrunPair && x >= k0 && x < k0 + nb && ((u >> (x - k0)) & 1u) && ((u >> (y - k0)) & 1u))
                v = cmul_v(f, v);
        }
        if (low) tlo[u] = v;
        else thi[u] = v;
    }
    __syncthreads();
    const uint32_t lmask = nlo - 1u;
    if constexpr (B > 0 && (1 << B) >= THREADS) {
        constexpr int PER = (1 << B) / THREADS;
#pragma unroll 4
        for (int m = 0; m < PER; ++m) {
            const uint32_t e = t + (uint32_t)(m * THREADS), se = L::at(e);
            sm[se] = cmul_v(cmul_v(tlo[e & lmask], thi[e >> lob]), sm[se]);
        }
    } else {
        for (uint32_t e = t; e < N; e += THREADS) {
            const uint32_t se = L::at(e);
            sm[se] = cmul_v(cmul_v(tlo[e & lmask], thi[e >> lob]), sm[se]);
        }
    }
}

template <class R, int THREADS, int B = 0, class L = FlatLayout>
__device__ __forceinline__ bool tile_apply(typename Amp<R>::T* sm, uint32_t N, const TileOp<R>& op, uint64_t base) {
    if (op.kind == OP_SWAP) {
        tile_swap<R, THREADS, L>(sm, N, op.tb, op.cb);
        return true;
    }
    int cb = -1;
    if (op.kind == OP_CU) {
        if (op.cb < 0) {
            if (((base >> op.cq) & 1ull) == 0) return false;  // control outside the tile is 0 here
        } else {
            cb = op.cb;
        }
    }
    if (op.tb < 0) {  // diagonal gate whose target is not a tile bit: one factor for the (half-)tile
        const bool bit = (base >> op.tq) & 1ull;
        if (op.cls == GC_DIAG1 && !bit) return false;
        tile_scale<R, THREADS, L>(sm, N, bit ? op.m[6] : op.m[0], bit ? op.m[7] : op.m[1], cb);
        return true;
    }
    tile_pairs<R, THREADS, B, L>(sm, N, op.cls, cb, op.tb, op.m);
    return true;
}

}  // namespace qs
