// tile_df_ops.cuh -- shared-memory gate updates on a tile held as double-float
// pairs (float4 = re.hi, re.lo, im.hi, im.lo; see df.cuh).  Same contract as
// tile_ops.cuh: tile bits, per-tile factors for diagonal gates whose target
// is not a tile bit, per-tile predicates for controls outside the tile.
#pragma once

#include "device.cuh"
#include "df.cuh"

namespace qs {

template <int CLS>
__device__ __forceinline__ void df_pair_update(const float* c, float4& a, float4& b) {
    if constexpr (CLS == GC_GENERAL) {
        const float4 a2 = df_cmul2(c, 0, 1, a, 2, 3, b);
        const float4 b2 = df_cmul2(c, 4, 5, a, 6, 7, b);
        a = a2; b = b2;
    } else if constexpr (CLS == GC_REAL) {
        const float4 a2 = df_rmul2(c, 0, a, 2, b);
        const float4 b2 = df_rmul2(c, 4, a, 6, b);
        a = a2; b = b2;
    } else if constexpr (CLS == GC_REAL_BAL) {  // signs in the unused imaginary slots c[2], c[10]
        const float4 a2 = df_bal(c, 0, c[2], a, b);
        const float4 b2 = df_bal(c, 4, c[10], a, b);
        a = a2; b = b2;
    } else if constexpr (CLS == GC_REAL_BAL1) {  // signs in c[2], c[10], c[8]
        const dfl ar = df_addsig(a.x, a.y, c[2], b.x, b.y), ai = df_addsig(a.z, a.w, c[2], b.z, b.w);
        const dfl br = df_addsig(a.x, a.y, c[10], b.x, b.y), bi = df_addsig(a.z, a.w, c[10], b.z, b.w);
        const float r = c[8];
        a = make_float4(ar.h, ar.l, ai.h, ai.l);
        b = make_float4(r * br.h, r * br.l, r * bi.h, r * bi.l);
    } else if constexpr (CLS == GC_PRP || CLS == GC_PRP_NZ) {
        df_prp<CLS == GC_PRP>(c, a, b);
    } else if constexpr (CLS == GC_PRP_X || CLS == GC_PRP_X_NZ) {
        df_prp<CLS == GC_PRP_X>(c, b, a);  // U = U' X: the pair enters swapped, U' = PRP
        const float4 t = a; a = b; b = t;
    } else if constexpr (CLS == GC_DIAG) {
        a = df_cmul(c, 0, 1, a);
        b = df_cmul(c, 6, 7, b);
    } else if constexpr (CLS == GC_DIAG1) {
        b = df_cmul(c, 6, 7, b);
    } else if constexpr (CLS == GC_ANTIDIAG) {
        const float4 a2 = df_cmul(c, 2, 3, b);
        const float4 b2 = df_cmul(c, 4, 5, a);
        a = a2; b = b2;
    } else {
        const float4 t = a; a = b; b = t;
    }
}

// Each thread takes two pairs per step (p and p + THREADS), loads both before
// computing: the two double-float updates are independent chains the
// scheduler can interleave.  GUARD is needed only when the pair count is not
// a multiple of 2 * THREADS (tiles smaller than 4 * THREADS amplitudes).
template <int CLS, int THREADS, bool GUARD, class L = FlatLayout>
__device__ __forceinline__ void df_tile_1q_body(float4* sm, uint32_t half, int tb, const float* c) {
    for (uint32_t p = threadIdx.x; p < half; p += 2 * THREADS) {
        const uint32_t q = p + THREADS;
        const bool two = !GUARD || q < half;
        const uint32_t i0 = insert_zero32(p, tb), i1 = i0 | (1u << tb);
        const uint32_t j0 = insert_zero32(two ? q : p, tb), j1 = j0 | (1u << tb);
        float4 a, b, x, y;
        if (CLS != GC_DIAG1) { a = sm[L::at(i0)]; x = sm[L::at(j0)]; }
        b = sm[L::at(i1)];
        y = sm[L::at(j1)];
        df_pair_update<CLS>(c, a, b);
        df_pair_update<CLS>(c, x, y);
        if (CLS != GC_DIAG1) sm[L::at(i0)] = a;
        sm[L::at(i1)] = b;
        if (two) {
            if (CLS != GC_DIAG1) sm[L::at(j0)] = x;
            sm[L::at(j1)] = y;
        }
    }
}

// Tiles of exactly 2^B amplitudes with 2^(B-1) >= 2 * THREADS: thread t's
// pairs are p = t + m * THREADS, and since t < THREADS and m * THREADS share no
// bit, insert_zero(p) = insert_zero(t) + insert_zero(m * THREADS).  One
// per-thread base index per op plus per-step offsets that are uniform over the
// CTA (compile-time m, per-op tb) leave almost no integer work per pair, and
// the fully unrolled steps expose independent pairs to the scheduler.
#ifndef QS_DF_ILP
#define QS_DF_ILP 2
#endif
// independent pairs loaded before any is computed, per step of the fixed paths
constexpr int kDfIlp = QS_DF_ILP;

// Unroll depth of the step loops of the fixed-size paths (each step applies
// STEP independent pairs).  Full unrolling removes the loop's integer work but
// multiplies the code of every gate class; compile with -DQS_DF_STEP_UNROLL=n to bound it.
#ifndef QS_DF_STEP_UNROLL
#define QS_DF_STEP_UNROLL 2  // n = 30 step: 771 ms at 2, 773 at 1, 794 fully unrolled (instruction-cache misses)
#endif

template <int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void df_tile_1q_fixed(float4* sm, int tb, const float* c) {
    constexpr int PAIRS = (1 << (B - 1)) / THREADS;
    static_assert(PAIRS >= 2 && PAIRS % 2 == 0, "tile too small for the fixed path");
    static_assert(THREADS % 32 == 0, "step offsets must leave bits 0..4 alone");
    constexpr int STEP = (PAIRS % kDfIlp == 0) ? kDfIlp : 2;
    const uint32_t e0 = insert_zero32(threadIdx.x, tb), hm = ~0u << tb;
    float4* s0 = sm + L::at(e0);
    float4* s1 = sm + L::at(e0 | (1u << tb));
QS_UNROLL(QS_DF_STEP_UNROLL)
    for (int m = 0; m < PAIRS; m += STEP) {
        uint32_t d[STEP];
        float4 a[STEP], b[STEP];
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            d[u] = insert_zero32_hm((uint32_t)((m + u) * THREADS), hm);
            if (CLS != GC_DIAG1) a[u] = s0[d[u]];
            b[u] = s1[d[u]];
        }
#pragma unroll
        for (int u = 0; u < STEP; ++u) df_pair_update<CLS>(c, a[u], b[u]);
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            if (CLS != GC_DIAG1) s0[d[u]] = a[u];
            s1[d[u]] = b[u];
        }
    }
}

template <int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void df_tile_cu_fixed(float4* sm, int cb, int tb, const float* c) {
    constexpr int ITEMS = (1 << (B - 2)) / THREADS;
    static_assert(ITEMS >= 2 && ITEMS % 2 == 0, "tile too small for the fixed path");
    static_assert(THREADS % 32 == 0, "step offsets must leave bits 0..4 alone");
    constexpr int STEP = (ITEMS % kDfIlp == 0) ? kDfIlp : 2;
    const int lo = min(cb, tb), hi = max(cb, tb);
    const uint32_t e0 = insert_two_zeros32(threadIdx.x, lo, hi) | (1u << cb);
    const uint32_t hlo = ~0u << lo, hhi = ~0u << hi;
    float4* s0 = sm + L::at(e0);
    float4* s1 = sm + L::at(e0 | (1u << tb));
QS_UNROLL(QS_DF_STEP_UNROLL)
    for (int m = 0; m < ITEMS; m += STEP) {
        uint32_t d[STEP];
        float4 a[STEP], b[STEP];
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            d[u] = insert_zero32_hm(insert_zero32_hm((uint32_t)((m + u) * THREADS), hlo), hhi);
            if (CLS != GC_DIAG1) a[u] = s0[d[u]];
            b[u] = s1[d[u]];
        }
#pragma unroll
        for (int u = 0; u < STEP; ++u) df_pair_update<CLS>(c, a[u], b[u]);
#pragma unroll
        for (int u = 0; u < STEP; ++u) {
            if (CLS != GC_DIAG1) s0[d[u]] = a[u];
            s1[d[u]] = b[u];
        }
    }
}

template <int CLS, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void df_tile_1q(float4* sm, uint32_t N, int tb, const float* c) {
    const uint32_t half = N >> 1;
    if ((half & (2 * THREADS - 1)) == 0) df_tile_1q_body<CLS, THREADS, false, L>(sm, half, tb, c);
    else df_tile_1q_body<CLS, THREADS, true, L>(sm, half, tb, c);
}

template <int CLS, int THREADS, bool GUARD, class L = FlatLayout>
__device__ __forceinline__ void df_tile_cu_body(float4* sm, uint32_t quarter, int cb, int tb, const float* c) {
    const int lo = min(cb, tb), hi = max(cb, tb);
    for (uint32_t p = threadIdx.x; p < quarter; p += 2 * THREADS) {
        const uint32_t q = p + THREADS;
        const bool two = !GUARD || q < quarter;
        const uint32_t i0 = insert_two_zeros32(p, lo, hi) | (1u << cb), i1 = i0 | (1u << tb);
        const uint32_t j0 = insert_two_zeros32(two ? q : p, lo, hi) | (1u << cb), j1 = j0 | (1u << tb);
        float4 a, b, x, y;
        if (CLS != GC_DIAG1) { a = sm[L::at(i0)]; x = sm[L::at(j0)]; }
        b = sm[L::at(i1)];
        y = sm[L::at(j1)];
        df_pair_update<CLS>(c, a, b);
        df_pair_update<CLS>(c, x, y);
        if (CLS != GC_DIAG1) sm[L::at(i0)] = a;
        sm[L::at(i1)] = b;
        if (two) {
            if (CLS != GC_DIAG1) sm[L::at(j0)] = x;
            sm[L::at(j1)] = y;
        }
    }
}

template <int CLS, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void df_tile_cu(float4* sm, uint32_t N, int cb, int tb, const float* c) {
    const uint32_t quarter = N >> 2;
    if ((quarter & (2 * THREADS - 1)) == 0) df_tile_cu_body<CLS, THREADS, false, L>(sm, quarter, cb, tb, c);
    else df_tile_cu_body<CLS, THREADS, true, L>(sm, quarter, cb, tb, c);
}

template <bool USE22, int THREADS, class L = FlatLayout>
__device__ __forceinline__ void df_tile_scale(float4* sm, uint32_t N, const float* c, int cb) {
    if (cb < 0) {
#pragma unroll 2
        for (uint32_t e = threadIdx.x; e < N; e += THREADS) {
            const uint32_t se = L::at(e);
            sm[se] = USE22 ? df_cmul(c, 6, 7, sm[se]) : df_cmul(c, 0, 1, sm[se]);
        }
    } else {
#pragma unroll 2
        for (uint32_t p = threadIdx.x; p < (N >> 1); p += THREADS) {
            const uint32_t e = L::at(insert_zero32(p, cb) | (1u << cb));
            sm[e] = USE22 ? df_cmul(c, 6, 7, sm[e]) : df_cmul(c, 0, 1, sm[e]);
        }
    }
}

template <int THREADS, class L = FlatLayout>
__device__ __forceinline__ void df_tile_swap(float4* sm, uint32_t N, int ab, int bb) {
    const int lo = min(ab, bb), hi = max(ab, bb);
    for (uint32_t p = threadIdx.x; p < (N >> 2); p += THREADS) {
        const uint32_t i = insert_two_zeros32(p, lo, hi);
        const uint32_t ia = L::at(i | (1u << ab)), ib = L::at(i | (1u << bb));
        const float4 x = sm[ia];
        sm[ia] = sm[ib];
        sm[ib] = x;
    }
}

template <int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void df_tile_1q_any(float4* sm, uint32_t N, int tb, const float* c) {
    if constexpr (B > 0 && (1 << (B - 1)) / THREADS >= 2) df_tile_1q_fixed<CLS, THREADS, B, L>(sm, tb, c);
    else df_tile_1q<CLS, THREADS, L>(sm, N, tb, c);
}
template <int CLS, int THREADS, int B, class L = FlatLayout>
__device__ __forceinline__ void df_tile_cu_any(float4* sm, uint32_t N, int cb, int tb, const float* c) {
    if constexpr (B > 0 && (1 << (B - 2)) / THREADS >= 2) df_tile_cu_fixed<CLS, THREADS, B, L>(sm, cb, tb, c);
    else df_tile_cu<CLS, THREADS, L>(sm, N, cb, tb, c);
}

// B > 0: the tile has exactly 2^B amplitudes (fixed-size paths); B = 0: any size.
template <int THREADS, int B = 0, class L = FlatLayout>
__device__ __forceinline__ void df_tile_pairs(float4* sm, uint32_t N, int cls, int cb, int tb, const float* c) {
    if (cb < 0) {
        switch (cls) {
        case GC_GENERAL: df_tile_1q_any<GC_GENERAL, THREADS, B, L>(sm, N, tb, c); break;
        case GC_REAL: df_tile_1q_any<GC_REAL, THREADS, B, L>(sm, N, tb, c); break;
        case GC_REAL_BAL: df_tile_1q_any<GC_REAL_BAL, THREADS, B, L>(sm, N, tb, c); break;
        case GC_REAL_BAL1: df_tile_1q_any<GC_REAL_BAL1, THREADS, B, L>(sm, N, tb, c); break;
        case GC_PRP: df_tile_1q_any<GC_PRP, THREADS, B, L>(sm, N, tb, c); break;
        case GC_PRP_X: df_tile_1q_any<GC_PRP_X, THREADS, B, L>(sm, N, tb, c); break;
        case GC_PRP_NZ: df_tile_1q_any<GC_PRP_NZ, THREADS, B, L>(sm, N, tb, c); break;
        case GC_PRP_X_NZ: df_tile_1q_any<GC_PRP_X_NZ, THREADS, B, L>(sm, N, tb, c); break;
        case GC_DIAG: df_tile_1q_any<GC_DIAG, THREADS, B, L>(sm, N, tb, c); break;
        case GC_DIAG1: df_tile_1q_any<GC_DIAG1, THREADS, B, L>(sm, N, tb, c); break;
        case GC_ANTIDIAG: df_tile_1q_any<GC_ANTIDIAG, THREADS, B, L>(sm, N, tb, c); break;
        default: df_tile_1q_any<GC_PERM, THREADS, B, L>(sm, N, tb, c); break;
        }
    } else {
        switch (cls) {
        case GC_GENERAL: df_tile_cu_any<GC_GENERAL, THREADS, B, L>(sm, N, cb, tb, c); break;
        case GC_REAL: df_tile_cu_any<GC_REAL, THREADS, B, L>(sm, N, cb, tb, c); break;
        case GC_REAL_BAL: df_tile_cu_any<GC_REAL_BAL, THREADS, B, L>(sm, N, cb, tb, c); break;
        case GC_DIAG: df_tile_cu_any<GC_DIAG, THREADS, B, L>(sm, N, cb, tb, c); break;
        case GC_DIAG1: df_tile_cu_any<GC_DIAG1, THREADS, B, L>(sm, N, cb, tb, c); break;
        case GC_ANTIDIAG: df_tile_cu_any<GC_ANTIDIAG, THREADS, B, L>(sm, N, cb, tb, c); break;
        default: df_tile_cu_any<GC_PERM, THREADS, B, L>(sm, N, cb, tb, c); break;
        }
    }
}

// ---- fused phase runs (record layout in qs_internal.h) ------------------------

// q * x for two complex DF values
__device__ __forceinline__ float4 df_cmul_v(float4 q, float4 x) {
    const dfl re = df_dot2(df_mul(q.x, q.y, x.x, x.y), df_mul(-q.z, -q.w, x.z, x.w));
    const dfl im = df_dot2(df_mul(q.x, q.y, x.z, x.w), df_mul(q.z, q.w, x.x, x.y));
    return make_float4(re.h, re.l, im.h, im.l);
}
__device__ __forceinline__ float4 df_slot(const TileOpDF& r, int f) {
    return make_float4(r.c[4 * f], r.c[4 * f + 1], r.c[4 * f + 2], r.c[4 * f + 3]);
}
__device__ __forceinline__ int slot_qubit(const TileOpDF& r, int f) {
    return f == 0 ? r.tb : f == 1 ? r.tq : f == 2 ? r.cb : r.cq;
}

// Applies the run whose header is record g.  Three steps, each ended by a
// barrier (the caller's barrier ends the last):
//   1. threads [0, 2^lob) form T_lo without C, the next 2^hib threads T_hi;
//      the last warp forms C (a butterfly product of its lanes' outside
//      factors, taken from lane 0);
//   2. T_lo *= C;
//   3. every amplitude with bit jb = 1 is multiplied by T_lo * T_hi.
template <int THREADS, int B, class L, class OpAt>
__device__ __forceinline__ void df_phase_run(float4* sm, float4* tab, uint32_t N, int b, const TileOpDF& h,
                                             OpAt op_at, int g, uint64_t base) {
    const int jb = h.tb, n_out = h.cb, lob = h.cq, hib = b - lob;
    const int tile_rec = (b + 3) >> 2;
    const uint32_t nlo = 1u << lob, nhi = 1u << hib;
    float4* tlo = tab;
    float4* thi = tab + nlo;
    float4* tc = tab + nlo + nhi;
    const uint32_t t = threadIdx.x;
    const float4 one = make_float4(1.f, 0.f, 0.f, 0.f);
    if (t < nlo) {
        float4 v = one;
        for (int k = 0; k < lob; ++k)
            if ((t >> k) & 1u) v = df_cmul_v(df_slot(op_at(g + 1 + (k >> 2)), k & 3), v);
        tlo[t] = v;
    } else if (t < nlo + nhi) {
        const uint32_t u = t - nlo;
        float4 v = one;
        for (int k = 0; k < hib; ++k)
            if ((u >> k) & 1u) v = df_cmul_v(df_slot(op_at(g + 1 + ((lob + k) >> 2)), (lob + k) & 3), v);
        thi[u] = v;
    }
    if (t >= THREADS - 32) {
        const int lane = (int)(t & 31u);
        float4 v = one;
        for (int i = lane; i < n_out; i += 32) {
            const TileOpDF& r = op_at(g + 1 + tile_rec + (i >> 2));
            if ((base >> slot_qubit(r, i & 3)) & 1ull) v = df_cmul_v(df_slot(r, i & 3), v);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            float4 o;
            o.x = __shfl_xor_sync(0xffffffffu, v.x, off);
            o.y = __shfl_xor_sync(0xffffffffu, v.y, off);
            o.z = __shfl_xor_sync(0xffffffffu, v.z, off);
            o.w = __shfl_xor_sync(0xffffffffu, v.w, off);
            v = df_cmul_v(o, v);
        }
        if (lane == 0) *tc = df_cmul_v(df_slot(h, 0), v);
    }
    __syncthreads();
    if (t < nlo) tlo[t] = df_cmul_v(*tc, tlo[t]);
    __syncthreads();
    const uint32_t lmask = nlo - 1u;
    if constexpr (B > 0 && (1 << (B - 1)) / THREADS >= 1) {
        constexpr int ITEMS = (1 << (B - 1)) / THREADS;
        const uint32_t e0 = insert_zero32(t, jb) | (1u << jb), s0 = L::at(e0), hm = ~0u << jb;
#pragma unroll
        for (int m = 0; m < ITEMS; ++m) {
            const uint32_t d = insert_zero32_hm((uint32_t)(m * THREADS), hm);
            const uint32_t e = e0 + d;  // tables by tile index, the amplitude by its SMEM place
            sm[s0 + d] = df_cmul_v(df_cmul_v(tlo[e & lmask], thi[e >> lob]), sm[s0 + d]);
        }
    } else {
        for (uint32_t p = t; p < (N >> 1); p += THREADS) {
            const uint32_t e = insert_zero32(p, jb) | (1u << jb), se = L::at(e);
            sm[se] = df_cmul_v(df_cmul_v(tlo[e & lmask], thi[e >> lob]), sm[se]);
        }
    }
}

// Term i of the diagonal run whose header is record g: its factor, and its
// type and indices from the int field of its slot (qs_internal.h).
template <class OpAt>
__device__ __forceinline__ float4 df_drun_term(OpAt op_at, int g, int i, int& type, int& x, int& y) {
    const TileOpDF& r = op_at(g + 1 + (i >> 2));
    const int f = i & 3;
    const int code = slot_qubit(r, f);
    type = code >> 16;
    x = (code >> 8) & 255;
    y = code & 255;
    return df_slot(r, f);
}

// Applies the diagonal run whose header is record g.  Three steps, each ended
// by a barrier (the caller's barrier ends the last):
//   1. thread k < b forms psi_k from the bit terms of tile bit k whose outside
//      condition holds for this tile; the last thread forms C from the scalar terms;
//   2. threads [0, 2^lob) form T_lo (times C), the next 2^hib threads T_hi, each
//      with the pair terms of its half;
//   3. every amplitude is multiplied by T_lo[e & (2^lob - 1)] * T_hi[e >> lob].
template <int THREADS, int B, class L, class OpAt>
__device__ __forceinline__ void df_diag_run(float4* sm, float4* tab, uint32_t N, int b, const TileOpDF& h,
                                            OpAt op_at, int g, uint64_t base) {
    const int n_terms = h.tb, lob = h.cq, hib = b - lob;
    const uint32_t nlo = 1u << lob, nhi = 1u << hib;
    float4* tlo = tab;
    float4* thi = tab + nlo;
    float4* tc = tab + nlo + nhi;
    float4* psi = tc + 1;
    const uint32_t t = threadIdx.x;
    const float4 one = make_float4(1.f, 0.f, 0.f, 0.f);
    auto holds = [&](int q) { return q == kDrunNone || ((base >> q) & 1ull) != 0; };
    if ((int)t < b) {
        float4 v = one;
        for (int i = 0; i < n_terms; ++i) {
            int type, x, y;
            const float4 f = df_drun_term(op_at, g, i, type, x, y);
            if (type == kDrunBit && x == (int)t && holds(y)) v = df_cmul_v(f, v);
        }
        psi[t] = v;
    } else if (t == THREADS - 1) {
        float4 v = one;
        for (int i = 0; i < n_terms; ++i) {
            int type, x, y;
            const float4 f = df_drun_term(op_at, g, i, type, x, y);
            if (type == kDrunScalar && holds(x) && holds(y)) v = df_cmul_v(f, v);
        }
        *tc = v;
    }
    __syncthreads();
    if (t < nlo + nhi) {
        const bool low = t < nlo;
        const uint32_t u = low ? t : t - nlo;
        const int k0 = low ? 0 : lob, nb = low ? lob : hib;
        float4 v = low ? *tc : one;
        for (int k = 0; k < nb; ++k)
            if ((u >> k) & 1u) v = df_cmul_v(psi[k0 + k], v);
        for (int i = 0; i < n_terms; ++i) {
            int type, x, y;
            const float4 f = df_drun_term(op_at, g, i, type, x, y);
            if (type == kDrunPair && x >= k0 && x < k0 + nb && ((u >> (x - k0)) & 1u) && ((u >> (y - k0)) & 1u))
                v = df_cmul_v(f, v);
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
            sm[se] = df_cmul_v(df_cmul_v(tlo[e & lmask], thi[e >> lob]), sm[se]);
        }
    } else {
        for (uint32_t e = t; e < N; e += THREADS) {
            const uint32_t se = L::at(e);
            sm[se] = df_cmul_v(df_cmul_v(tlo[e & lmask], thi[e >> lob]), sm[se]);
        }
    }
}

template <int THREADS, int B = 0, class L = FlatLayout>
__device__ __forceinline__ bool df_tile_apply(float4* sm, uint32_t N, const TileOpDF& op, uint64_t base) {
    if (op.kind == OP_SWAP) {
        df_tile_swap<THREADS, L>(sm, N, op.tb, op.cb);
        return true;
    }
    int cb = -1;
    if (op.kind == OP_CU) {
        if (op.cb < 0) {
            if (((base >> op.cq) & 1ull) == 0) return false;
        } else {
            cb = op.cb;
        }
    }
    if (op.tb < 0) {
        const bool bit = (base >> op.tq) & 1ull;
        if (op.cls == GC_DIAG1 && !bit) return false;
        if (bit) df_tile_scale<true, THREADS, L>(sm, N, op.c, cb);
        else df_tile_scale<false, THREADS, L>(sm, N, op.c, cb);
        return true;
    }
    df_tile_pairs<THREADS, B, L>(sm, N, op.cls, cb, op.tb, op.c);
    return true;
}

}  // namespace qs
