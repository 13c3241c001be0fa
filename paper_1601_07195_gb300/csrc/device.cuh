// device.cuh -- device-side building blocks shared by the gate, tile and
// reduction kernels: amplitude types, index insertion, and the 2x2 update of
// Eq. 2 specialised by gate class.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_internal.h"

#define QS_PRAGMA(x) _Pragma(#x)
#define QS_UNROLL(n) QS_PRAGMA(unroll n)

namespace qs {

template <class R> struct Amp;
template <> struct Amp<double> { using T = double2; };
template <> struct Amp<float> { using T = float2; };

// 2x2 matrix (q11, q12, q21, q22) as (re, im), passed to kernels by value.
template <class R> struct Mat2 { R v[8]; };

// Insert a zero bit at position k of p: the index of the |0>-member of pair p
// for a gate on qubit k (the pair partner is 2^k above, Section 2).
__device__ __forceinline__ uint64_t insert_zero(uint64_t p, int k) {
    const uint64_t lo = p & ((1ull << k) - 1ull);
    return ((p >> k) << (k + 1)) | lo;
}
// Insert zero bits at positions lo < hi.
__device__ __forceinline__ uint64_t insert_two_zeros(uint64_t p, int lo, int hi) {
    return insert_zero(insert_zero(p, lo), hi);
}
__device__ __forceinline__ uint32_t insert_zero32(uint32_t p, int k) {
    const uint32_t lo = p & ((1u << k) - 1u);
    return ((p >> k) << (k + 1)) | lo;
}
__device__ __forceinline__ uint32_t insert_two_zeros32(uint32_t p, int lo, int hi) {
    return insert_zero32(insert_zero32(p, lo), hi);
}
// The same with the mask of the bits at and above k precomputed (hm = ~0u << k):
// moving those bits up by one is adding them once more, p + (p & hm).  Two
// integer instructions per index where p is a compile-time offset.
__device__ __forceinline__ uint32_t insert_zero32_hm(uint32_t p, uint32_t hm) { return p + (p & hm); }
__device__ __forceinline__ uint64_t insert_zero_hm(uint64_t p, uint64_t hm) { return p + (p & hm); }

// Deposit the low bits of v into the set bits of mask (software pdep).
__device__ __forceinline__ uint64_t deposit_bits(uint64_t v, uint64_t mask) {
    uint64_t out = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1ull);
        if (v & 1ull) out |= low;
        v >>= 1;
        mask ^= low;
    }
    return out;
}

// Shared-memory layout of a tile: amplitude e of the tile sits at L::at(e).
struct FlatLayout {
    static __device__ __forceinline__ uint32_t at(uint32_t e) { return e; }
};
// complex64 tiles (8-byte amplitudes, 32 four-byte banks): the partners of a
// gate on tile bit t <= 3 are 1..8 elements apart, so a warp's 32 lanes would
// hit half of the banks and a 64-bit access would take four wavefronts instead
// of two.  Storing amplitude e at e ^ (15 * bit4(e)) spreads them over all
// banks (every single-qubit gate and most controlled ones back to two).  The
// per-step offsets of the fixed-size loops (multiples of the CTA size with
// zeros inserted) leave bits 0..4 alone, so there L::at(base + d) =
// L::at(base) + d and the swizzle costs nothing per access.
struct SwizzledLayout {
    static __device__ __forceinline__ uint32_t at(uint32_t e) { return e ^ ((0u - ((e >> 4) & 1u)) & 15u); }
};
// The same for 16-byte amplitudes (complex128 as float pairs or doubles): the
// bank period is 8 amplitudes, and e ^ (7 * bit3(e)) spreads the partners of
// gates on tile bits 0..2; the fixed-size loops' offsets leave bits 0..3 alone.
struct Swizzled16Layout {
    static __device__ __forceinline__ uint32_t at(uint32_t e) { return e ^ ((0u - ((e >> 3) & 1u)) & 7u); }
};

// ---- complex products, written as FMA chains --------------------------------
// q * a with q = (qr, qi)
template <class T, class R>
__device__ __forceinline__ T cmul(R qr, R qi, T a) {
    T o;
    o.x = fma(-qi, a.y, qr * a.x);
    o.y = fma(qi, a.x, qr * a.y);
    return o;
}
// p * a + q * b
template <class T, class R>
__device__ __forceinline__ T cmul2(R pr, R pi, T a, R qr, R qi, T b) {
    T o;
    o.x = fma(-qi, b.y, fma(qr, b.x, fma(-pi, a.y, pr * a.x)));
    o.y = fma(qi, b.x, fma(qr, b.y, fma(pi, a.x, pr * a.y)));
    return o;
}
// real p, q: p * a + q * b
template <class T, class R>
__device__ __forceinline__ T rmul2(R p, T a, R q, T b) {
    T o;
    o.x = fma(q, b.x, p * a.x);
    o.y = fma(q, b.y, p * a.y);
    return o;
}

// Eq. 2 on one pair (a = alpha_{..0_k..}, b = alpha_{..1_k..}), specialised by
// the gate class the planner derived from the exact matrix entries.
template <int CLS, class T, class R>
__device__ __forceinline__ void pair_update(const R* m, T& a, T& b) {
    if constexpr (CLS == GC_GENERAL) {
        const T a2 = cmul2(m[0], m[1], a, m[2], m[3], b);
        const T b2 = cmul2(m[4], m[5], a, m[6], m[7], b);
        a = a2; b = b2;
    } else if constexpr (CLS == GC_REAL) {
        const T a2 = rmul2(m[0], a, m[2], b);
        const T b2 = rmul2(m[4], a, m[6], b);
        a = a2; b = b2;
    } else if constexpr (CLS == GC_DIAG) {
        a = cmul(m[0], m[1], a);
        b = cmul(m[6], m[7], b);
    } else if constexpr (CLS == GC_DIAG1) {
        b = cmul(m[6], m[7], b);
    } else if constexpr (CLS == GC_ANTIDIAG) {
        const T a2 = cmul(m[2], m[3], b);
        const T b2 = cmul(m[4], m[5], a);
        a = a2; b = b2;
    } else {  // GC_PERM: [[0,1],[1,0]] exactly: a move, bit-exact
        const T t = a; a = b; b = t;
    }
}

}  // namespace qs
