// df.cuh -- double-float ("DF") arithmetic for complex128 gate updates.
//
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, so a complex128 gate
// evaluated with FP64 instructions is bound by that pipe long before HBM.  DF
// arithmetic carries each double as an unevaluated pair hi + lo of floats and
// builds every product and sum from error-free transformations on the FP32
// pipes:
//   TwoProd  (p, e) = (a*b, fma(a, b, -a*b))        exact: a*b = p + e
//   TwoSum   (s, e) = Knuth's branch-free sum         exact: a + b = s + e
// (T. J. Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18, 1971; D. E. Knuth, TAOCP vol. 2, 4.2.2.)
//
// A pair holds about 48 significant bits.  Storage in HBM stays IEEE double:
// the split at load uses integer and FP32 instructions only, and the
// recombination at store is a single FP64 addition, rounded to nearest.
//
// Pairs are left unnormalised between gates: the high part of a sum is the
// rounded sum of the high parts of its products, and the low part is the
// rounded sum of all error terms, so |lo| stays within a few units in the last
// place of |hi| (or of the inputs' magnitudes, after cancellation).  Every
// operation here accepts such pairs; skipping the renormalisation (Fast2Sum)
// after each gate saves 3 of about 43 FP32 instructions per real component
// and keeps the error at the level of the dropped ql*xl term, below 2^-45 of
// the magnitudes involved.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qs {

struct dfl { float h, l; };

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// Product of a DF constant (qh, ql) and a DF value (xh, xl), left unnormalised:
// the exact product qh*xh split by TwoProd, plus the two cross terms; the term
// ql*xl (relative size 2^-48) is dropped.
__device__ __forceinline__ dfl df_mul(float qh, float ql, float xh, float xl) {
    const float ph = qh * xh;
    float pl = fmaf(qh, xh, -ph);
    pl = fmaf(qh, xl, pl);
    pl = fmaf(ql, xh, pl);
    return {ph, pl};
}

// sum of two unnormalised products (an unnormalised pair)
__device__ __forceinline__ dfl df_dot2(dfl a, dfl b) {
    const dfl s = two_sum(a.h, b.h);
    return {s.h, s.l + (a.l + b.l)};
}

// sum of four unnormalised products (an unnormalised pair)
__device__ __forceinline__ dfl df_dot4(dfl a, dfl b, dfl c, dfl d) {
    dfl s = two_sum(a.h, b.h);
    float lo = s.l + (a.l + b.l);
    s = two_sum(s.h, c.h);
    lo += s.l + c.l;
    s = two_sum(s.h, d.h);
    lo += s.l + d.l;
    return {s.h, lo};
}

// Split of a double into hi = its leading 24 significant bits (truncated,
// from the IEEE bit fields) and lo = the remaining 29 bits, converted to float
// (rounded to 24 bits) and scaled by the power of two 2^(e - 1075) built from
// its exponent bits.  |x - (hi + lo)| < 2^-47 |x|.  Integer and FP32
// instructions only, branch-free.  |x| < 2^-126 is flushed to zero and lo is
// dropped for |x| < 2^-74 (absolute changes below 2^-97); |x| >= 2^128
// saturates to an infinity (not reachable from a normalised state).
__device__ __forceinline__ dfl split_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu);
    const int e32 = e - 1023 + 127;
    const unsigned top23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    unsigned hi = sign | ((unsigned)e32 << 23) | top23;
    hi = e32 <= 0 ? sign : hi;
    hi = e32 >= 255 ? (sign | 0x7F800000u) : hi;
    const unsigned rem = lw & 0x1FFFFFFFu;  // weight 2^(e - 1023 - 52) per unit
    const float scale = __int_as_float((e - 1075 + 127) << 23);  // valid for 949 <= e < 1151
    const float lo = (e >= 949 && e32 < 255) ? __uint2float_rn(rem) * scale : 0.0f;
    return {__int_as_float((int)hi), __int_as_float(__float_as_int(lo) | (int)sign)};
}

// float -> double by the bit fields (exact; no FP64 instruction), branch-free.
// Zero and normal floats (a subnormal maps to a signed zero: below 1.2e-38).
__device__ __forceinline__ double float_to_double_bits(float f) {
    const unsigned u = (unsigned)__float_as_int(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned ef = (u >> 23) & 0xFFu;
    const unsigned long long ed = (unsigned long long)(ef + (1023 - 127)) << 52;
    const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
    unsigned long long r = sign | ed | m;
    r = ef == 0u ? sign : r;
    r = ef == 0xFFu ? (sign | 0x7FF0000000000000ull) : r;
    return __longlong_as_double((long long)r);
}

// hi + lo rounded to the nearest double (one FP64 addition).
__device__ __forceinline__ double join_double(dfl v) {
    return float_to_double_bits(v.h) + float_to_double_bits(v.l);
}

// ---- complex DF values: float4 (re.h, re.l, im.h, im.l) ---------------------

__device__ __forceinline__ float4 df_load(double2 a) {
    const dfl r = split_double(a.x), i = split_double(a.y);
    return make_float4(r.h, r.l, i.h, i.l);
}
__device__ __forceinline__ double2 df_store(float4 v) {
    return make_double2(join_double({v.x, v.y}), join_double({v.z, v.w}));
}

// ---- lean conversions for the single-gate kernels ------------------------------
// The strided kernels (gates.cu) are bound by the integer pipe, so their split
// and join use the forms below: 0.72 -> 0.93 of HBM for a single Haar gate at
// n = 30.  The tile kernels keep the forms above, which convert once per run of
// passes: with the lean forms compiled in, their n = 30 step took 800 instead of
// 771 ms (the kernel's code changed shape), so they are not used there.

// The split of split_double, bit for bit for every finite |x| < 2^128, in about
// half the integer instructions: hi's bits are the magnitude bits shifted right by 29 (a funnel
// shift over both words) with the exponent rebased from 1023 to 127 by one
// subtraction, and lo's scale is hi's exponent field lowered by 52.
// |x| < 2^-126 gives a signed zero and lo is dropped for |x| < 2^-74 (absolute
// changes below 2^-97); |x| >= 2^128 is not handled (not reachable from a
// normalised state).
__device__ __forceinline__ dfl split_double_lean(double x) {
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const unsigned sign = hw & 0x80000000u;
    const unsigned habs = hw & 0x7FFFFFFFu;
    unsigned hi = __funnelshift_r(lw, habs, 29) - (896u << 23);  // 896 << 23 wraps to 384 << 23: the same field
    hi = habs >= (897u << 20) ? (hi | sign) : sign;
    const int sb = (int)(hi & 0x7F800000u) - (52 << 23);
    const float lo = __uint2float_rn(lw & 0x1FFFFFFFu) * __int_as_float(max(sb, 0));
    return {__int_as_float((int)hi), __int_as_float(__float_as_int(lo) | (int)sign)};
}

// float_to_double_bits in fewer integer instructions, bit for bit for finite
// floats (exact; no FP64 instruction), branch-free:
// the magnitude bits shifted right by 3 with the exponent rebased from 127 to
// 1023 by one addition form the high word, the last three significand bits the
// low word.  Zero and subnormal floats give a signed zero; infinities and NaNs
// are not handled (not reachable from a normalised state).
__device__ __forceinline__ double float_to_double_bits_lean(float f) {
    const unsigned u = (unsigned)__float_as_int(f), ua = u & 0x7FFFFFFFu, s = u & 0x80000000u;
    const bool nz = ua >= 0x00800000u;
    const unsigned hi = ((ua >> 3) + (896u << 20)) | s;
    return __hiloint2double((int)(nz ? hi : s), (int)(nz ? (u << 29) : 0u));
}

__device__ __forceinline__ double join_double_lean(dfl v) {
    return float_to_double_bits_lean(v.h) + float_to_double_bits_lean(v.l);
}
__device__ __forceinline__ float4 df_load_lean(double2 a) {
    const dfl r = split_double_lean(a.x), i = split_double_lean(a.y);
    return make_float4(r.h, r.l, i.h, i.l);
}
__device__ __forceinline__ double2 df_store_lean(float4 v) {
    return make_double2(join_double_lean({v.x, v.y}), join_double_lean({v.z, v.w}));
}

// Gate constants: 8 doubles (q11r, q11i, q12r, q12i, q21r, q21i, q22r, q22i),
// each as (hi, lo) floats: c[2j] = hi, c[2j+1] = lo of double j.
#define QH(j) c[2 * (j)]
#define QL(j) c[2 * (j) + 1]

// q * x for complex DF constant q = double pair (jr, ji) and complex DF value x
__device__ __forceinline__ float4 df_cmul(const float* c, int jr, int ji, float4 x) {
    const dfl re = df_dot2(df_mul(QH(jr), QL(jr), x.x, x.y), df_mul(-QH(ji), -QL(ji), x.z, x.w));
    const dfl im = df_dot2(df_mul(QH(jr), QL(jr), x.z, x.w), df_mul(QH(ji), QL(ji), x.x, x.y));
    return make_float4(re.h, re.l, im.h, im.l);
}
// p * a + q * b, p = pair (pr, pi), q = pair (qr, qi)
__device__ __forceinline__ float4 df_cmul2(const float* c, int pr, int pi, float4 a, int qr, int qi, float4 b) {
    const dfl re = df_dot4(df_mul(QH(pr), QL(pr), a.x, a.y), df_mul(-QH(pi), -QL(pi), a.z, a.w),
                           df_mul(QH(qr), QL(qr), b.x, b.y), df_mul(-QH(qi), -QL(qi), b.z, b.w));
    const dfl im = df_dot4(df_mul(QH(pr), QL(pr), a.z, a.w), df_mul(QH(pi), QL(pi), a.x, a.y),
                           df_mul(QH(qr), QL(qr), b.z, b.w), df_mul(QH(qi), QL(qi), b.x, b.y));
    return make_float4(re.h, re.l, im.h, im.l);
}
// real p, q: p * a + q * b
__device__ __forceinline__ float4 df_rmul2(const float* c, int p, float4 a, int q, float4 b) {
    const dfl re = df_dot2(df_mul(QH(p), QL(p), a.x, a.y), df_mul(QH(q), QL(q), b.x, b.y));
    const dfl im = df_dot2(df_mul(QH(p), QL(p), a.z, a.w), df_mul(QH(q), QL(q), b.z, b.w));
    return make_float4(re.h, re.l, im.h, im.l);
}

// balanced real gate: q * (a + s b) for real DF constant q = double j and s = +-1
// (a and b complex DF values): the sum is exact (TwoSum), then one product
__device__ __forceinline__ dfl df_addsig(float ah, float al, float s, float bh, float bl) {
    const dfl t = two_sum(ah, s * bh);  // s * bh is exact
    return {t.h, t.l + fmaf(s, bl, al)};
}
__device__ __forceinline__ float4 df_bal(const float* c, int j, float s, float4 a, float4 b) {
    const dfl tr = df_addsig(a.x, a.y, s, b.x, b.y), ti = df_addsig(a.z, a.w, s, b.z, b.w);
    const dfl re = df_mul(QH(j), QL(j), tr.h, tr.l), im = df_mul(QH(j), QL(j), ti.h, ti.l);
    return make_float4(re.h, re.l, im.h, im.l);
}

// phase, shear, phase (GC_PRP): bt = y b; a' = a + t bt; b' = z (bt - t a),
// with y = doubles (0, 1), the real t = double 2, z = doubles (4, 5); Z = false
// leaves out the product by z (z = 1, GC_PRP_NZ)
template <bool Z>
__device__ __forceinline__ void df_prp(const float* c, float4& a, float4& b) {
    const float4 bt = df_cmul(c, 0, 1, b);
    const dfl ar = df_dot2({a.x, a.y}, df_mul(QH(2), QL(2), bt.x, bt.y));
    const dfl ai = df_dot2({a.z, a.w}, df_mul(QH(2), QL(2), bt.z, bt.w));
    const dfl br = df_dot2({bt.x, bt.y}, df_mul(-QH(2), -QL(2), a.x, a.y));
    const dfl bi = df_dot2({bt.z, bt.w}, df_mul(-QH(2), -QL(2), a.z, a.w));
    a = make_float4(ar.h, ar.l, ai.h, ai.l);
    if constexpr (Z) b = df_cmul(c, 4, 5, make_float4(br.h, br.l, bi.h, bi.l));
    else b = make_float4(br.h, br.l, bi.h, bi.l);
}

#undef QH
#undef QL

}  // namespace qs
