// batch.cu -- energies and adjoint gradients of many variational circuits at
// once (qs_batch_*, qs_grad).  Not in the paper.
//
// Adjoint differentiation (T. Jones and J. Gacon, arXiv:2009.02823): for
// psi = U_P .. U_1 |0..0> and rotations U_j = exp(-i theta_j G_j / 2),
//   lambda = H psi,  E = Re <psi|lambda>,  phi = psi,
//   for j = P .. 1:  if U_j is a rotation, dE/dtheta_j += Im <lambda| G_j |phi>;
//                    phi <- U_j^dagger phi,  lambda <- U_j^dagger lambda.
// A gate may be swept past gates it commutes with (disjoint qubits, or both
// diagonal): such a gate U_k also commutes with G_j, so Im <lambda|G_j|phi> is
// unchanged when U_k^dagger has (or has not yet) been applied to both states.
//
// Work split:
//   * small instances (phi and lambda fit in one CTA's shared memory) run in
//     one persistent kernel: each CTA takes instances from an atomic work
//     counter and does the forward pass, lambda, E and the whole reverse sweep
//     in shared memory, with block-level FP64 reductions;
//   * larger instances are grouped by identical circuit structure; each group
//     runs batched tile passes (grid.y = instances): forward passes on psi,
//     then reverse tile passes that hold phi and lambda tiles together and
//     write one FP64 partial per rotation gate and tile, summed in fixed order.
// All launches (and the upload of the gate matrices for the current angles)
// are captured once into a CUDA graph and replayed by qs_batch_execute.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "device.cuh"
#include "df.cuh"
#include "tile_df_ops.cuh"
#include "tile_ops.cuh"

namespace qs {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kSmallThreads = 512;
constexpr int kRedThreadsB = 256;
constexpr int kMaxCrossB = 64;
constexpr int kMaxXB = 64;

__device__ __forceinline__ double warp_sum_b(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Sum over the block, valid in thread 0; barriers on entry and exit keep `red` reusable.
__device__ __forceinline__ double block_sum_b(double v, double* red) {
    v = warp_sum_b(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        r = warp_sum_b(r);
    }
    return r;
}

template <class T> __device__ __forceinline__ double re_cb(const T& a, const T& b) {
    return fma((double)a.x, (double)b.x, (double)a.y * (double)b.y);
}

// Per-thread gradient and energy sums: a float pair (hi, lo) fed with products
// split exactly (TwoProd) or as double-float products; converted to double once
// per reduction and summed across the block in FP64.  No FP64 instruction per
// amplitude pair.
struct GAcc { float h = 0.0f, l = 0.0f; };
__device__ __forceinline__ void gacc_add(GAcc& a, float ph, float pl) {
    const dfl s = two_sum(a.h, ph);
    a.h = s.h;
    a.l += s.l + pl;
}
__device__ __forceinline__ void gacc_prod(GAcc& a, float x, float y) {
    const float p = x * y;
    gacc_add(a, p, fmaf(x, y, -p));
}
__device__ __forceinline__ void gacc_dfprod(GAcc& a, float xh, float xl, float yh, float yl) {
    const dfl p = df_mul(xh, xl, yh, yl);
    gacc_add(a, p.h, p.l);
}
__device__ __forceinline__ double gacc_value(const GAcc& a) { return (double)a.h + (double)a.l; }

// a + b for two accumulators, renormalised (TwoSum of the high parts, then
// Fast2Sum of the result), so that later sums keep the pair's ~47 bits
__device__ __forceinline__ GAcc gacc_plus(GAcc a, GAcc b) {
    const dfl s = two_sum(a.h, b.h);
    const float t = s.l + (a.l + b.l);
    const float h = s.h + t;
    return {h, t - (h - s.h)};
}
// Sum over the warp in float pairs (valid in every lane).  A rotation's
// gradient partial is reduced per gate; in FP64 (a conversion and five
// additions per thread at 1/64 of the FP32 rate) that reduction cost as much
// as the gate's double-float arithmetic on both tiles.
__device__ __forceinline__ GAcc gacc_warp_sum(GAcc a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        GAcc b;
        b.h = __shfl_xor_sync(0xffffffffu, a.h, o);
        b.l = __shfl_xor_sync(0xffffffffu, a.l, o);
        a = gacc_plus(a, b);
    }
    return a;
}
// Sum over the block, as a double valid in thread 0: warps in float pairs, then
// the per-warp pairs (in `red`, 32 float2) summed by warp 0 and converted once.
// Barriers on entry and exit keep `red` reusable.
__device__ __forceinline__ double gacc_block_sum(GAcc a, float2* red) {
    a = gacc_warp_sum(a);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = make_float2(a.h, a.l);
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        GAcc w;
        if (lane < (int)(blockDim.x >> 5)) { w.h = red[lane].x; w.l = red[lane].y; }
        r = gacc_value(gacc_warp_sum(w));
    }
    return r;
}

// ---- arithmetic traits: complex64 (FP32) and complex128 (double-float) ----------
struct TrF {
    using E = float2;               // tile element
    using G = float2;               // element in device memory
    using Op = TileOp<float>;
    static __device__ __forceinline__ E load(G g) { return g; }
    static __device__ __forceinline__ G store(E e) { return e; }
    template <int CLS> static __device__ __forceinline__ void pair(const Op& op, E& a, E& b) { pair_update<CLS>(op.m, a, b); }
    static __device__ __forceinline__ E scale(const Op& op, bool use22, E x) {
        return use22 ? cmul(op.m[6], op.m[7], x) : cmul(op.m[0], op.m[1], x);
    }
    // +Re(conj(a) b) or +Im(conj(a) b), with sign s = +1 / -1
    static __device__ __forceinline__ void re(GAcc& c, E a, E b, float s) { gacc_prod(c, s * a.x, b.x); gacc_prod(c, s * a.y, b.y); }
    static __device__ __forceinline__ void im(GAcc& c, E a, E b, float s) { gacc_prod(c, s * a.x, b.y); gacc_prod(c, -s * a.y, b.x); }
    static __device__ __forceinline__ double2 to_d(E e) { return make_double2(e.x, e.y); }
    static __device__ __forceinline__ E from_d(double2 d) { return make_float2((float)d.x, (float)d.y); }
    template <int THREADS>
    static __device__ __forceinline__ bool fwd(E* sm, uint32_t N, const Op& op, uint64_t base) {
        return tile_apply<float, THREADS>(sm, N, op, base);
    }
};

struct TrDF {
    using E = float4;
    using G = double2;
    using Op = TileOpDF;
    static __device__ __forceinline__ E load(G g) { return df_load(g); }
    static __device__ __forceinline__ G store(E e) { return df_store(e); }
    template <int CLS> static __device__ __forceinline__ void pair(const Op& op, E& a, E& b) { df_pair_update<CLS>(op.c, a, b); }
    static __device__ __forceinline__ E scale(const Op& op, bool use22, E x) {
        return use22 ? df_cmul(op.c, 6, 7, x) : df_cmul(op.c, 0, 1, x);
    }
    static __device__ __forceinline__ void re(GAcc& c, E a, E b, float s) {
        gacc_dfprod(c, s * a.x, s * a.y, b.x, b.y);
        gacc_dfprod(c, s * a.z, s * a.w, b.z, b.w);
    }
    static __device__ __forceinline__ void im(GAcc& c, E a, E b, float s) {
        gacc_dfprod(c, s * a.x, s * a.y, b.z, b.w);
        gacc_dfprod(c, -s * a.z, -s * a.w, b.x, b.y);
    }
    static __device__ __forceinline__ double2 to_d(E e) { return df_store(e); }
    static __device__ __forceinline__ E from_d(double2 d) { return df_load(d); }
    template <int THREADS>
    static __device__ __forceinline__ bool fwd(E* sm, uint32_t N, const Op& op, uint64_t base) {
        return df_tile_apply<THREADS>(sm, N, op, base);
    }
};

// Im <lambda| G |phi> restricted to one pair; gen 1 = X, 2 = Y, 3 = Z.
template <class Tr>
__device__ __forceinline__ void gen_acc(GAcc& c, int gen, const typename Tr::E& f0, const typename Tr::E& f1,
                                        const typename Tr::E& l0, const typename Tr::E& l1) {
    if (gen == 1) { Tr::im(c, l0, f1, 1.0f); Tr::im(c, l1, f0, 1.0f); }
    else if (gen == 2) { Tr::re(c, l1, f0, 1.0f); Tr::re(c, l0, f1, -1.0f); }
    else { Tr::im(c, l0, f0, 1.0f); Tr::im(c, l1, f1, -1.0f); }
}

// ---- one reversed op on (phi, lambda) tiles ------------------------------------
// op.pad0 = generator (0 = not a rotation), op.pad1 = output slot.
template <class Tr, int CLS, int THREADS>
__device__ __forceinline__ void adj_pairs(typename Tr::E* f, typename Tr::E* l, uint32_t N, int cb, int tb,
                                          const typename Tr::Op& op, int gen, GAcc& acc) {
    using E = typename Tr::E;
    if (cb < 0) {
        for (uint32_t p = threadIdx.x; p < (N >> 1); p += THREADS) {
            const uint32_t i0 = insert_zero32(p, tb), i1 = i0 | (1u << tb);
            E f0 = f[i0], f1 = f[i1], l0 = l[i0], l1 = l[i1];
            if (gen) gen_acc<Tr>(acc, gen, f0, f1, l0, l1);
            Tr::template pair<CLS>(op, f0, f1);
            Tr::template pair<CLS>(op, l0, l1);
            f[i0] = f0; f[i1] = f1; l[i0] = l0; l[i1] = l1;
        }
    } else {
        const int lo = min(cb, tb), hi = max(cb, tb);
        for (uint32_t p = threadIdx.x; p < (N >> 2); p += THREADS) {
            const uint32_t i0 = insert_two_zeros32(p, lo, hi) | (1u << cb), i1 = i0 | (1u << tb);
            E f0 = f[i0], f1 = f[i1], l0 = l[i0], l1 = l[i1];
            if (gen) gen_acc<Tr>(acc, gen, f0, f1, l0, l1);
            Tr::template pair<CLS>(op, f0, f1);
            Tr::template pair<CLS>(op, l0, l1);
            f[i0] = f0; f[i1] = f1; l[i0] = l0; l[i1] = l1;
        }
    }
}

// Fixed-size tiles (2^B amplitudes): per-thread base index plus CTA-uniform
// offsets, two pairs of both states per unrolled step (see tile_df_ops.cuh).
template <class Tr, int CLS, int THREADS, int B>
__device__ __forceinline__ void adj_pairs_fixed(typename Tr::E* f, typename Tr::E* l, int cb, int tb,
                                                const typename Tr::Op& op, int gen, GAcc& acc) {
    using E = typename Tr::E;
    if (cb < 0) {
        constexpr int PAIRS = (1 << (B - 1)) / THREADS;
        const uint32_t i0 = insert_zero32(threadIdx.x, tb), h = 1u << tb, hm = ~0u << tb;
#pragma unroll
        for (int m = 0; m < PAIRS; m += 2) {
            const uint32_t a = i0 + insert_zero32_hm((uint32_t)(m * THREADS), hm);
            const uint32_t b = i0 + insert_zero32_hm((uint32_t)((m + 1) * THREADS), hm);
            E f0 = f[a], f1 = f[a + h], l0 = l[a], l1 = l[a + h];
            E g0 = f[b], g1 = f[b + h], k0 = l[b], k1 = l[b + h];
            if (gen) { gen_acc<Tr>(acc, gen, f0, f1, l0, l1); gen_acc<Tr>(acc, gen, g0, g1, k0, k1); }
            Tr::template pair<CLS>(op, f0, f1);
            Tr::template pair<CLS>(op, l0, l1);
            Tr::template pair<CLS>(op, g0, g1);
            Tr::template pair<CLS>(op, k0, k1);
            f[a] = f0; f[a + h] = f1; l[a] = l0; l[a + h] = l1;
            f[b] = g0; f[b + h] = g1; l[b] = k0; l[b + h] = k1;
        }
    } else {
        constexpr int ITEMS = (1 << (B - 2)) / THREADS;
        const int lo = min(cb, tb), hi = max(cb, tb);
        const uint32_t i0 = insert_two_zeros32(threadIdx.x, lo, hi) | (1u << cb), h = 1u << tb;
        const uint32_t hlo = ~0u << lo, hhi = ~0u << hi;
#pragma unroll
        for (int m = 0; m < ITEMS; m += 2) {
            const uint32_t a = i0 + insert_zero32_hm(insert_zero32_hm((uint32_t)(m * THREADS), hlo), hhi);
            const uint32_t b = i0 + insert_zero32_hm(insert_zero32_hm((uint32_t)((m + 1) * THREADS), hlo), hhi);
            E f0 = f[a], f1 = f[a + h], l0 = l[a], l1 = l[a + h];
            E g0 = f[b], g1 = f[b + h], k0 = l[b], k1 = l[b + h];
            if (gen) { gen_acc<Tr>(acc, gen, f0, f1, l0, l1); gen_acc<Tr>(acc, gen, g0, g1, k0, k1); }
            Tr::template pair<CLS>(op, f0, f1);
            Tr::template pair<CLS>(op, l0, l1);
            Tr::template pair<CLS>(op, g0, g1);
            Tr::template pair<CLS>(op, k0, k1);
            f[a] = f0; f[a + h] = f1; l[a] = l0; l[a + h] = l1;
            f[b] = g0; f[b + h] = g1; l[b] = k0; l[b + h] = k1;
        }
    }
}

template <class Tr, int CLS, int THREADS, int B>
__device__ __forceinline__ void adj_pairs_any(typename Tr::E* f, typename Tr::E* l, uint32_t N, int cb, int tb,
                                              const typename Tr::Op& op, int gen, GAcc& acc) {
    if constexpr (B > 0 && (1 << (B - 2)) / THREADS >= 2) adj_pairs_fixed<Tr, CLS, THREADS, B>(f, l, cb, tb, op, gen, acc);
    else adj_pairs<Tr, CLS, THREADS>(f, l, N, cb, tb, op, gen, acc);
}


// One reversed op on the (phi, lambda) tiles.  A rotation's gradient partial is
// written to out[op.pad1]: reduced over the CTA (WARP_SLOTS = false), or only
// over each warp into out[op.pad1 * warps + warp] (WARP_SLOTS = true; the caller
// sums the warps once after the pass, saving two barriers per rotation).
template <class Tr, int THREADS, int B = 0, bool WARP_SLOTS = false>
__device__ __forceinline__ void adj_apply(typename Tr::E* f, typename Tr::E* l, uint32_t N, const typename Tr::Op& op,
                                          uint64_t base, double* red, double* out) {
    using E = typename Tr::E;
    const int gen = op.pad0;
    GAcc acc;
    bool active = true;
    int cb = -1;
    if (op.kind == OP_SWAP) {
        const int lo = min(op.tb, op.cb), hi = max(op.tb, op.cb);
        for (uint32_t p = threadIdx.x; p < (N >> 2); p += THREADS) {
            const uint32_t i = insert_two_zeros32(p, lo, hi), a = i | (1u << op.tb), b = i | (1u << op.cb);
            const E x = f[a]; f[a] = f[b]; f[b] = x;
            const E y = l[a]; l[a] = l[b]; l[b] = y;
        }
        active = false;
    } else if (op.kind == OP_CU) {
        if (op.cb < 0) active = ((base >> op.cq) & 1ull) != 0;
        else cb = op.cb;
    }
    if (active && op.kind != OP_SWAP) {
        if (op.tb < 0) {  // diagonal with its target outside the tile: one factor per (half-)tile
            const bool bit = (base >> op.tq) & 1ull;
            const bool skip = op.cls == GC_DIAG1 && !bit;
            const float zs = bit ? -1.0f : 1.0f;  // Z eigenvalue of the target bit (only Z rotations are diagonal)
            if (cb < 0) {
                for (uint32_t e = threadIdx.x; e < N; e += THREADS) {
                    if (gen) Tr::im(acc, l[e], f[e], zs);
                    if (!skip) { f[e] = Tr::scale(op, bit, f[e]); l[e] = Tr::scale(op, bit, l[e]); }
                }
            } else {
                for (uint32_t p = threadIdx.x; p < (N >> 1); p += THREADS) {
                    const uint32_t e = insert_zero32(p, cb) | (1u << cb);
                    if (gen) Tr::im(acc, l[e], f[e], zs);
                    if (!skip) { f[e] = Tr::scale(op, bit, f[e]); l[e] = Tr::scale(op, bit, l[e]); }
                }
            }
        } else {
            switch (op.cls) {
            case GC_GENERAL: adj_pairs_any<Tr, GC_GENERAL, THREADS, B>(f, l, N, cb, op.tb, op, gen, acc); break;
            case GC_REAL: adj_pairs_any<Tr, GC_REAL, THREADS, B>(f, l, N, cb, op.tb, op, gen, acc); break;
            case GC_DIAG: adj_pairs_any<Tr, GC_DIAG, THREADS, B>(f, l, N, cb, op.tb, op, gen, acc); break;
            case GC_DIAG1: adj_pairs_any<Tr, GC_DIAG1, THREADS, B>(f, l, N, cb, op.tb, op, gen, acc); break;
            case GC_ANTIDIAG: adj_pairs_any<Tr, GC_ANTIDIAG, THREADS, B>(f, l, N, cb, op.tb, op, gen, acc); break;
            default: adj_pairs_any<Tr, GC_PERM, THREADS, B>(f, l, N, cb, op.tb, op, gen, acc); break;
            }
        }
    }
    if (gen) {  // uniform over the CTA: every thread takes part in the reduction
        if constexpr (WARP_SLOTS) {
            // per-warp float pairs; the pass sums them in FP64 once at its end
            const GAcc w = gacc_warp_sum(active ? acc : GAcc{});
            if ((threadIdx.x & 31) == 0)
                reinterpret_cast<float2*>(out)[op.pad1 * (THREADS / 32) + (threadIdx.x >> 5)] = make_float2(w.h, w.l);
        } else {
            const double s = gacc_block_sum(active ? acc : GAcc{}, reinterpret_cast<float2*>(red));
            if (threadIdx.x == 0) out[op.pad1] = s;
        }
    }
}

// ---- reverse tile pass over a group of instances --------------------------------
constexpr int kMaxAdjSlots = 1024;  // rotation gates per reverse tile pass (per-warp slots in dynamic SMEM)

template <class Tr, int B>
__global__ void __launch_bounds__(kAdjThreads) k_tile_adj(typename Tr::G* __restrict__ phi,
                                                          typename Tr::G* __restrict__ lam,
                                                          const typename Tr::Op* __restrict__ ops, TilePass P,
                                                          double* __restrict__ partials, int n_slots) {
    using E = typename Tr::E;
    constexpr int kWarps = kAdjThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const int b = P.b, b0 = P.b0, nh = b - b0;
    const uint32_t N = 1u << b;
    E* f = reinterpret_cast<E*>(smem_raw);
    E* l = f + N;
    double* wslots = reinterpret_cast<double*>(l + N);        // n_slots x warps, each a float pair
    uint64_t* hioff = reinterpret_cast<uint64_t*>(wslots + (size_t)n_slots * kWarps);
    phi += (uint64_t)blockIdx.y * P.inst_stride;
    lam += (uint64_t)blockIdx.y * P.inst_stride;
    ops += (uint64_t)blockIdx.y * (uint64_t)P.ops_stride;
    double* out = partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * n_slots;
    const uint64_t base = deposit_bits((uint64_t)blockIdx.x, P.nontile_mask);
    for (uint32_t h = threadIdx.x; h < (1u << nh); h += kAdjThreads) {
        uint64_t off = 0;
        for (int j = 0; j < nh; ++j)
            if ((h >> j) & 1u) off |= 1ull << P.hi_q[j];
        hioff[h] = off;
    }
    __syncthreads();
    const uint32_t lomask = (1u << b0) - 1u;
    constexpr bool kDF = std::is_same<E, float4>::value;
    // double-float: consecutive reverse passes hand phi and lambda over as float
    // pairs (kIoPairsIn / kIoPairsOut), the last one does not store them at all
    const bool pairs_in = kDF && (P.io & kIoPairsIn);
    auto take = [&](typename Tr::G raw) -> E {
        if constexpr (kDF) {
            if (pairs_in) return *reinterpret_cast<const E*>(&raw);
        }
        return Tr::load(raw);
    };
    if constexpr (B > 0 && (1 << B) >= kAdjThreads) {
        // fixed tile size: four amplitudes of each state in flight per thread
        constexpr int PER = (1 << B) / kAdjThreads;
        constexpr int BATCH = PER < 4 ? PER : 4;
#pragma unroll
        for (int u0 = 0; u0 < PER; u0 += BATCH) {
            typename Tr::G vf[BATCH], vl[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const uint32_t e = threadIdx.x + (uint32_t)((u0 + k) * kAdjThreads);
                const uint64_t g = base + hioff[e >> b0] + (e & lomask);
                vf[k] = phi[g];
                vl[k] = lam[g];
            }
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const uint32_t e = threadIdx.x + (uint32_t)((u0 + k) * kAdjThreads);
                f[e] = take(vf[k]);
                l[e] = take(vl[k]);
            }
        }
    } else {
        for (uint32_t e = threadIdx.x; e < N; e += kAdjThreads) {
            const uint64_t g = base + hioff[e >> b0] + (e & lomask);
            f[e] = take(phi[g]);
            l[e] = take(lam[g]);
        }
    }
    __syncthreads();
    for (int g = 0; g < P.nops; ++g) {
        const typename Tr::Op op = ops[P.op0 + g];
        adj_apply<Tr, kAdjThreads, B, true>(f, l, N, op, base, red, wslots);
        __syncthreads();
    }
    if (!(P.io & kIoDiscard)) {
        for (uint32_t e = threadIdx.x; e < N; e += kAdjThreads) {
            const uint64_t g = base + hioff[e >> b0] + (e & lomask);
            if constexpr (kDF) {
                if (P.io & kIoPairsOut) {  // renormalised by TwoSum, as in the forward passes
                    const E a = f[e], c = l[e];
                    const dfl ar = two_sum(a.x, a.y), ai = two_sum(a.z, a.w);
                    const dfl cr = two_sum(c.x, c.y), ci = two_sum(c.z, c.w);
                    reinterpret_cast<E*>(phi)[g] = make_float4(ar.h, ar.l, ai.h, ai.l);
                    reinterpret_cast<E*>(lam)[g] = make_float4(cr.h, cr.l, ci.h, ci.l);
                    continue;
                }
            }
            phi[g] = Tr::store(f[e]);
            lam[g] = Tr::store(l[e]);
        }
    }
    // rotation partials: the warps' sums in fixed order (slots this pass does not use are never read)
    const float2* wpairs = reinterpret_cast<const float2*>(wslots);
    for (int sl = threadIdx.x; sl < n_slots; sl += kAdjThreads) {
        double acc = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            const float2 v = wpairs[sl * kWarps + w];
            acc += (double)v.x + (double)v.y;
        }
        out[sl] = acc;
    }
}

// rot_vals[inst * n_rot + slot_rot[s]] = sum over tiles of partials[inst][tile][s]
__global__ void k_adj_finalize(const double* __restrict__ partials, int n_tiles, int n_slots, int count,
                               const int* __restrict__ slot_rot, double* __restrict__ rot_vals, int n_rot) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count * n_slots) return;
    const int inst = k / n_slots, s = k % n_slots;
    const int r = slot_rot[s];
    if (r < 0) return;
    double acc = 0.0;
    for (int t = 0; t < n_tiles; ++t) acc += partials[((size_t)inst * n_tiles + t) * n_slots + s];
    rot_vals[(size_t)inst * n_rot + r] = acc;
}

// ---- lambda = H psi and E = Re <psi|lambda> for a group --------------------------
struct HGroup {
    int lo_bits;
    int tab_stride;            // doubles per instance: lo table then hi table
    int n_cross, n_x;          // per instance (same structure within the group)
};

template <class T>
__global__ void k_apply_h_b(const T* __restrict__ psi, T* __restrict__ lam, uint64_t N, HGroup H,
                            const double* __restrict__ tabs, const int* __restrict__ cross_q,
                            const double* __restrict__ cross_c, const int* __restrict__ x_q,
                            const double* __restrict__ x_c) {
    const uint64_t inst = blockIdx.y;
    psi += inst * N;
    lam += inst * N;
    const double* lo_tab = tabs + inst * (uint64_t)H.tab_stride;
    const double* hi_tab = lo_tab + (1ull << H.lo_bits);
    cross_c += inst * H.n_cross;
    x_c += inst * H.n_x;
    const uint64_t lo_mask = (1ull << H.lo_bits) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        double e = lo_tab[i & lo_mask] + hi_tab[i >> H.lo_bits];
        for (int k = 0; k < H.n_cross; ++k) {
            const uint64_t par = ((i >> cross_q[2 * k]) ^ (i >> cross_q[2 * k + 1])) & 1ull;
            e += par ? -cross_c[k] : cross_c[k];
        }
        const T v = psi[i];
        double ox = e * (double)v.x, oy = e * (double)v.y;
        for (int k = 0; k < H.n_x; ++k) {
            const T w = psi[i ^ (1ull << x_q[k])];
            ox = fma(x_c[k], (double)w.x, ox);
            oy = fma(x_c[k], (double)w.y, oy);
        }
        T o;
        o.x = (decltype(o.x))ox;
        o.y = (decltype(o.y))oy;
        lam[i] = o;
    }
}

template <class T>
__global__ void __launch_bounds__(kRedThreadsB) k_dot_b(const T* __restrict__ a, const T* __restrict__ b, uint64_t N,
                                                        double* __restrict__ partials) {
    __shared__ double red[32];
    const uint64_t inst = blockIdx.y;
    a += inst * N;
    b += inst * N;
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kRedThreadsB;
    for (uint64_t i = (uint64_t)blockIdx.x * kRedThreadsB + threadIdx.x; i < N; i += stride) acc += re_cb(a[i], b[i]);
    const double s = block_sum_b(acc, red);
    if (threadIdx.x == 0) partials[inst * gridDim.x + blockIdx.x] = s;
}

// out[r] = sum_c partials[r * cols + c], fixed order
__global__ void k_sum_rows(const double* __restrict__ partials, int rows, int cols, double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double s = 0.0;
    for (int c = 0; c < cols; ++c) s += partials[(size_t)r * cols + c];
    out[r] = s;
}

// |0..0> for `count` instances of N amplitudes (memset to zero beforehand)
template <class T>
__global__ void k_set_zero_basis(T* psi, uint64_t N, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        T one;
        one.x = 1;
        one.y = 0;
        psi[(uint64_t)i * N] = one;
    }
}

// ---- small instances: one CTA does everything in shared memory ------------------
struct SmallDesc {
    int32_t n, n_ops, op_off, n_terms, term_off, rot_off, e_out, pad;
};

template <class Tr>
__global__ void __launch_bounds__(kSmallThreads) k_batch_small(const SmallDesc* __restrict__ descs, int n_desc,
                                                               const typename Tr::Op* __restrict__ fwd,
                                                               const typename Tr::Op* __restrict__ rev,
                                                               const qs_term* __restrict__ terms,
                                                               double* __restrict__ rot_vals,
                                                               double* __restrict__ energies, int* counter) {
    using E = typename Tr::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= n_desc) break;
        const SmallDesc d = descs[item];
        const uint32_t N = 1u << d.n;
        E* psi = reinterpret_cast<E*>(smem_raw);
        E* lam = psi + N;
        for (uint32_t e = threadIdx.x; e < N; e += kSmallThreads) psi[e] = Tr::from_d(make_double2(e == 0 ? 1.0 : 0.0, 0.0));
        __syncthreads();
        for (int g = 0; g < d.n_ops; ++g) {
            const typename Tr::Op op = fwd[d.op_off + g];
            if (Tr::template fwd<kSmallThreads>(psi, N, op, 0ull)) __syncthreads();
        }
        // lambda = H psi; the diagonal part is evaluated from the index bits, per element in FP64
        for (uint32_t e = threadIdx.x; e < N; e += kSmallThreads) {
            double ev = 0.0, ox = 0.0, oy = 0.0;
            for (int k = 0; k < d.n_terms; ++k) {
                const qs_term t = terms[d.term_off + k];
                if (t.kind == QS_P_X) {
                    const double2 w = Tr::to_d(psi[e ^ (1u << t.q0)]);
                    ox = fma(t.coef, w.x, ox);
                    oy = fma(t.coef, w.y, oy);
                } else {
                    const uint32_t par = t.kind == QS_P_Z ? ((e >> t.q0) & 1u) : (((e >> t.q0) ^ (e >> t.q1)) & 1u);
                    ev += par ? -t.coef : t.coef;
                }
            }
            const double2 v = Tr::to_d(psi[e]);
            lam[e] = Tr::from_d(make_double2(fma(ev, v.x, ox), fma(ev, v.y, oy)));
        }
        __syncthreads();
        GAcc acc;
        for (uint32_t e = threadIdx.x; e < N; e += kSmallThreads) Tr::re(acc, psi[e], lam[e], 1.0f);
        const double en = gacc_block_sum(acc, reinterpret_cast<float2*>(red));
        if (threadIdx.x == 0) energies[d.e_out] = en;
        for (int g = 0; g < d.n_ops; ++g) {  // rev[] is already in reverse circuit order
            const typename Tr::Op op = rev[d.op_off + g];
            adj_apply<Tr, kSmallThreads>(psi, lam, N, op, 0ull, red, rot_vals + d.rot_off);
            __syncthreads();
        }
    }
}

// ---- host side -------------------------------------------------------------------

int rot_gen(int kind) { return kind == QS_G_RX ? 1 : kind == QS_G_RY ? 2 : kind == QS_G_RZ ? 3 : 0; }

void dagger(const double m[8], double d[8]) {
    d[0] = m[0]; d[1] = -m[1];
    d[2] = m[4]; d[3] = -m[5];
    d[4] = m[2]; d[5] = -m[3];
    d[6] = m[6]; d[7] = -m[7];
}

// Lower an instance's gates; rotation classes are fixed by kind so that every
// angle gives the same plan (RX general, RY real, RZ a phase gate).
//
// RZ(theta) = e^{-i theta/2} diag(1, e^{i theta}) is applied as diag(1, e^{i theta}),
// which changes only the |1> amplitudes (half the arithmetic of a diagonal gate).
// The dropped factor is a global phase: every forward state, and in the reverse
// sweep phi and lambda alike, carries the same phase e^{i A} (A = half the sum of
// the RZ angles applied so far), so E = <psi|H|psi> and the gradient terms
// Im <lambda|Z|phi> are unchanged.  (With diag(1, e^{i theta}) as the gate, its
// derivative is i diag(0, 1) U = (i/2)(I - Z) U, which adds -Im <lambda|phi> to
// the term; <lambda|phi> = <H psi|psi> = E is real, so that addition is zero.)
// Batches return energies and gradients only, never the state, so the phase
// is unobservable; plans (qs_run) keep the exact RZ matrix.
qs_status lower_instance(const qs_instance& in, std::vector<Op>& ops) {
    if (qs_status st = lower_gates(in.gates, in.n_gates, in.theta, in.n_params, in.n, ops)) return st;
    for (int j = 0; j < in.n_gates; ++j) {
        const int k = in.gates[j].kind;
        if (k == QS_G_RX) ops[j].cls = GC_GENERAL;
        else if (k == QS_G_RY) ops[j].cls = GC_REAL;
        else if (k == QS_G_RZ) {
            const double th = in.theta[in.gates[j].param];
            double* m = ops[j].m;
            m[0] = 1.0; m[1] = 0.0; m[2] = m[3] = m[4] = m[5] = 0.0;
            m[6] = std::cos(th); m[7] = std::sin(th);
            ops[j].cls = GC_DIAG1;
        }
    }
    return QS_OK;
}

// reversed, daggered op list
void reverse_ops(const std::vector<Op>& f, std::vector<Op>& r) {
    r.assign(f.rbegin(), f.rend());
    for (Op& o : r) {
        if (o.kind == OP_SWAP) continue;
        double d[8];
        dagger(o.m, d);
        std::memcpy(o.m, d, sizeof(d));
        if (o.cls == GC_DIAG1) o.cls = classify(o.m) == GC_DIAG1 ? GC_DIAG1 : GC_DIAG;
    }
}

template <class OpT>
void rec_common(OpT& t, const Op& o, const int* bit_of, int gen, int slot) {
    t.kind = o.kind;
    t.cls = o.cls;
    t.tq = o.t;
    t.tb = bit_of ? bit_of[o.t] : o.t;
    t.cq = o.c;
    t.cb = o.c >= 0 ? (bit_of ? bit_of[o.c] : o.c) : -1;
    t.pad0 = gen;
    t.pad1 = slot;
}

// Device record of a lowered op: FP32 matrix (complex64) or double-float pairs (complex128).
template <class OpT> OpT make_rec(const Op& o, const int* bit_of, int gen, int slot);
template <> TileOp<float> make_rec<TileOp<float>>(const Op& o, const int* bit_of, int gen, int slot) {
    TileOp<float> t{};
    rec_common(t, o, bit_of, gen, slot);
    for (int j = 0; j < 8; ++j) t.m[j] = (float)o.m[j];
    return t;
}
template <> TileOpDF make_rec<TileOpDF>(const Op& o, const int* bit_of, int gen, int slot) {
    TileOpDF t{};
    rec_common(t, o, bit_of, gen, slot);
    for (int j = 0; j < 8; ++j) split_to_floats(o.m[j], t.c[2 * j], t.c[2 * j + 1]);
    return t;
}

std::vector<long long> signature(const qs_instance& in) {
    std::vector<long long> s;
    s.push_back(in.n);
    s.push_back(in.n_params);
    for (int j = 0; j < in.n_gates; ++j) {
        const qs_gate& g = in.gates[j];
        s.push_back(g.kind);
        s.push_back(g.t);
        s.push_back(g.c);
        s.push_back(g.param);
        if (g.kind == QS_G_U1 || g.kind == QS_G_CU) s.push_back(classify(g.m));
    }
    for (int j = 0; j < in.n_terms; ++j) {
        s.push_back(100 + in.terms[j].kind);
        s.push_back(in.terms[j].q0);
        s.push_back(in.terms[j].q1);
    }
    return s;
}

struct Region { size_t off = 0, bytes = 0; };

struct Group {
    int n = 0;
    std::vector<int> members;
    std::vector<PassDesc> fwd, rev;
    std::vector<int> rev_nslot_used;
    int n_slots = 0, n_rot = 0;
    size_t fwd_per = 0, rev_per = 0;  // op records per instance
    // forward passes: per member, the length of the diagonal run that starts
    // there (0: a record of its own, or inside a run), the pass's record count,
    // and whether it holds runs
    std::vector<std::vector<int>> fwd_runs;
    std::vector<int> fwd_nrec;
    std::vector<char> fwd_dr;
    Region st_fwd, st_rev;            // in the staging / device op buffer
    std::vector<int> slot_rot;        // rev.size() * n_slots
    int* d_slot_rot = nullptr;
    void* phi = nullptr;
    void* lam = nullptr;
    double* d_part = nullptr;         // reverse partials: count * tiles * n_slots
    double* d_epart = nullptr;        // energy partials: count * eblocks
    int eblocks = 0;
    HGroup H{};
    double* d_tabs = nullptr;
    int* d_cross_q = nullptr;
    double* d_cross_c = nullptr;
    int* d_x_q = nullptr;
    double* d_x_c = nullptr;
    int b_fwd = 0, b_adj = 0;
    size_t rot_out = 0, e_out = 0;    // offsets into the result buffer (doubles)
};

}  // namespace
}  // namespace qs

struct qs_batch {
    qs_dtype dt;
    cudaStream_t user_stream = nullptr;
    cudaStream_t own_stream = nullptr;  // used when the caller passes the legacy default stream
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    int flags = 0;
    std::vector<qs_instance> inst;      // shallow copies (structure only)
    std::vector<std::vector<qs_gate>> gates;
    std::vector<std::vector<qs_term>> terms;
    std::vector<int> n_params;
    std::vector<size_t> param_off;
    size_t total_params = 0;
    // small instances
    std::vector<int> small;
    std::vector<qs::Region> small_fwd;  // per small instance, offsets (records) in the small op arrays
    size_t small_ops = 0;
    qs::Region st_small_fwd, st_small_rev;
    qs::SmallDesc* d_small = nullptr;
    qs_term* d_terms = nullptr;
    int* d_counter = nullptr;
    int small_nmax = 0;
    std::vector<qs::Group> groups;
    // op staging (pinned) and its device mirror
    unsigned char* h_stage = nullptr;
    unsigned char* d_stage = nullptr;
    size_t stage_bytes = 0;
    // results: rotation values and energies (device and pinned host)
    double* d_res = nullptr;
    double* h_res = nullptr;
    size_t res_doubles = 0;
    std::vector<size_t> rot_of_inst;     // offset of instance i's rotation values in the result
    std::vector<std::vector<int>> rot_param;  // instance i: parameter index of its r-th rotation (in gate order)
    std::vector<size_t> e_of_inst;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

namespace qs {
namespace {

cudaStream_t main_stream(qs_batch* b) { return b->own_stream ? b->own_stream : b->user_stream; }

// Fill the staging buffer with op records for the given angles (host work).
template <class Tr>
qs_status stage_ops(qs_batch* bt, const double* theta_all) {
    using OpT = typename Tr::Op;
    for (size_t si = 0; si < bt->small.size(); ++si) {
        const int idx = bt->small[si];
        qs_instance in = bt->inst[idx];
        if (theta_all) in.theta = theta_all + bt->param_off[idx];
        std::vector<Op> ops, rops;
        if (qs_status st = lower_instance(in, ops)) return st;
        reverse_ops(ops, rops);
        const Region& reg = bt->small_fwd[si];
        OpT* f = reinterpret_cast<OpT*>(bt->h_stage + bt->st_small_fwd.off) + reg.off;
        OpT* r = reinterpret_cast<OpT*>(bt->h_stage + bt->st_small_rev.off) + reg.off;
        int rot = 0;
        std::vector<int> rank(ops.size(), -1);
        for (size_t j = 0; j < ops.size(); ++j)
            if (rot_gen(in.gates[j].kind)) rank[j] = rot++;
        for (size_t j = 0; j < ops.size(); ++j) {
            f[j] = make_rec<OpT>(ops[j], nullptr, 0, -1);
            const size_t orig = ops.size() - 1 - j;
            const int gen = rot_gen(in.gates[orig].kind);
            r[j] = make_rec<OpT>(rops[j], nullptr, gen, gen ? rank[orig] : -1);
        }
    }
    for (Group& g : bt->groups) {
        for (size_t k = 0; k < g.members.size(); ++k) {
            const int idx = g.members[k];
            qs_instance in = bt->inst[idx];
            if (theta_all) in.theta = theta_all + bt->param_off[idx];
            std::vector<Op> ops, rops;
            if (qs_status st = lower_instance(in, ops)) return st;
            reverse_ops(ops, rops);
            OpT* f = reinterpret_cast<OpT*>(bt->h_stage + g.st_fwd.off) + k * g.fwd_per;
            size_t w = 0;
            std::vector<Op> pass_ops;
            std::vector<OpT> run_recs;
            for (size_t pi = 0; pi < g.fwd.size(); ++pi) {
                const PassDesc& d = g.fwd[pi];
                pass_ops.clear();
                for (int j : d.members) pass_ops.push_back(ops[j]);
                for (size_t i = 0; i < pass_ops.size();) {
                    const int len = g.fwd_runs[pi][i];
                    if (len > 0) {  // a diagonal run: the same records for every member, other factors
                        run_recs.clear();
                        diag_run_records(pass_ops, i, i + (size_t)len, d.bit_of, d.tp.b, run_recs);
                        for (const OpT& r : run_recs) f[w++] = r;
                        i += (size_t)len;
                    } else {
                        f[w++] = make_rec<OpT>(pass_ops[i], d.bit_of, 0, -1);
                        ++i;
                    }
                }
            }
            if (w != g.fwd_per) return fail(QS_EINVAL, "batch: forward records differ between members of a group");
            // reverse: a rotation's gradient goes to its slot within the pass
            OpT* r = reinterpret_cast<OpT*>(bt->h_stage + g.st_rev.off) + k * g.rev_per;
            w = 0;
            for (const PassDesc& d : g.rev) {
                int slot = 0;
                for (int j : d.members) {
                    const size_t orig = ops.size() - 1 - (size_t)j;
                    const int gen = rot_gen(in.gates[orig].kind);
                    r[w++] = make_rec<OpT>(rops[j], d.bit_of, gen, gen ? slot++ : -1);
                }
            }
        }
    }
    return QS_OK;
}

template <class Tr>
qs_status record(qs_batch* bt) {
    using T = typename Tr::G;
    using OpT = typename Tr::Op;
    cudaStream_t ms = main_stream(bt);
    QS_CUDA_TRY(cudaMemcpyAsync(bt->d_stage, bt->h_stage, bt->stage_bytes, cudaMemcpyHostToDevice, ms));
    QS_CUDA_TRY(cudaEventRecord(bt->events[0], ms));
    const int ns = (int)bt->streams.size();
    std::vector<char> forked(ns, 0);  // only streams that joined the fork are joined back
    // small instances: one persistent kernel on stream 0
    if (!bt->small.empty()) {
        cudaStream_t st = bt->streams[0];
        QS_CUDA_TRY(cudaStreamWaitEvent(st, bt->events[0], 0));
        forked[0] = 1;
        QS_CUDA_TRY(cudaMemsetAsync(bt->d_counter, 0, sizeof(int), st));
        const size_t smem = (size_t)2 * sizeof(T) << bt->small_nmax;
        int grid = std::min<int>((int)bt->small.size(), sm_count());
        k_batch_small<Tr><<<grid, kSmallThreads, smem, st>>>(
            bt->d_small, (int)bt->small.size(), reinterpret_cast<const OpT*>(bt->d_stage + bt->st_small_fwd.off),
            reinterpret_cast<const OpT*>(bt->d_stage + bt->st_small_rev.off), bt->d_terms, bt->d_res, bt->d_res,
            bt->d_counter);
        QS_CUDA_TRY(cudaGetLastError());
    }
    // groups round robin over the remaining streams
    for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
        Group& g = bt->groups[gi];
        cudaStream_t st = bt->streams[(gi + 1) % ns];
        if (!forked[(gi + 1) % ns]) QS_CUDA_TRY(cudaStreamWaitEvent(st, bt->events[0], 0));
        forked[(gi + 1) % ns] = 1;
        const uint64_t N = 1ull << g.n;
        const unsigned count = (unsigned)g.members.size();
        QS_CUDA_TRY(cudaMemsetAsync(g.phi, 0, sizeof(T) * N * count, st));
        k_set_zero_basis<T><<<(count + 127) / 128, 128, 0, st>>>((T*)g.phi, N, (int)count);
        QS_CUDA_TRY(cudaGetLastError());
        qs_state sv{};
        sv.n = g.n;
        sv.dt = bt->dt;
        sv.data = g.phi;
        sv.stream = st;
        size_t op0 = 0;
        const bool df = std::is_same<OpT, TileOpDF>::value;
        for (size_t fi = 0; fi < g.fwd.size(); ++fi) {
            const PassDesc& d = g.fwd[fi];
            TilePass tp = d.tp;
            tp.op0 = (int)op0;
            tp.nops = g.fwd_nrec[fi];
            tp.inst_stride = N;
            tp.ops_stride = (int)g.fwd_per;
            // double-float forward passes hand the state over as float pairs;
            // the last one leaves doubles for lambda = H psi and the reverse sweep
            tp.io = df ? ((fi > 0 ? kIoPairsIn : 0) | (fi + 1 < g.fwd.size() ? kIoPairsOut : 0)) : 0;
            if (g.fwd_dr[fi]) tp.io |= kIoDiagRuns;
            if (qs_status s = launch_tile_pass(&sv, bt->d_stage + g.st_fwd.off, tp, false, count)) return s;
            op0 += (size_t)g.fwd_nrec[fi];
        }
        // lambda = H psi, energy
        dim3 hg((unsigned)std::min<uint64_t>((N + 255) / 256, (uint64_t)sm_count() * 4), count);
        k_apply_h_b<T><<<hg, 256, 0, st>>>((const T*)g.phi, (T*)g.lam, N, g.H, g.d_tabs, g.d_cross_q, g.d_cross_c,
                                          g.d_x_q, g.d_x_c);
        dim3 eg((unsigned)g.eblocks, count);
        k_dot_b<T><<<eg, kRedThreadsB, 0, st>>>((const T*)g.phi, (const T*)g.lam, N, g.d_epart);
        k_sum_rows<<<(count + 127) / 128, 128, 0, st>>>(g.d_epart, (int)count, g.eblocks, bt->d_res + g.e_out);
        QS_CUDA_TRY(cudaGetLastError());
        // reverse sweep
        op0 = 0;
        for (size_t pi = 0; pi < g.rev.size(); ++pi) {
            const PassDesc& d = g.rev[pi];
            TilePass tp = d.tp;
            // phi and lambda tiles, the per-warp rotation slots, and the 2^(b - b0)
            // run offsets of this pass (sized per pass: 16 KiB for all 2^b would
            // leave room for only two CTAs per SM instead of three)
            const size_t smem = ((size_t)2 * sizeof(T) << tp.b) +
                                (size_t)g.n_slots * (kAdjThreads / 32) * sizeof(double) +
                                ((size_t)8 << (tp.b - tp.b0));
            tp.op0 = (int)op0;
            tp.nops = (int)d.members.size();
            tp.inst_stride = N;
            tp.ops_stride = (int)g.rev_per;
            // phi and lambda pass from one reverse pass to the next as float pairs
            // (double-float); after the last pass nothing reads them
            tp.io = (df && pi > 0 ? kIoPairsIn : 0) | (pi + 1 < g.rev.size() ? (df ? kIoPairsOut : 0) : kIoDiscard);
            const unsigned tiles = (unsigned)(1ull << (g.n - tp.b));
            const OpT* rops = reinterpret_cast<const OpT*>(bt->d_stage + g.st_rev.off);
            const dim3 grid(tiles, count);
            if (tp.b == 11) k_tile_adj<Tr, 11><<<grid, kAdjThreads, smem, st>>>((T*)g.phi, (T*)g.lam, rops, tp, g.d_part, g.n_slots);
            else if (tp.b == 12) k_tile_adj<Tr, 12><<<grid, kAdjThreads, smem, st>>>((T*)g.phi, (T*)g.lam, rops, tp, g.d_part, g.n_slots);
            else k_tile_adj<Tr, 0><<<grid, kAdjThreads, smem, st>>>((T*)g.phi, (T*)g.lam, rops, tp, g.d_part, g.n_slots);
            QS_CUDA_TRY(cudaGetLastError());
            if (g.rev_nslot_used[pi] > 0) {
                const int work = (int)count * g.n_slots;
                k_adj_finalize<<<(work + 127) / 128, 128, 0, st>>>(g.d_part, (int)tiles, g.n_slots, (int)count,
                                                                   g.d_slot_rot + pi * g.n_slots, bt->d_res + g.rot_out,
                                                                   g.n_rot);
                QS_CUDA_TRY(cudaGetLastError());
            }
            op0 += d.members.size();
        }
    }
    // join and read the results back
    for (int s = 0; s < ns; ++s) {
        if (!forked[s]) continue;
        QS_CUDA_TRY(cudaEventRecord(bt->events[1 + s], bt->streams[s]));
        QS_CUDA_TRY(cudaStreamWaitEvent(ms, bt->events[1 + s], 0));
    }
    QS_CUDA_TRY(cudaMemcpyAsync(bt->h_res, bt->d_res, bt->res_doubles * sizeof(double), cudaMemcpyDeviceToHost, ms));
    return QS_OK;
}

// Let a kernel use all the opt-in shared memory left beside its static shared memory.
template <class K>
qs_status allow_dynamic_smem(K* kernel) {
    cudaFuncAttributes a;
    QS_CUDA_TRY(cudaFuncGetAttributes(&a, kernel));
    QS_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(smem_optin() - a.sharedSizeBytes)));
    return QS_OK;
}

qs_status build_batch(qs_batch* bt) {
    const bool c128 = bt->dt == QS_C128;
    const size_t amp = c128 ? 16 : 8;
    const size_t rec_native = c128 ? sizeof(TileOpDF) : sizeof(TileOp<float>);
    const size_t rec_fwd = rec_native;
    // instances whose phi and lambda fit in one CTA's shared memory run whole in the persistent kernel
    int small_max = 0;
    while (small_max < 16 && ((size_t)2 * amp << (small_max + 1)) + 1024 <= smem_optin()) ++small_max;
    std::map<std::vector<long long>, int> by_sig;
    size_t res = 0;
    bt->rot_of_inst.assign(bt->inst.size(), 0);
    bt->e_of_inst.assign(bt->inst.size(), 0);
    bt->rot_param.assign(bt->inst.size(), {});
    for (size_t i = 0; i < bt->inst.size(); ++i) {
        const qs_instance& in = bt->inst[i];
        for (int j = 0; j < in.n_gates; ++j)
            if (rot_gen(in.gates[j].kind)) bt->rot_param[i].push_back(in.gates[j].param);
    }
    // result layout: energies first, then rotation values
    res = bt->inst.size();
    for (size_t i = 0; i < bt->inst.size(); ++i) bt->e_of_inst[i] = i;
    size_t small_rec = 0;
    std::vector<SmallDesc> sd;
    std::vector<qs_term> all_terms;
    for (size_t i = 0; i < bt->inst.size(); ++i) {
        const qs_instance& in = bt->inst[i];
        if (in.n <= small_max) {
            SmallDesc d{};
            d.n = in.n;
            d.n_ops = in.n_gates;
            d.op_off = (int)small_rec;
            d.n_terms = in.n_terms;
            d.term_off = (int)all_terms.size();
            d.rot_off = (int)res;
            d.e_out = (int)i;
            for (int j = 0; j < in.n_terms; ++j) all_terms.push_back(in.terms[j]);
            bt->rot_of_inst[i] = res;
            res += bt->rot_param[i].size();
            Region r;
            r.off = small_rec;
            small_rec += in.n_gates;
            bt->small.push_back((int)i);
            bt->small_fwd.push_back(r);
            bt->small_nmax = std::max(bt->small_nmax, in.n);
            sd.push_back(d);
            continue;
        }
        auto sig = signature(in);
        auto it = by_sig.find(sig);
        if (it == by_sig.end()) {
            by_sig[sig] = (int)bt->groups.size();
            bt->groups.emplace_back();
            bt->groups.back().n = in.n;
            it = by_sig.find(sig);
        }
        bt->groups[it->second].members.push_back((int)i);
    }
    // plans for every group (structure of its first member)
    size_t stage = 0;
    auto take = [&](size_t bytes) { size_t o = (stage + 255) & ~(size_t)255; stage = o + bytes; return o; };
    bt->small_ops = small_rec;
    bt->st_small_fwd.off = take(small_rec * rec_native);
    bt->st_small_rev.off = take(small_rec * rec_native);
    for (Group& g : bt->groups) {
        const qs_instance& in = bt->inst[g.members[0]];
        std::vector<Op> ops, rops;
        if (qs_status st = lower_instance(in, ops)) return st;
        reverse_ops(ops, rops);
        g.b_fwd = std::min(g.n, c128 ? 12 : 13);
        g.b_adj = std::min(g.n, c128 ? 11 : 12);
        const int b0 = std::min(4, std::max(0, g.b_adj - 3));
        if (qs_status st = plan_passes(g.n, ops, g.b_fwd, b0, true, 1, g.fwd)) return st;
        if (qs_status st = plan_passes(g.n, rops, g.b_adj, b0, true, 1, g.rev)) return st;
        for (const PassDesc& d : g.fwd)
            if (!d.tile) return fail(QS_EINVAL, "batch: a gate does not fit a tile");
        // diagonal runs of the forward passes (the RZ layers: phases on
        // consecutive qubits), found on the group's shared structure
        g.fwd_per = 0;
        g.fwd_runs.assign(g.fwd.size(), {});
        g.fwd_nrec.assign(g.fwd.size(), 0);
        g.fwd_dr.assign(g.fwd.size(), 0);
        {
            std::vector<Op> pass_ops;
            std::vector<TileOpDF> recs;
            for (size_t pi = 0; pi < g.fwd.size(); ++pi) {
                const PassDesc& d = g.fwd[pi];
                pass_ops.clear();
                for (int j : d.members) pass_ops.push_back(ops[j]);
                g.fwd_runs[pi].assign(pass_ops.size(), 0);
                for (size_t i = 0; i < pass_ops.size();) {
                    const size_t len = diag_run_length(pass_ops, i, d.bit_of, d.tp.b, bt->dt);
                    if (len > 0) {
                        recs.clear();
                        diag_run_records(pass_ops, i, i + len, d.bit_of, d.tp.b, recs);
                        g.fwd_runs[pi][i] = (int)len;
                        g.fwd_nrec[pi] += (int)recs.size();
                        g.fwd_dr[pi] = 1;
                        i += len;
                    } else {
                        g.fwd_nrec[pi] += 1;
                        ++i;
                    }
                }
                g.fwd_per += (size_t)g.fwd_nrec[pi];
            }
        }
        g.rev_per = rops.size();
        // rotation slots per reverse pass
        std::vector<int> rank(ops.size(), -1);
        int rot = 0;
        for (size_t j = 0; j < ops.size(); ++j)
            if (rot_gen(in.gates[j].kind)) rank[j] = rot++;
        g.n_rot = rot;
        g.n_slots = 1;
        for (const PassDesc& d : g.rev) {
            if (!d.tile) return fail(QS_EINVAL, "batch: a gate does not fit a tile");
            int c = 0;
            for (int j : d.members)
                if (rot_gen(in.gates[ops.size() - 1 - j].kind)) ++c;
            g.n_slots = std::max(g.n_slots, c);
        }
        if (g.n_slots > kMaxAdjSlots) return fail(QS_EINVAL, "batch: more than 1024 rotation gates in one reverse tile pass");
        g.slot_rot.assign(g.rev.size() * g.n_slots, -1);
        g.rev_nslot_used.assign(g.rev.size(), 0);
        for (size_t pi = 0; pi < g.rev.size(); ++pi) {
            int slot = 0;
            for (int j : g.rev[pi].members) {
                const size_t orig = ops.size() - 1 - j;
                if (rot_gen(in.gates[orig].kind)) g.slot_rot[pi * g.n_slots + slot++] = rank[orig];
            }
            g.rev_nslot_used[pi] = slot;
        }
        g.st_fwd.off = take(g.members.size() * g.fwd_per * rec_fwd);
        g.st_rev.off = take(g.members.size() * g.rev_per * rec_native);
        g.e_out = res;
        for (size_t k = 0; k < g.members.size(); ++k) bt->e_of_inst[g.members[k]] = res + k;
        res += g.members.size();
        g.rot_out = res;
        for (size_t k = 0; k < g.members.size(); ++k) bt->rot_of_inst[g.members[k]] = res + k * g.n_rot;
        res += g.members.size() * g.n_rot;
    }
    bt->stage_bytes = std::max<size_t>(stage, 256);
    bt->res_doubles = std::max<size_t>(res, 1);
    // allocations
    if (cudaMallocHost(&bt->h_stage, bt->stage_bytes) != cudaSuccess) { cudaGetLastError(); return fail(QS_ENOMEM, "batch: pinned staging"); }
    if (cudaMalloc(&bt->d_stage, bt->stage_bytes) != cudaSuccess) { cudaGetLastError(); return fail(QS_ENOMEM, "batch: device ops"); }
    if (cudaMallocHost(&bt->h_res, bt->res_doubles * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return fail(QS_ENOMEM, "batch: pinned results"); }
    if (cudaMalloc(&bt->d_res, bt->res_doubles * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return fail(QS_ENOMEM, "batch: device results"); }
    QS_CUDA_TRY(cudaMemset(bt->d_res, 0, bt->res_doubles * sizeof(double)));
    if (!bt->small.empty()) {
        if (cudaMalloc(&bt->d_small, sd.size() * sizeof(SmallDesc)) != cudaSuccess ||
            cudaMalloc(&bt->d_terms, std::max<size_t>(1, all_terms.size()) * sizeof(qs_term)) != cudaSuccess ||
            cudaMalloc(&bt->d_counter, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(QS_ENOMEM, "batch: small-instance tables");
        }
        QS_CUDA_TRY(cudaMemcpy(bt->d_small, sd.data(), sd.size() * sizeof(SmallDesc), cudaMemcpyHostToDevice));
        if (!all_terms.empty())
            QS_CUDA_TRY(cudaMemcpy(bt->d_terms, all_terms.data(), all_terms.size() * sizeof(qs_term), cudaMemcpyHostToDevice));
    }
    for (Group& g : bt->groups) {
        const uint64_t N = 1ull << g.n;
        const size_t count = g.members.size();
        const size_t tiles = (size_t)1 << (g.n - g.b_adj);
        g.eblocks = (int)std::min<uint64_t>((N + kRedThreadsB - 1) / kRedThreadsB, 64);
        // H tables per member
        const qs_instance& first = bt->inst[g.members[0]];
        g.H.lo_bits = (g.n + 1) / 2;
        const size_t nlo = (size_t)1 << g.H.lo_bits, nhi = (size_t)1 << (g.n - g.H.lo_bits);
        g.H.tab_stride = (int)(nlo + nhi);
        std::vector<int> cq, xq;
        for (int j = 0; j < first.n_terms; ++j) {
            const qs_term& t = first.terms[j];
            if (t.kind == QS_P_X) xq.push_back(t.q0);
            else if (t.kind == QS_P_ZZ) {
                const int a = std::min(t.q0, t.q1), b = std::max(t.q0, t.q1);
                if (a < g.H.lo_bits && b >= g.H.lo_bits) { cq.push_back(a); cq.push_back(b); }
            }
        }
        g.H.n_cross = (int)cq.size() / 2;
        g.H.n_x = (int)xq.size();
        if (g.H.n_cross > kMaxCrossB || g.H.n_x > kMaxXB) return fail(QS_EINVAL, "batch: observable has too many terms");
        std::vector<double> tabs(count * (nlo + nhi), 0.0), cc(std::max<size_t>(1, count * g.H.n_cross)),
            xc(std::max<size_t>(1, count * g.H.n_x));
        auto zs = [](uint64_t x, int q) { return ((x >> q) & 1ull) ? -1.0 : 1.0; };
        for (size_t k = 0; k < count; ++k) {
            const qs_instance& in = bt->inst[g.members[k]];
            double* lo = tabs.data() + k * (nlo + nhi);
            double* hi = lo + nlo;
            int ci = 0, xi = 0;
            for (int j = 0; j < in.n_terms; ++j) {
                const qs_term& t = in.terms[j];
                const int L = g.H.lo_bits;
                if (t.kind == QS_P_X) { xc[k * g.H.n_x + xi++] = t.coef; continue; }
                if (t.kind == QS_P_Z) {
                    if (t.q0 < L) for (size_t x = 0; x < nlo; ++x) lo[x] += t.coef * zs(x, t.q0);
                    else for (size_t x = 0; x < nhi; ++x) hi[x] += t.coef * zs(x, t.q0 - L);
                    continue;
                }
                const int a = std::min(t.q0, t.q1), b = std::max(t.q0, t.q1);
                if (b < L) for (size_t x = 0; x < nlo; ++x) lo[x] += t.coef * zs(x, a) * zs(x, b);
                else if (a >= L) for (size_t x = 0; x < nhi; ++x) hi[x] += t.coef * zs(x, a - L) * zs(x, b - L);
                else cc[k * g.H.n_cross + ci++] = t.coef;
            }
        }
        if (cudaMalloc(&g.phi, amp * N * count) != cudaSuccess || cudaMalloc(&g.lam, amp * N * count) != cudaSuccess ||
            cudaMalloc(&g.d_part, std::max<size_t>(1, count * tiles * g.n_slots) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&g.d_epart, count * g.eblocks * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&g.d_slot_rot, g.slot_rot.size() * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&g.d_tabs, tabs.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&g.d_cross_q, std::max<size_t>(1, cq.size()) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&g.d_cross_c, cc.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&g.d_x_q, std::max<size_t>(1, xq.size()) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&g.d_x_c, xc.size() * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(QS_ENOMEM, "batch: group buffers");
        }
        QS_CUDA_TRY(cudaMemcpy(g.d_slot_rot, g.slot_rot.data(), g.slot_rot.size() * sizeof(int), cudaMemcpyHostToDevice));
        QS_CUDA_TRY(cudaMemcpy(g.d_tabs, tabs.data(), tabs.size() * sizeof(double), cudaMemcpyHostToDevice));
        if (!cq.empty()) QS_CUDA_TRY(cudaMemcpy(g.d_cross_q, cq.data(), cq.size() * sizeof(int), cudaMemcpyHostToDevice));
        QS_CUDA_TRY(cudaMemcpy(g.d_cross_c, cc.data(), cc.size() * sizeof(double), cudaMemcpyHostToDevice));
        if (!xq.empty()) QS_CUDA_TRY(cudaMemcpy(g.d_x_q, xq.data(), xq.size() * sizeof(int), cudaMemcpyHostToDevice));
        QS_CUDA_TRY(cudaMemcpy(g.d_x_c, xc.data(), xc.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    // kernels that take more than 48 KiB of dynamic shared memory (set outside any graph capture)
    if (c128) {
        if (qs_status st = allow_dynamic_smem(k_batch_small<TrDF>)) return st;
        if (qs_status st = allow_dynamic_smem(k_tile_adj<TrDF, 0>)) return st;
        if (qs_status st = allow_dynamic_smem(k_tile_adj<TrDF, 11>)) return st;
        if (qs_status st = allow_dynamic_smem(k_tile_adj<TrDF, 12>)) return st;
    } else {
        if (qs_status st = allow_dynamic_smem(k_batch_small<TrF>)) return st;
        if (qs_status st = allow_dynamic_smem(k_tile_adj<TrF, 0>)) return st;
        if (qs_status st = allow_dynamic_smem(k_tile_adj<TrF, 11>)) return st;
        if (qs_status st = allow_dynamic_smem(k_tile_adj<TrF, 12>)) return st;
    }
    return QS_OK;
}

void free_batch(qs_batch* bt) {
    cudaStream_t ms = main_stream(bt);
    if (ms || bt->user_stream == nullptr) cudaStreamSynchronize(ms);
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    for (Group& g : bt->groups) {
        cudaFree(g.phi); cudaFree(g.lam); cudaFree(g.d_part); cudaFree(g.d_epart); cudaFree(g.d_slot_rot);
        cudaFree(g.d_tabs); cudaFree(g.d_cross_q); cudaFree(g.d_cross_c); cudaFree(g.d_x_q); cudaFree(g.d_x_c);
    }
    cudaFree(bt->d_small); cudaFree(bt->d_terms); cudaFree(bt->d_counter);
    cudaFree(bt->d_stage); cudaFree(bt->d_res);
    if (bt->h_stage) cudaFreeHost(bt->h_stage);
    if (bt->h_res) cudaFreeHost(bt->h_res);
    for (cudaStream_t s : bt->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : bt->events) cudaEventDestroy(e);
    if (bt->own_stream) cudaStreamDestroy(bt->own_stream);
}

qs_status check_instance(const qs_instance& in) {
    if (in.n < 1 || in.n > 30) return fail(QS_EINVAL, "batch instance: n must be in [1, 30]");
    if (in.n_gates < 0 || in.n_params < 0 || in.n_terms < 0) return fail(QS_EINVAL, "batch instance: negative count");
    if ((in.n_gates && !in.gates) || (in.n_params && !in.theta) || (in.n_terms && !in.terms))
        return fail(QS_EINVAL, "batch instance: NULL array");
    for (int j = 0; j < in.n_terms; ++j) {
        const qs_term& t = in.terms[j];
        if (t.kind != QS_P_Z && t.kind != QS_P_ZZ && t.kind != QS_P_X) return fail(QS_EINVAL, "unknown Pauli term kind");
        if (t.q0 < 0 || t.q0 >= in.n) return fail(QS_EINVAL, "term qubit out of range");
        if (t.kind == QS_P_ZZ && (t.q1 < 0 || t.q1 >= in.n || t.q1 == t.q0)) return fail(QS_EINVAL, "bad ZZ term");
    }
    std::vector<Op> ops;
    return lower_gates(in.gates, in.n_gates, in.theta, in.n_params, in.n, ops);
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_batch_create(const qs_instance* batch, int n_inst, qs_dtype dt, void* cuda_stream, int flags,
                          qs_batch** out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_inst < 1 || !batch) return fail(QS_EINVAL, "empty batch");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EDTYPE, "unknown dtype");
    for (int i = 0; i < n_inst; ++i)
        if (qs_status st = check_instance(batch[i])) return st;
    qs_batch* bt = new (std::nothrow) qs_batch();
    if (!bt) return fail(QS_ENOMEM, "host allocation failed");
    bt->dt = dt;
    bt->flags = flags;
    bt->user_stream = (cudaStream_t)cuda_stream;
    // copy the instances' structure and angles (the caller's arrays may go away)
    bt->gates.resize(n_inst);
    bt->terms.resize(n_inst);
    bt->param_off.resize(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        const qs_instance& in = batch[i];
        bt->gates[i].assign(in.gates, in.gates + in.n_gates);
        bt->terms[i].assign(in.terms, in.terms + in.n_terms);
        bt->param_off[i] = bt->total_params;
        bt->total_params += in.n_params;
    }
    bt->inst.resize(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        bt->inst[i] = batch[i];
        bt->inst[i].gates = bt->gates[i].data();
        bt->inst[i].terms = bt->terms[i].data();
        bt->n_params.push_back(batch[i].n_params);
    }
    qs_status st = QS_OK;
    auto cuda_ok = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && st == QS_OK) st = cuda_fail(e, what);
        return e == cudaSuccess;
    };
    if (bt->user_stream == nullptr) cuda_ok(cudaStreamCreateWithFlags(&bt->own_stream, cudaStreamNonBlocking), "stream");
    const int ns = 4;
    for (int s = 0; s < ns && st == QS_OK; ++s) {
        cudaStream_t x;
        if (cuda_ok(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "stream")) bt->streams.push_back(x);
    }
    for (int e = 0; e < ns + 1 && st == QS_OK; ++e) {
        cudaEvent_t x;
        if (cuda_ok(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "event")) bt->events.push_back(x);
    }
    if (st == QS_OK) st = build_batch(bt);
    // first staging with the angles given here (they are read now, not kept)
    if (st == QS_OK) st = dt == QS_C128 ? stage_ops<TrDF>(bt, nullptr) : stage_ops<TrF>(bt, nullptr);
    for (int i = 0; i < n_inst; ++i) bt->inst[i].theta = nullptr;
    if (st != QS_OK) {
        free_batch(bt);
        delete bt;
        return st;
    }
    *out = bt;
    return QS_OK;
}

qs_status qs_batch_execute(qs_batch* bt, const double* theta_all, double* energies, double* grads) {
    if (!bt) return fail(QS_EINVAL, "batch is NULL");
    if (!energies || (bt->total_params && !grads)) return fail(QS_EINVAL, "NULL output");
    cudaStream_t ms = main_stream(bt);
    if (theta_all) {
        for (size_t i = 0; i < bt->inst.size(); ++i) bt->inst[i].theta = theta_all + bt->param_off[i];
        qs_status st = bt->dt == QS_C128 ? stage_ops<TrDF>(bt, theta_all) : stage_ops<TrF>(bt, theta_all);
        for (size_t i = 0; i < bt->inst.size(); ++i) bt->inst[i].theta = nullptr;
        if (st != QS_OK) return st;
    }
    const bool use_graph = !(bt->flags & 1);
    if (use_graph) {
        if (!bt->gexec) {
            QS_CUDA_TRY(cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal));
            qs_status st = bt->dt == QS_C128 ? record<TrDF>(bt) : record<TrF>(bt);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(ms, &g);
            if (st != QS_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
            bt->graph = g;
            QS_CUDA_TRY(cudaGraphInstantiate(&bt->gexec, g, 0));
        }
        QS_CUDA_TRY(cudaGraphLaunch(bt->gexec, ms));
    } else {
        qs_status st = bt->dt == QS_C128 ? record<TrDF>(bt) : record<TrF>(bt);
        if (st != QS_OK) return st;
    }
    QS_CUDA_TRY(cudaStreamSynchronize(ms));
    for (size_t i = 0; i < bt->inst.size(); ++i) {
        energies[i] = bt->h_res[bt->e_of_inst[i]];
        double* gi = grads + bt->param_off[i];
        for (int p = 0; p < bt->n_params[i]; ++p) gi[p] = 0.0;
        const std::vector<int>& rp = bt->rot_param[i];
        for (size_t r = 0; r < rp.size(); ++r) gi[rp[r]] += bt->h_res[bt->rot_of_inst[i] + r];
    }
    return QS_OK;
}

qs_status qs_batch_stats(const qs_batch* bt, int* n_small, int* n_groups, int* n_launches) {
    if (!bt) return fail(QS_EINVAL, "batch is NULL");
    int launches = bt->small.empty() ? 0 : 1;
    for (const Group& g : bt->groups) {
        launches += 1 + (int)g.fwd.size() + 3 + (int)g.rev.size();
        for (int u : g.rev_nslot_used) launches += u > 0;
    }
    if (n_small) *n_small = (int)bt->small.size();
    if (n_groups) *n_groups = (int)bt->groups.size();
    if (n_launches) *n_launches = launches;
    return QS_OK;
}

qs_status qs_batch_destroy(qs_batch* bt) {
    if (!bt) return QS_OK;
    free_batch(bt);
    delete bt;
    return QS_OK;
}

qs_status qs_grad(const qs_instance* batch, int n_inst, qs_dtype dt, void* cuda_stream, double* energies,
                  double* grads) {
    if (n_inst == 0) return QS_OK;
    qs_batch* bt = nullptr;
    if (qs_status st = qs_batch_create(batch, n_inst, dt, cuda_stream, 1, &bt)) return st;
    qs_status st = qs_batch_execute(bt, nullptr, energies, grads);
    qs_batch_destroy(bt);
    return st;
}

}  // extern "C"
