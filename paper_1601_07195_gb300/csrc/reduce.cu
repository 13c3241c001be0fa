// reduce.cu -- FP64 reductions over a state: norm, single-qubit marginals,
// the probability vector, and Pauli-sum expectation values.  None of these is
// in the paper; they read the state once (2^n amplitudes).
//
// Determinism: every reduction writes one FP64 partial per block of a fixed
// grid and a second single-block kernel adds the partials in a fixed order, so
// repeated calls give bit-identical results.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "device.cuh"
#include "df.cuh"

namespace qs {
namespace {

constexpr int kRedThreads = 256;
constexpr int kChunkBits = 12;                       // marginal chunk: 2^12 amplitudes per block step
constexpr int kPerThread = 1 << (kChunkBits - 8);    // 16 amplitudes per thread per chunk

template <class T>
__device__ __forceinline__ double prob(const T& a) {
    const double x = (double)a.x, y = (double)a.y;
    return fma(x, x, y * y);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// ---- norm ---------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_norm(const T* __restrict__ psi, uint64_t N, double* partials) {
    __shared__ double red[32];
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kRedThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += stride) acc += prob(psi[i]);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out[k] = sum_b partials[b * stride + k] for k < count, in block order.
__global__ void k_finalize(const double* __restrict__ partials, int n_blocks, int stride, int count, double* out) {
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < n_blocks; ++b) s += partials[(size_t)b * stride + k];
        out[k] = s;
    }
}

// ---- marginals: P(bit k = 1) for all k in one pass ---------------------------
// A block step covers a chunk of 2^12 amplitudes: thread t reads amplitudes
// chunk_base + (r << 8) + t, r < 16.  Bits 0..7 of the index are the thread id,
// bits 8..11 are r, bits >= 12 the chunk index.  Each thread keeps its total,
// the partial sums over r with bit m of r set, and per chunk-index bit the sum
// of its chunk totals with that bit set; the block then folds the thread-id
// bits.  Output per block: n + 1 partials (marginals, then the total).
//
// Within a chunk, |alpha|^2 and the 16-term tree are formed in double-float
// arithmetic on the FP32 pipes (about 47 significant bits; df.cuh), and only
// the five tree results per chunk are rounded to FP64 and accumulated there.
// In FP64 throughout (two operations per amplitude for |alpha|^2 and 30
// additions per 16) the FP64 pipe, not HBM, bounded the kernel: 11.3 ms for the
// n = 30 complex128 state against 2.6 ms to read it.  A chunk that holds a
// component of magnitude 2^60 or more (whose square would leave the FP32
// range) takes the FP64 form; components below 2^-126 contribute nothing in
// the double-float form (at most 2^-96 over a 2^30-amplitude state).
//
// With a power-of-two grid, chunk ch = blockIdx.x + j * gridDim.x keeps the low
// log2(gridDim.x) bits of blockIdx.x, so those marginals come from the block's
// total and only the bits of j are tracked per chunk.

// |alpha|^2 as an unnormalised double-float pair
__device__ __forceinline__ dfl prob_df(const double2& a) {
    const dfl x = split_double_lean(a.x), y = split_double_lean(a.y);
    const float px = x.h * x.h, py = y.h * y.h;
    float e = fmaf(x.h, x.h, -px) + fmaf(y.h, y.h, -py);  // the squares' exact rounding errors
    e = fmaf(2.0f * x.h, x.l, e);                         // cross terms (lo^2 is below 2^-48 of the square)
    e = fmaf(2.0f * y.h, y.l, e);
    const dfl s = two_sum(px, py);
    return {s.h, s.l + e};
}
__device__ __forceinline__ dfl prob_df(const float2& a) {
    const float px = a.x * a.x, py = a.y * a.y;
    const float e = fmaf(a.x, a.x, -px) + fmaf(a.y, a.y, -py);
    const dfl s = two_sum(px, py);
    return {s.h, s.l + e};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = two_sum(a.h, b.h);
    return {s.h, s.l + (a.l + b.l)};
}
__device__ __forceinline__ double df_to_double(dfl v) {
    return float_to_double_bits_lean(v.h) + float_to_double_bits_lean(v.l);
}
// exponent field of the larger component, as an unsigned integer comparable across types
__device__ __forceinline__ unsigned big_exp(const double2& a) {
    return max((unsigned)__double2hiint(a.x) & 0x7FF00000u, (unsigned)__double2hiint(a.y) & 0x7FF00000u);
}
__device__ __forceinline__ unsigned big_exp(const float2& a) {
    return max((unsigned)__float_as_int(a.x) & 0x7F800000u, (unsigned)__float_as_int(a.y) & 0x7F800000u);
}
template <class T> struct BigExp;
template <> struct BigExp<double2> { static constexpr unsigned v = (1023u + 60u) << 20; };
template <> struct BigExp<float2> { static constexpr unsigned v = (127u + 60u) << 23; };

// The chunk tree: t[0..3] = sums over r with bit m of r set, t[4] = the total.
template <class V, class Add>
__device__ __forceinline__ void chunk_tree(const V* p, V* t, Add add) {
    V q[8], o[4];
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = add(p[2 * j], p[2 * j + 1]);
    t[0] = add(add(add(p[1], p[3]), add(p[5], p[7])), add(add(p[9], p[11]), add(p[13], p[15])));
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = add(q[2 * j], q[2 * j + 1]);
    t[1] = add(add(q[1], q[3]), add(q[5], q[7]));
    t[2] = add(o[1], o[3]);
    t[3] = add(o[2], o[3]);
    t[4] = add(add(o[0], o[1]), t[3]);
}
struct AddD {
    __device__ __forceinline__ double operator()(double a, double b) const { return a + b; }
};
struct AddDF {
    __device__ __forceinline__ dfl operator()(dfl a, dfl b) const { return df_add(a, b); }
};

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_marginals(const T* __restrict__ psi, int n, uint64_t n_chunks,
                                                           double* partials) {
    __shared__ double red[32];
    // per thread, the sums of its chunk totals over chunks whose index bit g + k
    // is set (k < nh - g), one row of kRedThreads doubles per bit
    extern __shared__ double hsum[];
    double tot = 0.0, rbit[4] = {0, 0, 0, 0};
    const int nh = n - kChunkBits;
    // the grid has 2^g blocks (a power of two, at most the chunk count): chunk
    // ch = blockIdx.x + j * 2^g has the block's bits below g and j's above
    const int g = __ffs(gridDim.x) - 1;
    const int nv = nh - g;
    for (int k = 0; k < nv; ++k) hsum[k * kRedThreads + threadIdx.x] = 0.0;
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint64_t base = ch << kChunkBits;
        T a[kPerThread];
        unsigned big = 0;
#pragma unroll
        for (int r = 0; r < kPerThread; ++r) {
            a[r] = psi[base + ((uint64_t)r << 8) + threadIdx.x];
            big = max(big, big_exp(a[r]));
        }
        double t[5];
        if (__any_sync(0xffffffffu, big >= BigExp<T>::v)) {
            double p[kPerThread];
#pragma unroll
            for (int r = 0; r < kPerThread; ++r) p[r] = prob(a[r]);
            chunk_tree<double>(p, t, AddD{});
        } else {
            dfl p[kPerThread], u[5];
#pragma unroll
            for (int r = 0; r < kPerThread; ++r) p[r] = prob_df(a[r]);
            chunk_tree<dfl>(p, u, AddDF{});
#pragma unroll
            for (int m = 0; m < 5; ++m) t[m] = df_to_double(u[m]);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) rbit[m] += t[m];
        const double s = t[4];
        tot += s;
        uint64_t j = ch >> g;
        for (int k = 0; j != 0; ++k, j >>= 1)
            if (j & 1ull) hsum[k * kRedThreads + threadIdx.x] += s;
    }
    double* out = partials + (size_t)blockIdx.x * (n + 1);
    for (int k = 0; k < 8; ++k) {
        const double v = block_sum(((threadIdx.x >> k) & 1u) ? tot : 0.0, red);
        if (threadIdx.x == 0) out[k] = v;
    }
    for (int m = 0; m < 4; ++m) {
        const double v = block_sum(rbit[m], red);
        if (threadIdx.x == 0) out[8 + m] = v;
    }
    for (int k = 0; k < nh; ++k) {
        // bits below g are the block's own: its total or nothing
        const double h = k < g ? (((blockIdx.x >> k) & 1u) ? tot : 0.0) : hsum[(k - g) * kRedThreads + threadIdx.x];
        const double v = block_sum(h, red);
        if (threadIdx.x == 0) out[kChunkBits + k] = v;
    }
    const double v = block_sum(tot, red);
    if (threadIdx.x == 0) out[n] = v;
}

// Small states (n < 12): one block, every thread keeps all n bit sums.
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_marginals_small(const T* __restrict__ psi, int n, double* out) {
    __shared__ double red[32];
    double acc[kChunkBits + 1];
#pragma unroll
    for (int k = 0; k <= kChunkBits; ++k) acc[k] = 0.0;
    const uint32_t N = 1u << n;
    for (uint32_t i = threadIdx.x; i < N; i += kRedThreads) {
        const double p = prob(psi[i]);
        acc[kChunkBits] += p;
#pragma unroll
        for (int k = 0; k < kChunkBits; ++k)
            if (k < n && ((i >> k) & 1u)) acc[k] += p;
    }
    for (int k = 0; k < n; ++k) {
        const double v = block_sum(acc[k], red);
        if (threadIdx.x == 0) out[k] = v;
    }
    const double v = block_sum(acc[kChunkBits], red);
    if (threadIdx.x == 0) out[n] = v;
}

// ---- probability vector ---------------------------------------------------------
template <class T>
__global__ void k_probs(const T* __restrict__ psi, uint64_t off, uint64_t cnt, double* out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) out[i] = prob(psi[off + i]);
}

// ---- diagonal part of a Pauli sum ---------------------------------------------------
// e(i) = lo_tab[i & lo_mask] + hi_tab[i >> lo_bits] + sum over cross terms
// (Z_q Z_r with q below the split and r above it) of coef * z_q(i) * z_r(i);
// z_q(i) = 1 - 2 bit_q(i).  Accumulates sum_i |alpha_i|^2 e(i).
struct CrossTerm { int q, r; double coef; };
constexpr int kMaxCross = 64;
struct CrossList { int count; CrossTerm t[kMaxCross]; };

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_expect_diag(const T* __restrict__ psi, uint64_t N, int lo_bits,
                                                             const double* __restrict__ lo_tab,
                                                             const double* __restrict__ hi_tab, CrossList cross,
                                                             double* partials) {
    __shared__ double red[32];
    double acc = 0.0;
    const uint64_t lo_mask = (1ull << lo_bits) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * kRedThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += stride) {
        double e = lo_tab[i & lo_mask] + hi_tab[i >> lo_bits];
        for (int c = 0; c < cross.count; ++c) {
            const uint64_t par = ((i >> cross.t[c].q) ^ (i >> cross.t[c].r)) & 1ull;
            e += par ? -cross.t[c].coef : cross.t[c].coef;
        }
        acc = fma(prob(psi[i]), e, acc);
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// <X_q> = sum over pairs (i0, i0 + 2^q) of 2 Re(conj(alpha_i0) alpha_i1)
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_expect_x(const T* __restrict__ psi, uint64_t n_pairs, int q,
                                                          double* partials) {
    __shared__ double red[32];
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kRedThreads;
    for (uint64_t p = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; p < n_pairs; p += stride) {
        const uint64_t i0 = insert_zero(p, q);
        const T a = psi[i0], b = psi[i0 | (1ull << q)];
        acc += 2.0 * fma((double)a.x, (double)b.x, (double)a.y * (double)b.y);
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

int reduce_blocks(uint64_t work) {
    const uint64_t cap = (uint64_t)sm_count() * 8;
    uint64_t b = (work + kRedThreads - 1) / kRedThreads;
    if (b > cap) b = cap;
    return b ? (int)b : 1;
}

qs_status sync_result(qs_state* s, const double* d_out, int count, double* host) {
    QS_CUDA_TRY(cudaMemcpyAsync(s->h_result, d_out, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    std::memcpy(host, s->h_result, count * sizeof(double));
    return QS_OK;
}

template <class T>
qs_status norm_impl(qs_state* s, double* out) {
    const uint64_t N = 1ull << s->n;
    const int blocks = reduce_blocks(N);
    if (qs_status st = ensure_scratch(s, blocks + 1, 1)) return st;
    k_norm<T><<<blocks, kRedThreads, 0, s->stream>>>((const T*)s->data, N, s->d_partials);
    k_finalize<<<1, 32, 0, s->stream>>>(s->d_partials, blocks, 1, 1, s->d_partials + blocks);
    QS_CUDA_TRY(cudaGetLastError());
    return sync_result(s, s->d_partials + blocks, 1, out);
}

// Grid of the marginal kernel: a power of two (its chunk-index bit bookkeeping
// needs one); at least one resident wave, and up to 1024 blocks while each
// still gets 64 chunks or more; at most the chunk count and `fit`.  Measured
// (marginals and norm): n = 30 complex128 3.37 ms with 1024 blocks, 3.76 with
// 512, 3.81 with 256; n = 26 0.30 ms with 256 blocks, 0.44 with 1024.
template <class T>
int marginal_blocks(uint64_t chunks, uint64_t fit) {
    static int per_sm = 0;  // resident blocks per SM (registers bound it); the same on every device here
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_marginals<T>, kRedThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            v = 0;
        }
        per_sm = v > 0 ? v : 1;
    }
    const uint64_t wave = (uint64_t)per_sm * (uint64_t)sm_count();
    uint64_t want = 1;
    while (want * 2 <= wave) want *= 2;                          // the largest power of two in one wave
    while (want * 2 <= 1024 && want * 2 * 64 <= chunks) want *= 2;  // more blocks while each keeps 64 chunks
    uint64_t b = 1;
    while (b * 2 <= chunks && b * 2 <= fit && b * 2 <= want) b *= 2;
    return (int)b;
}
// its dynamic shared memory: one row of per-thread sums per chunk-index bit above log2(blocks)
size_t marginal_smem(int n, int blocks) {
    int g = 0;
    while ((1 << (g + 1)) <= blocks) ++g;
    const int nv = n - kChunkBits - g;
    return nv > 0 ? (size_t)nv * kRedThreads * sizeof(double) : 0;
}

template <class T>
qs_status marginals_impl(qs_state* s, double* out_all) {
    const int n = s->n;
    if (n < kChunkBits) {
        if (qs_status st = ensure_scratch(s, n + 1, n + 1)) return st;
        k_marginals_small<T><<<1, kRedThreads, 0, s->stream>>>((const T*)s->data, n, s->d_partials);
        QS_CUDA_TRY(cudaGetLastError());
        return sync_result(s, s->d_partials, n + 1, out_all);
    }
    const uint64_t chunks = 1ull << (n - kChunkBits);
    const int blocks = marginal_blocks<T>(chunks, ~0ull);
    if (qs_status st = ensure_scratch(s, (size_t)blocks * (n + 1) + (n + 1), n + 1)) return st;
    double* fin = s->d_partials + (size_t)blocks * (n + 1);
    k_marginals<T><<<blocks, kRedThreads, marginal_smem(n, blocks), s->stream>>>((const T*)s->data, n, chunks,
                                                                                  s->d_partials);
    k_finalize<<<1, 64, 0, s->stream>>>(s->d_partials, blocks, n + 1, n + 1, fin);
    QS_CUDA_TRY(cudaGetLastError());
    return sync_result(s, fin, n + 1, out_all);
}

// Sign of Z-string term on basis index x: +1 / -1.
inline double zsign(uint64_t x, int q) { return ((x >> q) & 1ull) ? -1.0 : 1.0; }

template <class T>
qs_status expect_impl(qs_state* s, const qs_term* terms, int nt, double* out) {
    const int n = s->n;
    const uint64_t N = 1ull << n;
    const int lo_bits = (n + 1) / 2, hi_bits = n - lo_bits;
    const size_t nlo = (size_t)1 << lo_bits, nhi = (size_t)1 << hi_bits;
    std::vector<double> lo_tab(nlo, 0.0), hi_tab(nhi, 0.0);
    CrossList cross{};
    std::vector<const qs_term*> xs;
    bool any_diag = false;
    for (int j = 0; j < nt; ++j) {
        const qs_term& t = terms[j];
        if (t.kind == QS_P_X) { xs.push_back(&t); continue; }
        any_diag = true;
        if (t.kind == QS_P_Z) {
            if (t.q0 < lo_bits) for (size_t x = 0; x < nlo; ++x) lo_tab[x] += t.coef * zsign(x, t.q0);
            else for (size_t x = 0; x < nhi; ++x) hi_tab[x] += t.coef * zsign(x, t.q0 - lo_bits);
        } else {
            const int a = std::min(t.q0, t.q1), b = std::max(t.q0, t.q1);
            if (b < lo_bits) for (size_t x = 0; x < nlo; ++x) lo_tab[x] += t.coef * zsign(x, a) * zsign(x, b);
            else if (a >= lo_bits) for (size_t x = 0; x < nhi; ++x) hi_tab[x] += t.coef * zsign(x, a - lo_bits) * zsign(x, b - lo_bits);
            else {
                if (cross.count >= kMaxCross) return fail(QS_EINVAL, "too many Z_q Z_r terms straddling the qubit split");
                cross.t[cross.count++] = CrossTerm{a, b, t.coef};
            }
        }
    }
    const int blocks = reduce_blocks(N);
    const int n_red = (any_diag ? 1 : 0) + (int)xs.size();
    const size_t part = (size_t)blocks * n_red;
    const size_t need = part + n_red + (any_diag ? nlo + nhi : 0);
    if (qs_status st = ensure_scratch(s, need, n_red > 0 ? n_red : 1)) return st;
    double* d_fin = s->d_partials + part;
    double* d_lo = d_fin + n_red;
    double* d_hi = d_lo + nlo;
    int r = 0;
    if (any_diag) {
        QS_CUDA_TRY(cudaMemcpyAsync(d_lo, lo_tab.data(), nlo * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        QS_CUDA_TRY(cudaMemcpyAsync(d_hi, hi_tab.data(), nhi * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        k_expect_diag<T><<<blocks, kRedThreads, 0, s->stream>>>((const T*)s->data, N, lo_bits, d_lo, d_hi, cross,
                                                                s->d_partials);
        ++r;
    }
    for (const qs_term* t : xs) {
        k_expect_x<T><<<blocks, kRedThreads, 0, s->stream>>>((const T*)s->data, N >> 1, t->q0,
                                                             s->d_partials + (size_t)r * blocks);
        ++r;
    }
    QS_CUDA_TRY(cudaGetLastError());
    if (n_red == 0) { *out = 0.0; return QS_OK; }
    // per-term sums in fixed block order, then the coefficient-weighted total on the host
    for (int k = 0; k < n_red; ++k)
        k_finalize<<<1, 32, 0, s->stream>>>(s->d_partials + (size_t)k * blocks, blocks, 1, 1, d_fin + k);
    QS_CUDA_TRY(cudaGetLastError());
    std::vector<double> sums(n_red);
    if (qs_status st = sync_result(s, d_fin, n_red, sums.data())) return st;
    double e = any_diag ? sums[0] : 0.0;
    for (size_t k = 0; k < xs.size(); ++k) e += xs[k]->coef * sums[(any_diag ? 1 : 0) + k];
    *out = e;
    return QS_OK;
}

}  // namespace

qs_status ensure_scratch(qs_state* s, size_t partial_doubles, size_t result_doubles) {
    if (partial_doubles > s->partials_cap) {
        if (s->d_partials) { cudaStreamSynchronize(s->stream); cudaFree(s->d_partials); s->d_partials = nullptr; s->partials_cap = 0; }
        cudaError_t e = cudaMalloc(&s->d_partials, partial_doubles * sizeof(double));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(QS_ENOMEM, "reduction scratch allocation failed"); }
        s->partials_cap = partial_doubles;
    }
    if (result_doubles > s->h_result_cap) {
        if (s->h_result) { cudaStreamSynchronize(s->stream); cudaFreeHost(s->h_result); s->h_result = nullptr; s->h_result_cap = 0; }
        cudaError_t e = cudaMallocHost(&s->h_result, result_doubles * sizeof(double));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(QS_ENOMEM, "pinned result allocation failed"); }
        s->h_result_cap = result_doubles;
    }
    return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_norm(qs_state* s, double* out) {
    if (!s || !s->data || !out) return fail(QS_EINVAL, "NULL argument");
    return s->dt == QS_C128 ? norm_impl<double2>(s, out) : norm_impl<float2>(s, out);
}

qs_status qs_prob(qs_state* s, int k, double* p1) {
    if (!s || !s->data || !p1) return fail(QS_EINVAL, "NULL argument");
    if (k < -2 || k >= s->n) return fail(QS_EINVAL, "qubit out of range");
    std::vector<double> all(s->n + 1);
    qs_status st = s->dt == QS_C128 ? marginals_impl<double2>(s, all.data()) : marginals_impl<float2>(s, all.data());
    if (st != QS_OK) return st;
    if (k >= 0) p1[0] = all[k];
    else std::memcpy(p1, all.data(), (s->n + (k == -2 ? 1 : 0)) * sizeof(double));
    return QS_OK;
}

qs_status qs_probs(qs_state* s, double* host_out) {
    if (!s || !s->data || !host_out) return fail(QS_EINVAL, "NULL argument");
    const uint64_t N = 1ull << s->n;
    const uint64_t chunk = N < (1ull << 24) ? N : (1ull << 24);
    if (qs_status st = ensure_scratch(s, chunk, 1)) return st;
    for (uint64_t off = 0; off < N; off += chunk) {
        const int blocks = reduce_blocks(chunk);
        if (s->dt == QS_C128) k_probs<double2><<<blocks, kRedThreads, 0, s->stream>>>((const double2*)s->data, off, chunk, s->d_partials);
        else k_probs<float2><<<blocks, kRedThreads, 0, s->stream>>>((const float2*)s->data, off, chunk, s->d_partials);
        QS_CUDA_TRY(cudaGetLastError());
        QS_CUDA_TRY(cudaMemcpyAsync(host_out + off, s->d_partials, chunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    }
    return QS_OK;
}

qs_status qs_expect(qs_state* s, const qs_term* terms, int n_terms, double* out) {
    if (!s || !s->data || !out) return fail(QS_EINVAL, "NULL argument");
    if (n_terms < 0 || (n_terms > 0 && !terms)) return fail(QS_EINVAL, "bad term array");
    for (int j = 0; j < n_terms; ++j) {
        const qs_term& t = terms[j];
        if (t.kind != QS_P_Z && t.kind != QS_P_ZZ && t.kind != QS_P_X) return fail(QS_EINVAL, "unknown Pauli term kind");
        if (t.q0 < 0 || t.q0 >= s->n) return fail(QS_EINVAL, "term qubit out of range");
        if (t.kind == QS_P_ZZ && (t.q1 < 0 || t.q1 >= s->n || t.q1 == t.q0)) return fail(QS_EINVAL, "bad ZZ term");
    }
    return s->dt == QS_C128 ? expect_impl<double2>(s, terms, n_terms, out) : expect_impl<float2>(s, terms, n_terms, out);
}

}  // extern "C"

// ---- marginals without any allocation ----------------------------------------------
// Same kernels as qs_prob(k = -1), but the per-block partial sums live in this
// file-scope device array instead of memory from cudaMalloc.  Every loaded
// library instance holds it on every GPU that loads the module until exit.
namespace qs {
namespace {

constexpr int kStaticPartials = 16384;  // doubles (128 KiB)
constexpr int kStaticMaxQubits = 36;
static __device__ __align__(256) double g_static_partials[kStaticPartials];

std::mutex g_static_mu;
void* g_static_addr[64] = {nullptr};

// Device address of g_static_partials for the current device (with that device
// current).  In host code the symbol is only a host-side stand-in, so kernels
// must be given this address.  It is looked up afresh on every call whose
// stream is not capturing, so a context torn down and created again (which
// may place the array elsewhere) never leaves a stale address in use; during
// a capture the address from the last such call on the device is used, which
// is why the first call on a device must come before any capture.
qs_status static_scratch(cudaStream_t st, double** out) {
    int dev = 0;
    QS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(QS_EINVAL, "device ordinal out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    QS_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_addr[dev] = p;
    } else if (!g_static_addr[dev]) {
        return fail(QS_EINVAL, "qs_marginals_noalloc: the first call on a device must not be captured");
    }
    *out = (double*)g_static_addr[dev];
    return QS_OK;
}

template <class T>
qs_status marginals_noalloc_impl(const void* psi, int n, cudaStream_t st, double* dev_out) {
    if (n < kChunkBits) {
        k_marginals_small<T><<<1, kRedThreads, 0, st>>>((const T*)psi, n, dev_out);
        QS_CUDA_TRY(cudaGetLastError());
        return QS_OK;
    }
    double* scratch = nullptr;
    if (qs_status s = static_scratch(st, &scratch)) return s;
    const uint64_t chunks = 1ull << (n - kChunkBits);
    const int blocks = marginal_blocks<T>(chunks, (uint64_t)kStaticPartials / (uint64_t)(n + 1));
    // every partial the finalize kernel reads is written first by k_marginals, so
    // nothing left over from an earlier call is ever read
    k_marginals<T><<<blocks, kRedThreads, marginal_smem(n, blocks), st>>>((const T*)psi, n, chunks, scratch);
    k_finalize<<<1, 64, 0, st>>>(scratch, blocks, n + 1, n + 1, dev_out);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace
}  // namespace qs

extern "C" qs_status qs_marginals_noalloc(const void* dev_state, int n, qs_dtype dt, void* cuda_stream,
                                          double* dev_out) {
    using namespace qs;
    if (!dev_state || !dev_out) return fail(QS_EINVAL, "qs_marginals_noalloc: NULL pointer");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EDTYPE, "qs_marginals_noalloc: unknown dtype");
    if (n < 1 || n > kStaticMaxQubits)
        return fail(QS_EINVAL, "qs_marginals_noalloc: n must be in [1, 36]; larger states exceed what the "
                               "static 16384-double scratch array is sized for");
    if ((uintptr_t)dev_state % amp_bytes(dt) != 0 || (uintptr_t)dev_out % 8 != 0)
        return fail(QS_EINVAL, "qs_marginals_noalloc: misaligned pointer");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return dt == QS_C128 ? marginals_noalloc_impl<double2>(dev_state, n, st, dev_out)
                         : marginals_noalloc_impl<float2>(dev_state, n, st, dev_out);
}
