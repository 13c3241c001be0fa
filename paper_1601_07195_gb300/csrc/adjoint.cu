// adjoint.cu -- energies and gradients of rotation angles by one reverse sweep
// (adjoint differentiation; T. Jones and J. Gacon, "Efficient calculation of
// gradients in classical simulations of variational quantum algorithms",
// arXiv:2009.02823).  Not in the paper.
//
// For psi = U_P .. U_1 |0..0>, U_j = exp(-i theta_j G_j / 2) for rotations:
//   lambda = H psi,  E = Re <psi|lambda>,  phi = psi;
//   for j = P .. 1:
//     if U_j is a rotation:  dE/dtheta_j += Im <lambda| G_j |phi>
//     phi <- U_j^dagger phi,  lambda <- U_j^dagger lambda.
// Each reverse step is one kernel that reads the pair of both states once,
// forms the FP64 gradient partial from the values before the update, and
// writes both updated pairs.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "device.cuh"

namespace qs {
namespace {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double red[32];
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        r = warp_sum_d(r);
    }
    return r;
}

// Im(conj(a) b) and Re(conj(a) b) in FP64
template <class T> __device__ __forceinline__ double im_cb(const T& a, const T& b) {
    return fma((double)a.x, (double)b.y, -(double)a.y * (double)b.x);
}
template <class T> __device__ __forceinline__ double re_cb(const T& a, const T& b) {
    return fma((double)a.x, (double)b.x, (double)a.y * (double)b.y);
}

// GEN: 0 = none, 1 = X, 2 = Y, 3 = Z.  MODE: 0 = single qubit, 1 = controlled, 2 = swap.
template <class R, int CLS, int MODE, int GEN>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_step(typename Amp<R>::T* __restrict__ phi,
                                                              typename Amp<R>::T* __restrict__ lam, uint64_t items,
                                                              int t, int c, Mat2<R> udag, double* partials) {
    using T = typename Amp<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * kAdjThreads;
    const int lo = min(t, c), hi = max(t, c);
    double acc = 0.0;
    for (uint64_t p = (uint64_t)blockIdx.x * kAdjThreads + threadIdx.x; p < items; p += stride) {
        uint64_t i0, i1;
        if (MODE == 0) { i0 = insert_zero(p, t); i1 = i0 | (1ull << t); }
        else if (MODE == 1) { i0 = insert_two_zeros(p, lo, hi) | (1ull << c); i1 = i0 | (1ull << t); }
        else { const uint64_t i = insert_two_zeros(p, lo, hi); i0 = i | (1ull << t); i1 = i | (1ull << c); }
        T f0 = phi[i0], f1 = phi[i1], l0 = lam[i0], l1 = lam[i1];
        if (GEN == 1) acc += im_cb(l0, f1) + im_cb(l1, f0);
        else if (GEN == 2) acc += re_cb(l1, f0) - re_cb(l0, f1);
        else if (GEN == 3) acc += im_cb(l0, f0) - im_cb(l1, f1);
        pair_update<CLS>(udag.v, f0, f1);
        pair_update<CLS>(udag.v, l0, l1);
        phi[i0] = f0; phi[i1] = f1; lam[i0] = l0; lam[i1] = l1;
    }
    if (GEN != 0) {
        const double s = block_sum_d(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

// lambda_i = e(i) psi_i + sum_q h_q psi_{i xor 2^q};  e(i) from the lo/hi tables.
struct XList { int count; int q[64]; double h[64]; };
struct ZZCross { int count; int a[64]; int b[64]; double coef[64]; };

template <class T>
__global__ void k_apply_h(const T* __restrict__ psi, T* __restrict__ lam, uint64_t N, int lo_bits,
                          const double* __restrict__ lo_tab, const double* __restrict__ hi_tab, ZZCross cross,
                          XList xs) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t lo_mask = (1ull << lo_bits) - 1ull;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        double e = lo_tab[i & lo_mask] + hi_tab[i >> lo_bits];
        for (int k = 0; k < cross.count; ++k) {
            const uint64_t par = ((i >> cross.a[k]) ^ (i >> cross.b[k])) & 1ull;
            e += par ? -cross.coef[k] : cross.coef[k];
        }
        const T v = psi[i];
        double ox = e * (double)v.x, oy = e * (double)v.y;
        for (int k = 0; k < xs.count; ++k) {
            const T w = psi[i ^ (1ull << xs.q[k])];
            ox = fma(xs.h[k], (double)w.x, ox);
            oy = fma(xs.h[k], (double)w.y, oy);
        }
        T o;
        o.x = (decltype(o.x))ox;
        o.y = (decltype(o.y))oy;
        lam[i] = o;
    }
}

template <class T>
__global__ void __launch_bounds__(kAdjThreads) k_dot_re(const T* __restrict__ a, const T* __restrict__ b, uint64_t N,
                                                        double* partials) {
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kAdjThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kAdjThreads + threadIdx.x; i < N; i += stride) acc += re_cb(a[i], b[i]);
    const double s = block_sum_d(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out[k] = sum over blocks of partials[k * n_blocks + b], block order fixed.
__global__ void k_finalize_rows(const double* __restrict__ partials, int n_rows, int n_blocks, double* out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_rows; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < n_blocks; ++b) s += partials[(size_t)k * n_blocks + b];
        out[k] = s;
    }
}

int adj_blocks(uint64_t items) {
    const uint64_t cap = (uint64_t)sm_count() * 8;
    uint64_t b = (items + kAdjThreads - 1) / kAdjThreads;
    if (b > cap) b = cap;
    return b ? (int)b : 1;
}

void dagger(const double m[8], double d[8]) {
    // (q11, q12, q21, q22)^dagger = (conj q11, conj q21, conj q12, conj q22)
    d[0] = m[0]; d[1] = -m[1];
    d[2] = m[4]; d[3] = -m[5];
    d[4] = m[2]; d[5] = -m[3];
    d[6] = m[6]; d[7] = -m[7];
}

template <class R, int CLS, int MODE>
cudaError_t step_gen(int gen, cudaStream_t st, void* phi, void* lam, uint64_t items, int t, int c, const Mat2<R>& u,
                     double* part, int blocks) {
    using T = typename Amp<R>::T;
    T* f = (T*)phi;
    T* l = (T*)lam;
    switch (gen) {
    case 1: k_adjoint_step<R, CLS, MODE, 1><<<blocks, kAdjThreads, 0, st>>>(f, l, items, t, c, u, part); break;
    case 2: k_adjoint_step<R, CLS, MODE, 2><<<blocks, kAdjThreads, 0, st>>>(f, l, items, t, c, u, part); break;
    case 3: k_adjoint_step<R, CLS, MODE, 3><<<blocks, kAdjThreads, 0, st>>>(f, l, items, t, c, u, part); break;
    default: k_adjoint_step<R, CLS, MODE, 0><<<blocks, kAdjThreads, 0, st>>>(f, l, items, t, c, u, part); break;
    }
    return cudaGetLastError();
}

template <class R, int MODE>
cudaError_t step_cls(int cls, int gen, cudaStream_t st, void* phi, void* lam, uint64_t items, int t, int c,
                     const Mat2<R>& u, double* part, int blocks) {
    switch (cls) {
    case GC_GENERAL: return step_gen<R, GC_GENERAL, MODE>(gen, st, phi, lam, items, t, c, u, part, blocks);
    case GC_REAL: return step_gen<R, GC_REAL, MODE>(gen, st, phi, lam, items, t, c, u, part, blocks);
    case GC_DIAG: return step_gen<R, GC_DIAG, MODE>(gen, st, phi, lam, items, t, c, u, part, blocks);
    case GC_DIAG1: return step_gen<R, GC_DIAG1, MODE>(gen, st, phi, lam, items, t, c, u, part, blocks);
    case GC_ANTIDIAG: return step_gen<R, GC_ANTIDIAG, MODE>(gen, st, phi, lam, items, t, c, u, part, blocks);
    default: return step_gen<R, GC_PERM, MODE>(gen, st, phi, lam, items, t, c, u, part, blocks);
    }
}

template <class R>
cudaError_t launch_step(const Op& op, int gen, cudaStream_t st, int n, void* phi, void* lam, double* part, int blocks) {
    double d[8];
    dagger(op.m, d);
    Mat2<R> u;
    for (int j = 0; j < 8; ++j) u.v[j] = (R)d[j];
    const uint64_t N = 1ull << n;
    if (op.kind == OP_SWAP) return step_gen<R, GC_PERM, 2>(0, st, phi, lam, N >> 2, op.t, op.c, u, part, blocks);
    const int cls = classify(d);
    if (op.kind == OP_CU) return step_cls<R, 1>(cls, 0, st, phi, lam, N >> 2, op.t, op.c, u, part, blocks);
    return step_cls<R, 0>(cls, gen, st, phi, lam, N >> 1, op.t, op.t, u, part, blocks);
}

// Host-side split of the diagonal part of H into lo/hi tables (as in reduce.cu).
struct HTables {
    int lo_bits = 0;
    std::vector<double> lo, hi;
    ZZCross cross{};
    XList xs{};
};

qs_status build_h(int n, const qs_term* terms, int nt, HTables& h) {
    h.lo_bits = (n + 1) / 2;
    const int hb = n - h.lo_bits;
    h.lo.assign((size_t)1 << h.lo_bits, 0.0);
    h.hi.assign((size_t)1 << hb, 0.0);
    auto zs = [](uint64_t x, int q) { return ((x >> q) & 1ull) ? -1.0 : 1.0; };
    for (int j = 0; j < nt; ++j) {
        const qs_term& t = terms[j];
        if (t.q0 < 0 || t.q0 >= n) return fail(QS_EINVAL, "term qubit out of range");
        if (t.kind == QS_P_X) {
            if (h.xs.count >= 64) return fail(QS_EINVAL, "at most 64 X terms per observable");
            h.xs.q[h.xs.count] = t.q0;
            h.xs.h[h.xs.count++] = t.coef;
        } else if (t.kind == QS_P_Z) {
            if (t.q0 < h.lo_bits) for (size_t x = 0; x < h.lo.size(); ++x) h.lo[x] += t.coef * zs(x, t.q0);
            else for (size_t x = 0; x < h.hi.size(); ++x) h.hi[x] += t.coef * zs(x, t.q0 - h.lo_bits);
        } else if (t.kind == QS_P_ZZ) {
            if (t.q1 < 0 || t.q1 >= n || t.q1 == t.q0) return fail(QS_EINVAL, "bad ZZ term");
            const int a = std::min(t.q0, t.q1), b = std::max(t.q0, t.q1);
            if (b < h.lo_bits) for (size_t x = 0; x < h.lo.size(); ++x) h.lo[x] += t.coef * zs(x, a) * zs(x, b);
            else if (a >= h.lo_bits) for (size_t x = 0; x < h.hi.size(); ++x) h.hi[x] += t.coef * zs(x, a - h.lo_bits) * zs(x, b - h.lo_bits);
            else {
                if (h.cross.count >= 64) return fail(QS_EINVAL, "too many ZZ terms straddling the qubit split");
                h.cross.a[h.cross.count] = a;
                h.cross.b[h.cross.count] = b;
                h.cross.coef[h.cross.count++] = t.coef;
            }
        } else {
            return fail(QS_EINVAL, "unknown Pauli term kind");
        }
    }
    return QS_OK;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes); }
};

template <class R>
qs_status grad_one(const qs_instance& in, cudaStream_t st, qs_dtype dt, void* phi, void* lam, double* d_part,
                   double* d_tab, double* d_out, double* h_pinned, double* energy, double* grads) {
    using T = typename Amp<R>::T;
    const int n = in.n;
    const uint64_t N = 1ull << n;
    std::vector<Op> ops;
    if (qs_status s = lower_gates(in.gates, in.n_gates, in.theta, in.n_params, n, ops)) return s;
    HTables h;
    if (qs_status s = build_h(n, in.terms, in.n_terms, h)) return s;
    // forward: psi = U_P .. U_1 |0>, fused plan on phi
    qs_state* s = nullptr;
    if (qs_status e = qs_wrap(phi, n, dt, st, &s)) return e;
    qs_status stt = qs_init_basis(s, 0);
    qs_plan* plan = nullptr;
    if (stt == QS_OK) stt = qs_plan_create(s, in.gates, in.n_gates, in.theta, in.n_params, QS_PLAN_DEFAULT, 0, &plan);
    if (stt == QS_OK) stt = qs_plan_execute(plan);
    if (stt != QS_OK) { qs_plan_destroy(plan); qs_destroy(s); return stt; }
    // lambda = H psi
    double* d_lo = d_tab;
    double* d_hi = d_tab + h.lo.size();
    QS_CUDA_TRY(cudaMemcpyAsync(d_lo, h.lo.data(), h.lo.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    QS_CUDA_TRY(cudaMemcpyAsync(d_hi, h.hi.data(), h.hi.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    int blocks = adj_blocks(N);
    k_apply_h<T><<<blocks, kAdjThreads, 0, st>>>((const T*)phi, (T*)lam, N, h.lo_bits, d_lo, d_hi, h.cross, h.xs);
    QS_CUDA_TRY(cudaGetLastError());
    // E = Re <psi|lambda>   (row 0 of the partials)
    k_dot_re<T><<<blocks, kAdjThreads, 0, st>>>((const T*)phi, (const T*)lam, N, d_part);
    QS_CUDA_TRY(cudaGetLastError());
    // reverse sweep; rotation j writes its partials into row 1 + (its rank among rotations)
    std::vector<int> rot_param;
    for (int j = (int)ops.size() - 1; j >= 0; --j) {
        const qs_gate& g = in.gates[j];
        int gen = 0;
        if (g.kind == QS_G_RX) gen = 1;
        else if (g.kind == QS_G_RY) gen = 2;
        else if (g.kind == QS_G_RZ) gen = 3;
        const uint64_t items = ops[j].kind == OP_1Q ? (N >> 1) : (N >> 2);
        const int sb = adj_blocks(items);
        double* row = d_part + (size_t)(1 + rot_param.size()) * blocks;
        if (gen) rot_param.push_back(g.param);
        cudaError_t e = launch_step<R>(ops[j], gen, st, n, phi, lam, row, sb);
        if (e != cudaSuccess) { qs_plan_destroy(plan); qs_destroy(s); return cuda_fail(e, "adjoint step launch"); }
        // all rows use the same width: pad rows of narrower steps with zeros
        if (gen && sb < blocks) QS_CUDA_TRY(cudaMemsetAsync(row + sb, 0, (size_t)(blocks - sb) * sizeof(double), st));
    }
    const int rows = 1 + (int)rot_param.size();
    k_finalize_rows<<<(rows + 127) / 128, 128, 0, st>>>(d_part, rows, blocks, d_out);
    QS_CUDA_TRY(cudaGetLastError());
    QS_CUDA_TRY(cudaMemcpyAsync(h_pinned, d_out, rows * sizeof(double), cudaMemcpyDeviceToHost, st));
    QS_CUDA_TRY(cudaStreamSynchronize(st));
    qs_plan_destroy(plan);
    qs_destroy(s);
    *energy = h_pinned[0];
    for (int p = 0; p < in.n_params; ++p) grads[p] = 0.0;
    for (size_t r = 0; r < rot_param.size(); ++r) grads[rot_param[r]] += h_pinned[1 + r];
    return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_grad(const qs_instance* batch, int n_inst, qs_dtype dt, void* cuda_stream, double* energies,
                             double* grads) {
    if (n_inst < 0 || (n_inst > 0 && (!batch || !energies))) return fail(QS_EINVAL, "bad batch arguments");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EDTYPE, "unknown dtype");
    int nmax = 0;
    size_t max_rot = 0, total_params = 0;
    for (int i = 0; i < n_inst; ++i) {
        const qs_instance& in = batch[i];
        if (in.n < 1 || in.n > 34) return fail(QS_EINVAL, "instance qubit count out of range");
        if (in.n_gates < 0 || in.n_params < 0 || in.n_terms < 0) return fail(QS_EINVAL, "negative count");
        if ((in.n_gates && !in.gates) || (in.n_params && !in.theta) || (in.n_terms && !in.terms))
            return fail(QS_EINVAL, "NULL array in instance");
        size_t rot = 0;
        for (int j = 0; j < in.n_gates; ++j) {
            const int k = in.gates[j].kind;
            if (k == QS_G_RX || k == QS_G_RY || k == QS_G_RZ) ++rot;
        }
        max_rot = std::max(max_rot, rot);
        nmax = std::max(nmax, in.n);
        total_params += in.n_params;
    }
    if (total_params && !grads) return fail(QS_EINVAL, "grads is NULL");
    if (n_inst == 0) return QS_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t amp = amp_bytes(dt);
    const int blocks = adj_blocks(1ull << nmax);
    const size_t rows = 1 + max_rot;
    const size_t tab = ((size_t)1 << ((nmax + 1) / 2)) + ((size_t)1 << (nmax / 2)) + 2;
    DevBuf phi, lam, part, dtab, dout;
    if (phi.alloc(amp << nmax) != cudaSuccess || lam.alloc(amp << nmax) != cudaSuccess ||
        part.alloc(rows * blocks * sizeof(double)) != cudaSuccess || dtab.alloc(tab * sizeof(double)) != cudaSuccess ||
        dout.alloc(rows * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "qs_grad: device allocation failed");
    }
    double* h_pinned = nullptr;
    if (cudaMallocHost(&h_pinned, rows * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "qs_grad: pinned allocation failed");
    }
    size_t goff = 0;
    qs_status st_all = QS_OK;
    for (int i = 0; i < n_inst && st_all == QS_OK; ++i) {
        st_all = dt == QS_C128
                     ? grad_one<double>(batch[i], st, dt, phi.p, lam.p, (double*)part.p, (double*)dtab.p,
                                        (double*)dout.p, h_pinned, &energies[i], grads + goff)
                     : grad_one<float>(batch[i], st, dt, phi.p, lam.p, (double*)part.p, (double*)dtab.p,
                                       (double*)dout.p, h_pinned, &energies[i], grads + goff);
        goff += batch[i].n_params;
    }
    cudaStreamSynchronize(st);
    cudaFreeHost(h_pinned);
    return st_all;
}
