// tile.cu -- gate fusion through a shared-memory tile (Section 4.4, Fig. 5).
//
// The paper iterates over blocks of 2^l_c consecutive amplitudes that stay in
// the last-level cache while every gate of a run with k < l_c is applied.  On
// the GPU one CTA owns one tile of 2^b amplitudes in shared memory, and the
// tile need not be consecutive: its b tile bits are qubits 0..b0-1 (so global
// memory is read in contiguous runs of 2^b0 amplitudes) plus any b - b0 other
// qubits the planner picked for the pass.  Every gate whose mixing qubits are
// tile bits is applied in shared memory; diagonal gates (T, phase, RZ,
// controlled phase) on qubits outside the tile are a per-tile constant factor,
// and controls outside the tile are a per-tile predicate.  One pass therefore
// reads and writes the state once for the whole run of gates.
#include "device.cuh"

namespace qs {

namespace {

constexpr int kTileThreads = 512;

template <class R, int CLS>
__device__ __forceinline__ void tile_1q(typename Amp<R>::T* sm, uint32_t N, int tb, const R* m) {
    using T = typename Amp<R>::T;
    for (uint32_t p = threadIdx.x; p < (N >> 1); p += kTileThreads) {
        const uint32_t i0 = insert_zero32(p, tb), i1 = i0 | (1u << tb);
        T a, b;
        if (CLS != GC_DIAG1) a = sm[i0];
        b = sm[i1];
        pair_update<CLS>(m, a, b);
        if (CLS != GC_DIAG1) sm[i0] = a;
        sm[i1] = b;
    }
}

template <class R, int CLS>
__device__ __forceinline__ void tile_cu(typename Amp<R>::T* sm, uint32_t N, int cb, int tb, const R* m) {
    using T = typename Amp<R>::T;
    const int lo = min(cb, tb), hi = max(cb, tb);
    for (uint32_t p = threadIdx.x; p < (N >> 2); p += kTileThreads) {
        const uint32_t i0 = insert_two_zeros32(p, lo, hi) | (1u << cb), i1 = i0 | (1u << tb);
        T a, b;
        if (CLS != GC_DIAG1) a = sm[i0];
        b = sm[i1];
        pair_update<CLS>(m, a, b);
        if (CLS != GC_DIAG1) sm[i0] = a;
        sm[i1] = b;
    }
}

// Multiply the tile (or, with cb >= 0, the half whose tile bit cb is 1) by f.
template <class R>
__device__ __forceinline__ void tile_scale(typename Amp<R>::T* sm, uint32_t N, R fr, R fi, int cb) {
    if (cb < 0) {
        for (uint32_t e = threadIdx.x; e < N; e += kTileThreads) sm[e] = cmul(fr, fi, sm[e]);
    } else {
        for (uint32_t p = threadIdx.x; p < (N >> 1); p += kTileThreads) {
            const uint32_t e = insert_zero32(p, cb) | (1u << cb);
            sm[e] = cmul(fr, fi, sm[e]);
        }
    }
}

template <class R>
__device__ __forceinline__ void tile_swap(typename Amp<R>::T* sm, uint32_t N, int ab, int bb) {
    using T = typename Amp<R>::T;
    const int lo = min(ab, bb), hi = max(ab, bb);
    for (uint32_t p = threadIdx.x; p < (N >> 2); p += kTileThreads) {
        const uint32_t i = insert_two_zeros32(p, lo, hi);
        const T x = sm[i | (1u << ab)];
        sm[i | (1u << ab)] = sm[i | (1u << bb)];
        sm[i | (1u << bb)] = x;
    }
}

template <class R>
__device__ __forceinline__ void tile_pairs(typename Amp<R>::T* sm, uint32_t N, int cls, int cb, int tb, const R* m) {
    if (cb < 0) {
        switch (cls) {
        case GC_GENERAL: tile_1q<R, GC_GENERAL>(sm, N, tb, m); break;
        case GC_REAL: tile_1q<R, GC_REAL>(sm, N, tb, m); break;
        case GC_DIAG: tile_1q<R, GC_DIAG>(sm, N, tb, m); break;
        case GC_DIAG1: tile_1q<R, GC_DIAG1>(sm, N, tb, m); break;
        case GC_ANTIDIAG: tile_1q<R, GC_ANTIDIAG>(sm, N, tb, m); break;
        default: tile_1q<R, GC_PERM>(sm, N, tb, m); break;
        }
    } else {
        switch (cls) {
        case GC_GENERAL: tile_cu<R, GC_GENERAL>(sm, N, cb, tb, m); break;
        case GC_REAL: tile_cu<R, GC_REAL>(sm, N, cb, tb, m); break;
        case GC_DIAG: tile_cu<R, GC_DIAG>(sm, N, cb, tb, m); break;
        case GC_DIAG1: tile_cu<R, GC_DIAG1>(sm, N, cb, tb, m); break;
        case GC_ANTIDIAG: tile_cu<R, GC_ANTIDIAG>(sm, N, cb, tb, m); break;
        default: tile_cu<R, GC_PERM>(sm, N, cb, tb, m); break;
        }
    }
}

// Apply one op to the tile whose non-tile qubits are fixed by `base`.  Every
// branch depends only on the op and on base, so it is uniform over the CTA.
// Returns false when the op leaves this tile unchanged (no barrier needed).
template <class R>
__device__ __forceinline__ bool tile_apply(typename Amp<R>::T* sm, uint32_t N, const TileOp<R>& op, uint64_t base) {
    if (op.kind == OP_SWAP) {
        tile_swap<R>(sm, N, op.tb, op.cb);
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
        tile_scale<R>(sm, N, bit ? op.m[6] : op.m[0], bit ? op.m[7] : op.m[1], cb);
        return true;
    }
    tile_pairs<R>(sm, N, op.cls, cb, op.tb, op.m);
    return true;
}

template <class R>
__global__ void __launch_bounds__(kTileThreads) k_tile(typename Amp<R>::T* __restrict__ psi,
                                                       const TileOp<R>* __restrict__ ops, TilePass P) {
    using T = typename Amp<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int b = P.b, b0 = P.b0, nh = b - b0;
    const uint32_t N = 1u << b;
    uint64_t* hioff = reinterpret_cast<uint64_t*>(sm + N);
    const uint64_t base = deposit_bits((uint64_t)blockIdx.x, P.nontile_mask);
    for (uint32_t h = threadIdx.x; h < (1u << nh); h += kTileThreads) {
        uint64_t off = 0;
        for (int j = 0; j < nh; ++j)
            if ((h >> j) & 1u) off |= 1ull << P.hi_q[j];
        hioff[h] = off;
    }
    __syncthreads();
    const uint32_t lomask = (1u << b0) - 1u;
    for (uint32_t e = threadIdx.x; e < N; e += kTileThreads) sm[e] = psi[base + hioff[e >> b0] + (e & lomask)];
    __syncthreads();
    for (int g = 0; g < P.nops; ++g) {
        const TileOp<R> op = ops[P.op0 + g];
        if (tile_apply<R>(sm, N, op, base)) __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < N; e += kTileThreads) psi[base + hioff[e >> b0] + (e & lomask)] = sm[e];
}

template <class R>
cudaError_t launch_tile(qs_state* s, const void* d_ops, const TilePass& P) {
    const size_t smem = tile_smem_bytes(s->dt, P.b) + ((size_t)8 << (P.b - P.b0));
    static bool configured[2] = {false, false};
    const int which = sizeof(R) == 8 ? 1 : 0;
    if (!configured[which]) {
        cudaError_t e = cudaFuncSetAttribute(k_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin());
        if (e != cudaSuccess) return e;
        configured[which] = true;
    }
    const unsigned grid = (unsigned)(1ull << (s->n - P.b));
    k_tile<R><<<grid, kTileThreads, smem, s->stream>>>(reinterpret_cast<typename Amp<R>::T*>(s->data),
                                                       reinterpret_cast<const TileOp<R>*>(d_ops), P);
    return cudaGetLastError();
}

}  // namespace

size_t tile_smem_bytes(qs_dtype dt, int b) { return amp_bytes(dt) << b; }

qs_status launch_tile_pass(qs_state* s, const void* d_ops, const TilePass& pass, bool arith_f64) {
    if (tile_smem_bytes(s->dt, pass.b) + ((size_t)8 << (pass.b - pass.b0)) > smem_optin())
        return fail(QS_EINVAL, "tile does not fit in shared memory");
    cudaError_t e;
    if (s->dt == QS_C64) e = launch_tile<float>(s, d_ops, pass);
    else if (arith_f64) e = launch_tile<double>(s, d_ops, pass);
    else e = launch_tile_df(s, d_ops, pass);
    if (e != cudaSuccess) return cuda_fail(e, "tile kernel launch");
    return QS_OK;
}

}  // namespace qs
