// tile_df.cu -- the fused tile pass of tile.cu for complex128 states with the
// gate arithmetic in double-float form (df.cuh) on the FP32 pipes.
//
// The tile is split into (hi, lo) float pairs once when it is loaded, every
// gate of the pass is applied to the pairs in shared memory, and the pairs are
// rounded back to doubles once when the tile is stored.  Layout, planner
// contract and control/diagonal handling are those of tile.cu (Section 4.4,
// Fig. 5, on a shared-memory tile over any qubit set).
#include "device.cuh"
#include "df.cuh"

namespace qs {
namespace {

#ifndef QS_TILE_DF_THREADS
#define QS_TILE_DF_THREADS 512
#endif
constexpr int kThreads = QS_TILE_DF_THREADS;

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

template <int CLS>
__device__ __forceinline__ void df_tile_1q(float4* sm, uint32_t N, int tb, const float* c) {
#pragma unroll 2
    for (uint32_t p = threadIdx.x; p < (N >> 1); p += kThreads) {
        const uint32_t i0 = insert_zero32(p, tb), i1 = i0 | (1u << tb);
        float4 a, b;
        if (CLS != GC_DIAG1) a = sm[i0];
        b = sm[i1];
        df_pair_update<CLS>(c, a, b);
        if (CLS != GC_DIAG1) sm[i0] = a;
        sm[i1] = b;
    }
}

template <int CLS>
__device__ __forceinline__ void df_tile_cu(float4* sm, uint32_t N, int cb, int tb, const float* c) {
    const int lo = min(cb, tb), hi = max(cb, tb);
#pragma unroll 2
    for (uint32_t p = threadIdx.x; p < (N >> 2); p += kThreads) {
        const uint32_t i0 = insert_two_zeros32(p, lo, hi) | (1u << cb), i1 = i0 | (1u << tb);
        float4 a, b;
        if (CLS != GC_DIAG1) a = sm[i0];
        b = sm[i1];
        df_pair_update<CLS>(c, a, b);
        if (CLS != GC_DIAG1) sm[i0] = a;
        sm[i1] = b;
    }
}

// Multiply the tile (or the half with tile bit cb = 1) by matrix entry q11
// (use22 = false) or q22 (use22 = true).
template <bool USE22>
__device__ __forceinline__ void df_tile_scale(float4* sm, uint32_t N, const float* c, int cb) {
    if (cb < 0) {
#pragma unroll 2
        for (uint32_t e = threadIdx.x; e < N; e += kThreads) sm[e] = USE22 ? df_cmul(c, 6, 7, sm[e]) : df_cmul(c, 0, 1, sm[e]);
    } else {
#pragma unroll 2
        for (uint32_t p = threadIdx.x; p < (N >> 1); p += kThreads) {
            const uint32_t e = insert_zero32(p, cb) | (1u << cb);
            sm[e] = USE22 ? df_cmul(c, 6, 7, sm[e]) : df_cmul(c, 0, 1, sm[e]);
        }
    }
}

__device__ __forceinline__ void df_tile_swap(float4* sm, uint32_t N, int ab, int bb) {
    const int lo = min(ab, bb), hi = max(ab, bb);
    for (uint32_t p = threadIdx.x; p < (N >> 2); p += kThreads) {
        const uint32_t i = insert_two_zeros32(p, lo, hi);
        const float4 x = sm[i | (1u << ab)];
        sm[i | (1u << ab)] = sm[i | (1u << bb)];
        sm[i | (1u << bb)] = x;
    }
}

__device__ __forceinline__ void df_tile_pairs(float4* sm, uint32_t N, int cls, int cb, int tb, const float* c) {
    if (cb < 0) {
        switch (cls) {
        case GC_GENERAL: df_tile_1q<GC_GENERAL>(sm, N, tb, c); break;
        case GC_REAL: df_tile_1q<GC_REAL>(sm, N, tb, c); break;
        case GC_DIAG: df_tile_1q<GC_DIAG>(sm, N, tb, c); break;
        case GC_DIAG1: df_tile_1q<GC_DIAG1>(sm, N, tb, c); break;
        case GC_ANTIDIAG: df_tile_1q<GC_ANTIDIAG>(sm, N, tb, c); break;
        default: df_tile_1q<GC_PERM>(sm, N, tb, c); break;
        }
    } else {
        switch (cls) {
        case GC_GENERAL: df_tile_cu<GC_GENERAL>(sm, N, cb, tb, c); break;
        case GC_REAL: df_tile_cu<GC_REAL>(sm, N, cb, tb, c); break;
        case GC_DIAG: df_tile_cu<GC_DIAG>(sm, N, cb, tb, c); break;
        case GC_DIAG1: df_tile_cu<GC_DIAG1>(sm, N, cb, tb, c); break;
        case GC_ANTIDIAG: df_tile_cu<GC_ANTIDIAG>(sm, N, cb, tb, c); break;
        default: df_tile_cu<GC_PERM>(sm, N, cb, tb, c); break;
        }
    }
}

__device__ __forceinline__ bool df_tile_apply(float4* sm, uint32_t N, const TileOpDF& op, uint64_t base) {
    if (op.kind == OP_SWAP) {
        df_tile_swap(sm, N, op.tb, op.cb);
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
        if (bit) df_tile_scale<true>(sm, N, op.c, cb);
        else df_tile_scale<false>(sm, N, op.c, cb);
        return true;
    }
    df_tile_pairs(sm, N, op.cls, cb, op.tb, op.c);
    return true;
}

__global__ void __launch_bounds__(kThreads) k_tile_df(double2* __restrict__ psi, const TileOpDF* __restrict__ ops,
                                                      TilePass P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sm = reinterpret_cast<float4*>(smem_raw);
    psi += (uint64_t)blockIdx.y * P.inst_stride;
    ops += (uint64_t)blockIdx.y * (uint64_t)P.ops_stride;
    const int b = P.b, b0 = P.b0, nh = b - b0;
    const uint32_t N = 1u << b;
    uint64_t* hioff = reinterpret_cast<uint64_t*>(sm + N);
    const uint64_t base = deposit_bits((uint64_t)blockIdx.x, P.nontile_mask);
    for (uint32_t h = threadIdx.x; h < (1u << nh); h += kThreads) {
        uint64_t off = 0;
        for (int j = 0; j < nh; ++j)
            if ((h >> j) & 1u) off |= 1ull << P.hi_q[j];
        hioff[h] = off;
    }
    __syncthreads();
    const uint32_t lomask = (1u << b0) - 1u;
    for (uint32_t e = threadIdx.x; e < N; e += kThreads) sm[e] = df_load(psi[base + hioff[e >> b0] + (e & lomask)]);
    __syncthreads();
    for (int g = 0; g < P.nops; ++g) {
        const TileOpDF op = ops[P.op0 + g];
        if (df_tile_apply(sm, N, op, base)) __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < N; e += kThreads) psi[base + hioff[e >> b0] + (e & lomask)] = df_store(sm[e]);
}

}  // namespace

void split_to_floats(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

cudaError_t launch_tile_df(qs_state* s, const void* d_ops, const TilePass& P, unsigned count) {
    const size_t smem = tile_smem_bytes(s->dt, P.b) + ((size_t)8 << (P.b - P.b0));
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((unsigned)(1ull << (s->n - P.b)), count);
    k_tile_df<<<grid, kThreads, smem, s->stream>>>(reinterpret_cast<double2*>(s->data),
                                                   reinterpret_cast<const TileOpDF*>(d_ops), P);
    return cudaGetLastError();
}

}  // namespace qs
