// tile_df.cu -- the fused tile pass of tile.cu for complex128 states with the
// gate arithmetic in double-float form (df.cuh) on the FP32 pipes.
//
// The tile is split into (hi, lo) float pairs when it is loaded, every gate of
// the pass is applied to the pairs in shared memory, and the pairs are rounded
// back to doubles when the tile is stored; between consecutive passes of a
// plan the state stays in HBM as float pairs instead (TilePass::io), so the
// split and the join run once per run of passes.  Planner contract and
// control/diagonal handling are those of tile.cu (Section 4.4, Fig. 5, on a
// shared-memory tile over any qubit set); the tile's shared-memory layout
// spreads the partners of gates on the lowest tile bits over all banks.
#include <cstring>
#include <type_traits>

#include "device.cuh"
#include "df.cuh"
#include "tile_df_ops.cuh"

namespace qs {
namespace {

#ifndef QS_TILE_DF_THREADS
#define QS_TILE_DF_THREADS 256
#endif
constexpr int kThreads = QS_TILE_DF_THREADS;
#ifndef QS_LOAD_BATCH
#define QS_LOAD_BATCH 8
#endif
constexpr int kLoadBatch = QS_LOAD_BATCH;
// shared-memory layout of the tile (device.cuh): bank-spreading for gates on tile bits 0..2
#ifndef QS_DF_SWIZZLE
#define QS_DF_SWIZZLE 1
#endif
using kDfLayout = std::conditional<QS_DF_SWIZZLE != 0, Swizzled16Layout, FlatLayout>::type;

// The pass body; OpAt(g) yields op g of the pass.  B > 0: the tile has
// exactly 2^B amplitudes and the fixed-size gate paths are used.  DR: the pass
// holds diagonal runs.  Passes without them use the variant without that code:
// compiled in, it raised the kernel's registers from 40 to 61 and slowed
// passes without any run by 10%.
template <int B = 0, bool DR = false, class OpAt>
__device__ __forceinline__ void tile_df_body(double2* __restrict__ psi, const TilePass& P, OpAt op_at) {
    using L = kDfLayout;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sm = reinterpret_cast<float4*>(smem_raw);
    const int b = P.b, b0 = P.b0, nh = b - b0;
    const uint32_t N = 1u << b;
    // tile, then the phase-run tables (qs_internal.h), then the run offsets
    float4* tab = sm + N;
    uint64_t* hioff = reinterpret_cast<uint64_t*>(tab + (1u << (b / 2)) + (1u << (b - b / 2)) + 1u + (uint32_t)b);
    const uint64_t base = deposit_bits((uint64_t)blockIdx.x, P.nontile_mask);
    for (uint32_t h = threadIdx.x; h < (1u << nh); h += kThreads) {
        uint64_t off = 0;
        for (int j = 0; j < nh; ++j)
            if ((h >> j) & 1u) off |= 1ull << P.hi_q[j];
        hioff[h] = off;
    }
    __syncthreads();
    const uint32_t lomask = (1u << b0) - 1u;
    // kIoPairsIn: the previous pass left float pairs in place of the doubles
    // (the same 16 bytes per amplitude), so the tile is taken without a split
    const bool pairs_in = (P.io & kIoPairsIn) != 0;
    auto to_tile = [&](double2 raw) -> float4 {
        if (pairs_in) {
            float4 v;
            v.x = __int_as_float((int)(unsigned)__double_as_longlong(raw.x));
            v.y = __int_as_float((int)(unsigned)((unsigned long long)__double_as_longlong(raw.x) >> 32));
            v.z = __int_as_float((int)(unsigned)__double_as_longlong(raw.y));
            v.w = __int_as_float((int)(unsigned)((unsigned long long)__double_as_longlong(raw.y) >> 32));
            return v;
        }
        return df_load(raw);
    };
    if constexpr (B > 0 && kLoadBatch > 0 && (1 << B) >= kThreads) {
        // fixed tile size: each thread issues kLoadBatch global loads before the
        // first conversion, so one tile costs a few memory latencies, not 2^B / threads
        constexpr int PER = (1 << B) / kThreads;
        constexpr int BATCH = PER < kLoadBatch ? PER : kLoadBatch;
#pragma unroll
        for (int u0 = 0; u0 < PER; u0 += BATCH) {
            double2 v[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const uint32_t e = threadIdx.x + (uint32_t)((u0 + k) * kThreads);
                v[k] = psi[base + hioff[e >> b0] + (e & lomask)];
            }
#pragma unroll
            for (int k = 0; k < BATCH; ++k) sm[L::at(threadIdx.x + (uint32_t)((u0 + k) * kThreads))] = to_tile(v[k]);
        }
    } else {
        for (uint32_t e = threadIdx.x; e < N; e += kThreads) sm[L::at(e)] = to_tile(psi[base + hioff[e >> b0] + (e & lomask)]);
    }
    __syncthreads();
    for (int g = 0; g < P.nops; ++g) {
        auto&& op = op_at(g);
        if (op.kind == OP_PRUN) {
            df_phase_run<kThreads, B, L>(sm, tab, N, b, op, op_at, g, base);
            g += op.cls;  // the run's payload records
            __syncthreads();
        } else if (DR && op.kind == OP_DRUN) {
            if constexpr (DR) df_diag_run<kThreads, B, L>(sm, tab, N, b, op, op_at, g, base);
            g += op.cls;
            __syncthreads();
        } else if (df_tile_apply<kThreads, B, L>(sm, N, op, base)) {
            __syncthreads();
        }
    }
    if (P.io & kIoPairsOut) {
        // the next pass reads float pairs: renormalised here by TwoSum (exact),
        // as the rounding to a double and the split would do, so that the low
        // parts do not grow relative to the high parts over many passes
        float4* dst = reinterpret_cast<float4*>(psi);
        for (uint32_t e = threadIdx.x; e < N; e += kThreads) {
            const float4 v = sm[L::at(e)];
            const dfl r = two_sum(v.x, v.y), i = two_sum(v.z, v.w);
            dst[base + hioff[e >> b0] + (e & lomask)] = make_float4(r.h, r.l, i.h, i.l);
        }
    } else {
        for (uint32_t e = threadIdx.x; e < N; e += kThreads) psi[base + hioff[e >> b0] + (e & lomask)] = df_store(sm[L::at(e)]);
    }
}

// ops in device memory (batched launches: one op array per instance)
template <int B, bool DR>
__global__ void __launch_bounds__(kThreads) k_tile_df(double2* __restrict__ psi, const TileOpDF* __restrict__ ops,
                                                      TilePass P) {
    psi += (uint64_t)blockIdx.y * P.inst_stride;
    ops += (uint64_t)blockIdx.y * (uint64_t)P.ops_stride + P.op0;
    tile_df_body<B, DR>(psi, P, [&](int g) -> const TileOpDF& { return ops[g]; });
}

template <int B, bool DR>
cudaError_t launch_df_ptr(qs_state* s, const void* d_ops, const TilePass& P, unsigned count, size_t smem) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_df<B, DR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((unsigned)(1ull << (s->n - P.b)), count);
    k_tile_df<B, DR><<<grid, kThreads, smem, s->stream>>>(reinterpret_cast<double2*>(s->data),
                                                          reinterpret_cast<const TileOpDF*>(d_ops), P);
    return cudaGetLastError();
}

// ops in the kernel's parameter block: read through the constant cache,
// uniform across the CTA, with no global-memory load per op
constexpr int kParamOps = 296;
struct TileParamsDF {
    TilePass P;
    TileOpDF ops[kParamOps];
};
static_assert(sizeof(TileParamsDF) <= 32000, "kernel parameter block too large");

template <int B, bool DR>
__global__ void __launch_bounds__(kThreads) k_tile_df_p(double2* __restrict__ psi,
                                                        const __grid_constant__ TileParamsDF L) {
    tile_df_body<B, DR>(psi, L.P, [&](int g) -> const TileOpDF& { return L.ops[g]; });
}

template <int B, bool DR>
cudaError_t launch_df_p(qs_state* s, const TileParamsDF& L, size_t smem) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_df_p<B, DR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((unsigned)(1ull << (s->n - L.P.b)), 1);
    k_tile_df_p<B, DR><<<grid, kThreads, smem, s->stream>>>(reinterpret_cast<double2*>(s->data), L);
    return cudaGetLastError();
}

}  // namespace

void split_to_floats(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

cudaError_t launch_tile_df_params(qs_state* s, const TileOpDF* h_ops, const TilePass& P) {
    if (P.nops > kParamOps) return cudaErrorInvalidValue;
    const size_t smem = tile_pass_smem(s->dt, P.b, P.b0);
    static thread_local TileParamsDF L;
    L.P = P;
    L.P.op0 = 0;
    std::memcpy(L.ops, h_ops + P.op0, sizeof(TileOpDF) * (size_t)P.nops);
    // fixed-size instantiations for the tile sizes the planner and autotuner use
    if (P.io & kIoDiagRuns) {
        switch (P.b) {
        case 12: return launch_df_p<12, true>(s, L, smem);
        case 13: return launch_df_p<13, true>(s, L, smem);
        default: return launch_df_p<0, true>(s, L, smem);
        }
    }
    switch (P.b) {
    case 10: return launch_df_p<10, false>(s, L, smem);
    case 11: return launch_df_p<11, false>(s, L, smem);
    case 12: return launch_df_p<12, false>(s, L, smem);
    case 13: return launch_df_p<13, false>(s, L, smem);
    default: return launch_df_p<0, false>(s, L, smem);
    }
}

int tile_df_param_ops() { return kParamOps; }

cudaError_t launch_tile_df(qs_state* s, const void* d_ops, const TilePass& P, unsigned count) {
    const size_t smem = tile_pass_smem(s->dt, P.b, P.b0);
    if (P.io & kIoDiagRuns) {
        if (P.b == 12) return launch_df_ptr<12, true>(s, d_ops, P, count, smem);
        return launch_df_ptr<0, true>(s, d_ops, P, count, smem);
    }
    switch (P.b) {
    case 12: return launch_df_ptr<12, false>(s, d_ops, P, count, smem);
    case 13: return launch_df_ptr<13, false>(s, d_ops, P, count, smem);
    default: return launch_df_ptr<0, false>(s, d_ops, P, count, smem);
    }
}

}  // namespace qs
