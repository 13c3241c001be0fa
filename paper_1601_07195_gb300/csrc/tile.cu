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
#include <cstring>
#include <type_traits>

#include "device.cuh"
#include "tile_ops.cuh"

namespace qs {

namespace {

#ifndef QS_TILE_THREADS
#define QS_TILE_THREADS 256
#endif
constexpr int kTileThreads = QS_TILE_THREADS;
#ifndef QS_LOAD_BATCH
#define QS_LOAD_BATCH 8
#endif
constexpr int kLoadBatch = QS_LOAD_BATCH;

// DR: the pass holds diagonal runs; passes without them use the variant
// without that code path (as in tile_df.cu).
template <class R, int B = 0, bool DR = false, class OpAt>
__device__ __forceinline__ void tile_body(typename Amp<R>::T* __restrict__ psi, const TilePass& P, OpAt op_at) {
    using T = typename Amp<R>::T;
    // complex64 tiles use the bank-spreading layout (tile_ops.cuh)
    using L = typename std::conditional<std::is_same<R, float>::value, SwizzledLayout, FlatLayout>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int b = P.b, b0 = P.b0, nh = b - b0;
    const uint32_t N = 1u << b;
    // tile, then the phase-run tables (16 bytes per entry, qs_internal.h), then the run offsets
    unsigned char* tab = smem_raw + (sizeof(T) << b);
    uint64_t* hioff = reinterpret_cast<uint64_t*>(tab + 16u * ((1u << (b / 2)) + (1u << (b - b / 2)) + 1u + (uint32_t)b));
    const uint64_t base = deposit_bits((uint64_t)blockIdx.x, P.nontile_mask);
    for (uint32_t h = threadIdx.x; h < (1u << nh); h += kTileThreads) {
        uint64_t off = 0;
        for (int j = 0; j < nh; ++j)
            if ((h >> j) & 1u) off |= 1ull << P.hi_q[j];
        hioff[h] = off;
    }
    __syncthreads();
    const uint32_t lomask = (1u << b0) - 1u;
    if constexpr (B > 0 && kLoadBatch > 0 && (1 << B) >= kTileThreads) {
        // fixed tile size: kLoadBatch global loads in flight per thread (tile_df.cu)
        constexpr int PER = (1 << B) / kTileThreads;
        constexpr int BATCH = PER < kLoadBatch ? PER : kLoadBatch;
#pragma unroll
        for (int u0 = 0; u0 < PER; u0 += BATCH) {
            T v[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const uint32_t e = threadIdx.x + (uint32_t)((u0 + k) * kTileThreads);
                v[k] = psi[base + hioff[e >> b0] + (e & lomask)];
            }
#pragma unroll
            for (int k = 0; k < BATCH; ++k) sm[L::at(threadIdx.x + (uint32_t)((u0 + k) * kTileThreads))] = v[k];
        }
    } else {
        for (uint32_t e = threadIdx.x; e < N; e += kTileThreads) sm[L::at(e)] = psi[base + hioff[e >> b0] + (e & lomask)];
    }
    __syncthreads();
    for (int g = 0; g < P.nops; ++g) {
        auto&& op = op_at(g);
        if (op.kind == OP_PRUN) {
            phase_run<R, kTileThreads, B, L>(sm, tab, N, b, op, op_at, g, base);
            g += op.cls;  // the run's payload records
            __syncthreads();
        } else if (DR && op.kind == OP_DRUN) {
            if constexpr (DR) diag_run<R, kTileThreads, B, L>(sm, tab, N, b, op, op_at, g, base);
            g += op.cls;
            __syncthreads();
        } else if (tile_apply<R, kTileThreads, B, L>(sm, N, op, base)) {
            __syncthreads();
        }
    }
    for (uint32_t e = threadIdx.x; e < N; e += kTileThreads) psi[base + hioff[e >> b0] + (e & lomask)] = sm[L::at(e)];
}

// ops in device memory (batched launches: one op array per instance)
template <class R, bool DR>
__global__ void __launch_bounds__(kTileThreads) k_tile(typename Amp<R>::T* __restrict__ psi,
                                                       const TileOp<R>* __restrict__ ops, TilePass P) {
    psi += (uint64_t)blockIdx.y * P.inst_stride;
    ops += (uint64_t)blockIdx.y * (uint64_t)P.ops_stride + P.op0;
    tile_body<R, 0, DR>(psi, P, [&](int g) -> const TileOp<R>& { return ops[g]; });
}

// ops in the kernel's parameter block (constant cache, no global load per op)
template <class R> struct TileParams {
    static constexpr int kOps = (31000 - (int)sizeof(TilePass)) / (int)sizeof(TileOp<R>);
    TilePass P;
    TileOp<R> ops[kOps];
};

template <class R, int B, bool DR>
__global__ void __launch_bounds__(kTileThreads) k_tile_p(typename Amp<R>::T* __restrict__ psi,
                                                         const __grid_constant__ TileParams<R> L) {
    tile_body<R, B, DR>(psi, L.P, [&](int g) -> const TileOp<R>& { return L.ops[g]; });
}

template <class R, int B, bool DR = false>
cudaError_t launch_p(qs_state* s, const TileParams<R>& L, size_t smem) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_p<R, B, DR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((unsigned)(1ull << (s->n - L.P.b)), 1);
    k_tile_p<R, B, DR><<<grid, kTileThreads, smem, s->stream>>>(reinterpret_cast<typename Amp<R>::T*>(s->data), L);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_tile(qs_state* s, const void* d_ops, const TilePass& P, unsigned count) {
    const size_t smem = tile_pass_smem(s->dt, P.b, P.b0);
    static bool configured[2][2] = {{false, false}, {false, false}};
    const int which = sizeof(R) == 8 ? 1 : 0, dr = (P.io & kIoDiagRuns) ? 1 : 0;
    if (!configured[which][dr]) {
        cudaError_t e = dr ? cudaFuncSetAttribute(k_tile<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin())
                           : cudaFuncSetAttribute(k_tile<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin());
        if (e != cudaSuccess) return e;
        configured[which][dr] = true;
    }
    const dim3 grid((unsigned)(1ull << (s->n - P.b)), count);
    auto* psi = reinterpret_cast<typename Amp<R>::T*>(s->data);
    auto* ops = reinterpret_cast<const TileOp<R>*>(d_ops);
    if (dr) k_tile<R, true><<<grid, kTileThreads, smem, s->stream>>>(psi, ops, P);
    else k_tile<R, false><<<grid, kTileThreads, smem, s->stream>>>(psi, ops, P);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_tile_p(qs_state* s, const void* h_ops, const TilePass& P) {
    if (P.nops > TileParams<R>::kOps) return cudaErrorInvalidValue;
    const size_t smem = tile_pass_smem(s->dt, P.b, P.b0);
    static thread_local TileParams<R> L;
    L.P = P;
    L.P.op0 = 0;
    std::memcpy(L.ops, reinterpret_cast<const TileOp<R>*>(h_ops) + P.op0, sizeof(TileOp<R>) * (size_t)P.nops);
    if (P.io & kIoDiagRuns) {
        switch (P.b) {
        case 12: return launch_p<R, 12, true>(s, L, smem);
        case 13: return launch_p<R, 13, true>(s, L, smem);
        default: return launch_p<R, 0, true>(s, L, smem);
        }
    }
    switch (P.b) {
    case 11: return launch_p<R, 11>(s, L, smem);
    case 12: return launch_p<R, 12>(s, L, smem);
    case 13: return launch_p<R, 13>(s, L, smem);
    case 14: return launch_p<R, 14>(s, L, smem);
    default: return launch_p<R, 0>(s, L, smem);
    }
}

}  // namespace

size_t tile_smem_bytes(qs_dtype dt, int b) { return amp_bytes(dt) << b; }

int tile_param_ops(bool f64) { return f64 ? TileParams<double>::kOps : TileParams<float>::kOps; }

qs_status launch_tile_pass_params(qs_state* s, const void* h_ops, const TilePass& pass, bool f64) {
    if (tile_pass_smem(s->dt, pass.b, pass.b0) > smem_optin())
        return fail(QS_EINVAL, "tile does not fit in shared memory");
    cudaError_t e = f64 ? launch_tile_p<double>(s, h_ops, pass) : launch_tile_p<float>(s, h_ops, pass);
    if (e != cudaSuccess) return cuda_fail(e, "tile kernel launch");
    return QS_OK;
}

qs_status launch_tile_pass(qs_state* s, const void* d_ops, const TilePass& pass, bool arith_f64, unsigned count) {
    if (tile_pass_smem(s->dt, pass.b, pass.b0) > smem_optin())
        return fail(QS_EINVAL, "tile does not fit in shared memory");
    cudaError_t e;
    if (s->dt == QS_C64) e = launch_tile<float>(s, d_ops, pass, count);
    else if (arith_f64) e = launch_tile<double>(s, d_ops, pass, count);
    else e = launch_tile_df(s, d_ops, pass, count);
    if (e != cudaSuccess) return cuda_fail(e, "tile kernel launch");
    return QS_OK;
}

}  // namespace qs
