// dense_tc.cu -- a dense 64 x 64 complex block on qubits 0..5 of a complex64
// state, on the fifth-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory).
//
// Not in the paper: the paper fuses runs of gates by keeping a block of the
// state in cache (Section 4.4, Fig. 5) and applies each gate of the run as
// Eq. 2 / Eq. 3.  Here the run's product U is formed once on the host and
// applied as one matrix: viewing the state as rows of 64 consecutive
// amplitudes (qubits 0..5 inside a row), every row x becomes U x.  In real
// arithmetic on the interleaved (re, im) layout a row is a vector of 128
// floats and the update is Y = X W with the real 128 x 128 matrix
//   W[2c][2r] = Re U[r][c],  W[2c+1][2r] = -Im U[r][c],
//   W[2c][2r+1] = Im U[r][c],  W[2c+1][2r+1] = Re U[r][c].
//
// Precision.  Each float x of the state is split exactly into three bf16
// pieces x = x1 + x2 + x3 (each the round-to-nearest bf16 of what remains),
// and W likewise on the host; the product keeps the six piece products whose
// combined weight is at least 2^-16 relative (x1 w1, x1 w2, x2 w1, x1 w3,
// x2 w2, x3 w1), accumulated in FP32 in tensor memory.  The dropped products
// weigh at most about 2^-24, the level of FP32 rounding, so the block has the
// accuracy of a complex64 state.
//
// Mapping.  The MMA computes D = A B with A = W^T (M = 128 output components,
// K = 128 input components) resident in shared memory, and B = a tile of 128
// state rows (N = 128, K-major: a row's 128 floats are contiguous, exactly the
// state's layout).  D row m (tensor-memory lane m) holds output component m
// of the tile's 128 rows (columns), so in the epilogue consecutive threads
// hold consecutive components of one row: every store of a warp writes 128
// contiguous bytes.
//
// Operands in shared memory use the K-major layout with the 128-byte swizzle:
// a K chunk of 64 bf16 (128 bytes) per row, rows 128 bytes apart, 8-row
// groups 1024 bytes apart, and the 16-byte unit u of row r stored at unit
// u ^ (r & 7).  K = 128 is held as two such chunks.
//
// Roles of the persistent CTA (one per SM: the operands take 192 KiB of
// shared memory):
//   warps 0-3   epilogue: tensor memory -> registers -> the state (in place)
//   warps 4-11  producers: state rows -> registers -> bf16 pieces in shared memory,
//               the loads of the next K chunk in flight while one is split and stored
//   warp 12     allocates tensor memory; its lane 0 issues the MMAs
// A tile passes through two shared-memory stages (one per K chunk) and two
// tensor-memory accumulators, so loads of the next tile, the MMAs of this one
// and the stores of the previous one overlap.  Every wait on an mbarrier is
// bounded; a wait that gives up records an error and its role stops, and the
// MMA lane drains its own MMAs before the tensor memory is freed.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "device.cuh"

namespace qs {

namespace {

constexpr int kRows = 128;             // state rows per tile (the MMA's N)
constexpr int kComps = 128;            // floats per row (64 complex amplitudes)
constexpr int kChunkBytes = 128 * 128; // one K chunk of one operand piece: 128 rows x 128 bytes
constexpr int kProducerWarps = 8;
constexpr int kProducerThreads = 32 * kProducerWarps;
constexpr int kUnits = kRows * 8 / kProducerThreads;  // 8-float units per producer thread per K chunk
constexpr int kMmaWarp = 4 + kProducerWarps;
constexpr int kThreads = 32 * (kMmaWarp + 1);      // epilogue 4 warps, producers, MMA warp
constexpr int kSmemBytes = 12 * kChunkBytes + 1024;  // W: 3 pieces x 2 chunks; X: 2 stages x 3 pieces; alignment
constexpr uint32_t kTmemCols = 256;    // two accumulators of 128 fp32 columns
constexpr long long kWaitLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, leading / stride byte
// offsets (>> 4), the fixed version bits 0b001 at 46..48, swizzle mode at 61..63
// (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused by swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 128 (bits 17..22 hold N >> 3), M = 128 (bits 24..28 hold M >> 4).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kRows >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_addr(bar))
                 : "memory");
}
// Wait until the phase of parity `parity` has completed; false if it did not
// within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}
// Arrive on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Exact split of two floats into three bf16 pieces each, packed in pairs.
__device__ __forceinline__ void split3(float a, float b, uint32_t& p1, uint32_t& p2, uint32_t& p3) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float a1 = a - __low2float(h), b1 = b - __high2float(h);
    __nv_bfloat162 m = __floats2bfloat162_rn(a1, b1);
    const float a2 = a1 - __low2float(m), b2 = b1 - __high2float(m);
    __nv_bfloat162 l = __floats2bfloat162_rn(a2, b2);
    p1 = *reinterpret_cast<uint32_t*>(&h);
    p2 = *reinterpret_cast<uint32_t*>(&m);
    p3 = *reinterpret_cast<uint32_t*>(&l);
}

struct DenseArgs {
    float* psi;                // the state as floats: row r at psi + r * 128
    const uint4* w;            // A = W^T pieces, row-major bf16: [piece][m][k], 3 x 128 x 128
    unsigned long long rows;   // 2^(n-6)
    unsigned long long tiles;  // ceil(rows / 128)
    int* err;                  // set to 1 when a bounded wait gave up
};

__global__ void __launch_bounds__(kThreads, 1) k_dense6_tc(DenseArgs args) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sW = smem;                     // piece p, chunk kc at (2p + kc) * kChunkBytes
    uint8_t* sX = smem + 6 * kChunkBytes;   // stage s, piece p at (3s + p) * kChunkBytes
    __shared__ uint64_t full_bar[2], empty_bar[2], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // W^T pieces into shared memory, swizzled (all threads)
    for (int idx = tid; idx < 3 * 128 * 16; idx += kThreads) {
        const int p = idx / (128 * 16), m = (idx / 16) % 128, u = idx % 16;  // 16 units of 8 bf16 per row
        const int kc = u >> 3, uu = u & 7;
        const uint4 v = args.w[idx];
        *reinterpret_cast<uint4*>(sW + (2 * p + kc) * kChunkBytes + m * 128 + ((uu ^ (m & 7)) << 4)) = v;
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full_bar[s], kProducerThreads);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&accf_bar[s], 1);
            mbar_init(&acce_bar[s], 128);
        }
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const unsigned long long tiles = args.tiles, rows = args.rows;

    if (warp >= 4 && warp < 4 + kProducerWarps) {
        // ---- producers: kProducerThreads threads, kUnits units of 8 floats each per K chunk.
        // Chunk j is K chunk (j & 1) of tile blockIdx.x + (j >> 1) gridDim.x; the loads of
        // chunk j + 1 are issued before chunk j is split and stored (two register sets).
        const int pt = tid - 128;
        auto tile_of = [&](unsigned long long j) { return (unsigned long long)blockIdx.x + (j >> 1) * gridDim.x; };
        auto load = [&](float4 (&v)[2 * kUnits], unsigned long long j) {
            const unsigned long long t = tile_of(j);
            const int kc = (int)(j & 1);
#pragma unroll
            for (int q = 0; q < kUnits; ++q) {
                const int unit = pt + kProducerThreads * q, r = unit >> 3, u = unit & 7;
                const unsigned long long row = t * kRows + r;
                if (row < rows) {
                    const float4* src = reinterpret_cast<const float4*>(args.psi + row * kComps + kc * 64 + u * 8);
                    v[2 * q] = src[0];
                    v[2 * q + 1] = src[1];
                } else {
                    v[2 * q] = v[2 * q + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        };
        auto store = [&](const float4 (&v)[2 * kUnits], unsigned long long j) -> bool {
            const int s = (int)(j & 1);
            if (!mbar_wait(&empty_bar[s], (uint32_t)(((j >> 1) & 1) ^ 1))) return false;
#pragma unroll
            for (int q = 0; q < kUnits; ++q) {
                const int unit = pt + kProducerThreads * q, r = unit >> 3, u = unit & 7;
                uint4 q1, q2, q3;
                split3(v[2 * q].x, v[2 * q].y, q1.x, q2.x, q3.x);
                split3(v[2 * q].z, v[2 * q].w, q1.y, q2.y, q3.y);
                split3(v[2 * q + 1].x, v[2 * q + 1].y, q1.z, q2.z, q3.z);
                split3(v[2 * q + 1].z, v[2 * q + 1].w, q1.w, q2.w, q3.w);
                const uint32_t off = r * 128 + ((u ^ (r & 7)) << 4);
                *reinterpret_cast<uint4*>(sX + (3 * s + 0) * kChunkBytes + off) = q1;
                *reinterpret_cast<uint4*>(sX + (3 * s + 1) * kChunkBytes + off) = q2;
                *reinterpret_cast<uint4*>(sX + (3 * s + 2) * kChunkBytes + off) = q3;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full_bar[s]);
            return true;
        };
        float4 va[2 * kUnits], vb[2 * kUnits];
        unsigned long long j = 0;
        if (tile_of(0) < tiles) {
            load(va, 0);
            for (;;) {
                bool next = tile_of(j + 1) < tiles;
                if (next) load(vb, j + 1);
                if (!store(va, j)) { atomicOr(args.err, 1); break; }
                ++j;
                if (!next) break;
                next = tile_of(j + 1) < tiles;
                if (next) load(va, j + 1);
                if (!store(vb, j)) { atomicOr(args.err, 1); break; }
                ++j;
                if (!next) break;
            }
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issue (one lane)
        if (lane == 0) {
            // the six piece products (W piece, X piece), smallest weights first
            const int pw[6] = {2, 1, 0, 1, 0, 0}, px[6] = {0, 1, 2, 0, 1, 0};
            unsigned long long chunk = 0, local = 0;
            bool ok = true;
            for (unsigned long long t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++local) {
                const int a = (int)(local & 1);
                if (!mbar_wait(&acce_bar[a], (uint32_t)(((local >> 1) & 1) ^ 1))) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(a * kRows);
                for (int kc = 0; kc < 2; ++kc, ++chunk) {
                    const int s = (int)(chunk & 1);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((chunk >> 1) & 1))) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    for (int pr = 0; pr < 6; ++pr) {
                        const uint32_t abase = smem_addr(sW + (2 * pw[pr] + kc) * kChunkBytes);
                        const uint32_t bbase = smem_addr(sX + (3 * s + px[pr]) * kChunkBytes);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            mma_bf16(d, smem_desc(abase + ks * 32), smem_desc(bbase + ks * 32),
                                     (kc | pr | ks) != 0);
                    }
                    mma_commit(&empty_bar[s]);  // the stage is free once these MMAs have read it
                }
                if (ok) mma_commit(&accf_bar[a]);
            }
            if (!ok) atomicOr(args.err, 1);
            // drain: every MMA issued above has completed before tensor memory is freed
            mma_commit(&drain_bar);
            if (!mbar_wait(&drain_bar, 0)) atomicOr(args.err, 1);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps 0-3, lane quarter w holds output components 32w..32w+31
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const int m = warp * 32 + lane;
        unsigned long long local = 0;
        for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
            const int a = (int)(local & 1);
            if (!mbar_wait(&accf_bar[a], (uint32_t)((local >> 1) & 1))) {
                atomicOr(args.err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int c0 = 0; c0 < kRows; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(a * kRows + c0), v);
                const unsigned long long row0 = t * kRows + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (row0 + j < rows) args.psi[(row0 + j) * kComps + m] = v[j];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acce_bar[a]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Round a double to the nearest bf16 value (ties to even), returned as a double.
double round_bf16(double x) {
    if (x == 0.0 || !std::isfinite(x)) return 0.0;
    int e;
    const double m = std::frexp(x, &e);  // |m| in [0.5, 1)
    if (e < -125) return 0.0;            // below the smallest normal bf16
    return std::ldexp(std::nearbyint(std::ldexp(m, 8)), e - 8);
}
uint16_t bf16_bits(double v) {  // v is exactly a bf16 value
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

}  // namespace

// Host image of the operand A = W^T of a 64 x 64 complex matrix U (row-major
// (re, im) doubles), split into three bf16 pieces: out[p][m][k], 3 x 128 x 128.
void dense_tc_operand(const double* U, uint16_t* out) {
    for (int m = 0; m < 128; ++m) {
        const int r = m >> 1;
        for (int k = 0; k < 128; ++k) {
            const int c = k >> 1;
            const double ur = U[2 * (r * 64 + c)], ui = U[2 * (r * 64 + c) + 1];
            double a;  // A[m][k] = W[k][m]
            if ((m & 1) == 0) a = (k & 1) == 0 ? ur : -ui;
            else a = (k & 1) == 0 ? ui : ur;
            const double a1 = round_bf16(a), a2 = round_bf16(a - a1), a3 = round_bf16(a - a1 - a2);
            out[(0 * 128 + m) * 128 + k] = bf16_bits(a1);
            out[(1 * 128 + m) * 128 + k] = bf16_bits(a2);
            out[(2 * 128 + m) * 128 + k] = bf16_bits(a3);
        }
    }
}

size_t dense_tc_operand_bytes() { return (size_t)3 * 128 * 128 * 2; }

// The kernel's shared-memory size, set once per device.  Plans call this when
// they are created, so a plan captured into a CUDA graph never sets it during
// the capture.
cudaError_t dense_tc_prepare() {
    static_assert(kSmemBytes <= 227 * 1024, "operands exceed shared memory");
    static bool configured[64] = {false};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(k_dense6_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    return cudaSuccess;
}

// Launch on s->stream: the operand image is at d_w (device), err a device int.
cudaError_t launch_dense_tc(qs_state* s, const void* d_w, int* d_err, int max_ctas) {
    DenseArgs a;
    a.psi = reinterpret_cast<float*>(s->data);
    a.w = reinterpret_cast<const uint4*>(d_w);
    a.rows = 1ull << (s->n - 6);
    a.tiles = (a.rows + kRows - 1) / kRows;
    a.err = d_err;
    cudaError_t e = dense_tc_prepare();
    if (e != cudaSuccess) return e;
    unsigned long long grid = a.tiles;
    const unsigned long long cap = (unsigned long long)(max_ctas > 0 ? max_ctas : sm_count());
    if (grid > cap) grid = cap;
    k_dense6_tc<<<(unsigned)grid, kThreads, kSmemBytes, s->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace qs

using namespace qs;

extern "C" qs_status qs_apply_dense(qs_state* s, int q, const double* U) {
    if (!s || !s->data) return fail(QS_EINVAL, "state handle is NULL");
    if (!U) return fail(QS_EINVAL, "matrix is NULL");
    if (s->dt != QS_C64) return fail(QS_EDTYPE, "the dense tensor-core block is available for complex64 states only");
    if (q < 1 || q > 6) return fail(QS_EINVAL, "q must be in [1, 6]");
    if (s->n < 6) return fail(QS_EINVAL, "the dense block needs n >= 6");
    for (int j = 0; j < (2 << (2 * q)); ++j)
        if (!std::isfinite(U[j])) return fail(QS_EINVAL, "non-finite matrix entry");
    // the 64 x 64 matrix on qubits 0..5: I (x) U for q < 6 (U on the low q qubits)
    static thread_local double full[2 * 64 * 64];
    const int G = 1 << q;
    std::memset(full, 0, sizeof(full));
    for (int hi = 0; hi < 64 / G; ++hi)
        for (int r = 0; r < G; ++r)
            for (int c = 0; c < G; ++c) {
                full[2 * ((hi * G + r) * 64 + hi * G + c)] = U[2 * (r * G + c)];
                full[2 * ((hi * G + r) * 64 + hi * G + c) + 1] = U[2 * (r * G + c) + 1];
            }
    const size_t wb = dense_tc_operand_bytes();
    if (!s->d_dense) {
        cudaError_t e = cudaMalloc(&s->d_dense, wb + 256);
        if (e != cudaSuccess) { cudaGetLastError(); s->d_dense = nullptr; return fail(QS_ENOMEM, "dense operand buffer"); }
    }
    if (!s->h_dense) {
        cudaError_t e = cudaMallocHost(&s->h_dense, wb);
        if (e != cudaSuccess) { cudaGetLastError(); s->h_dense = nullptr; return fail(QS_ENOMEM, "dense operand staging"); }
    }
    dense_tc_operand(full, reinterpret_cast<uint16_t*>(s->h_dense));
    int* d_err = reinterpret_cast<int*>(reinterpret_cast<char*>(s->d_dense) + wb);
    QS_CUDA_TRY(cudaMemcpyAsync(s->d_dense, s->h_dense, wb, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s->stream));
    cudaError_t e = launch_dense_tc(s, s->d_dense, d_err, 0);
    if (e != cudaSuccess) return cuda_fail(e, "dense block kernel launch");
    int h_err = 0;
    QS_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (h_err) return fail(QS_ETIMEOUT, "dense block: a bounded wait inside the kernel gave up");
    return QS_OK;
}
