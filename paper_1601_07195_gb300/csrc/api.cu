// api.cu -- state lifetime, copies, single-gate entry points, error reporting,
// and the host-side lowering of gate records (classification by gate class).
#include <sys/mman.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "device.cuh"

namespace qs {

namespace {
thread_local std::string g_last_error;

__global__ void k_init_basis_c128(double2* psi, uint64_t N, uint64_t x) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        psi[i] = make_double2(i == x ? 1.0 : 0.0, 0.0);
}
__global__ void k_init_basis_c64(float2* psi, uint64_t N, uint64_t x) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        psi[i] = make_float2(i == x ? 1.0f : 0.0f, 0.0f);
}

struct DevProps {
    int sms = 0;
    size_t smem = 0;
};
DevProps g_props[64];
std::mutex g_props_mu;

const DevProps& props() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(g_props_mu);
    if (g_props[dev].sms == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_props[dev].sms = v > 0 ? v : 1;
        v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        g_props[dev].smem = v > 0 ? (size_t)v : 48 * 1024;
    }
    return g_props[dev];
}
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

qs_status fail(qs_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

qs_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;
}

int sm_count() { return props().sms; }
size_t smem_optin() { return props().smem; }

// Gate class from the exact matrix entries (no tolerance: a class is only used
// when the specialised update computes exactly the same product).
int classify(const double m[8]) {
    const bool q12z = m[2] == 0.0 && m[3] == 0.0, q21z = m[4] == 0.0 && m[5] == 0.0;
    const bool q11z = m[0] == 0.0 && m[1] == 0.0, q22z = m[6] == 0.0 && m[7] == 0.0;
    if (q11z && q22z && m[2] == 1.0 && m[3] == 0.0 && m[4] == 1.0 && m[5] == 0.0) return GC_PERM;
    if (q12z && q21z) return (m[0] == 1.0 && m[1] == 0.0) ? GC_DIAG1 : GC_DIAG;
    if (q11z && q22z) return GC_ANTIDIAG;
    if (m[1] == 0.0 && m[3] == 0.0 && m[5] == 0.0 && m[7] == 0.0) return GC_REAL;
    return GC_GENERAL;
}

// exp(-i theta G / 2) for G = X, Y, Z.
static void rotation(int kind, double th, double m[8]) {
    const double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
    std::memset(m, 0, 8 * sizeof(double));
    if (kind == QS_G_RX) { m[0] = c; m[3] = -s; m[5] = -s; m[6] = c; }
    else if (kind == QS_G_RY) { m[0] = c; m[2] = -s; m[4] = s; m[6] = c; }
    else { m[0] = c; m[1] = -s; m[6] = c; m[7] = s; }
}

qs_status lower_gates(const qs_gate* g, int ng, const double* theta, int np, int n, std::vector<Op>& out) {
    if (ng < 0) return fail(QS_EINVAL, "negative gate count");
    if (ng > 0 && g == nullptr) return fail(QS_EINVAL, "gate array is NULL");
    out.clear();
    out.reserve(ng);
    for (int j = 0; j < ng; ++j) {
        const qs_gate& r = g[j];
        Op o;
        o.t = r.t;
        o.c = -1;
        if (r.t < 0 || r.t >= n) return fail(QS_EINVAL, "gate " + std::to_string(j) + ": qubit out of range");
        switch (r.kind) {
        case QS_G_U1:
            o.kind = OP_1Q;
            std::memcpy(o.m, r.m, sizeof(o.m));
            break;
        case QS_G_CU:
        case QS_G_SWAP:
            if (r.c < 0 || r.c >= n || r.c == r.t)
                return fail(QS_EINVAL, "gate " + std::to_string(j) + ": bad second qubit");
            o.kind = r.kind == QS_G_CU ? OP_CU : OP_SWAP;
            o.c = r.c;
            std::memcpy(o.m, r.m, sizeof(o.m));
            break;
        case QS_G_RX:
        case QS_G_RY:
        case QS_G_RZ:
            if (r.param < 0 || r.param >= np || theta == nullptr)
                return fail(QS_EINVAL, "gate " + std::to_string(j) + ": bad parameter index");
            o.kind = OP_1Q;
            rotation(r.kind, theta[r.param], o.m);
            break;
        default:
            return fail(QS_EINVAL, "gate " + std::to_string(j) + ": unknown kind");
        }
        for (int q = 0; q < 8; ++q)
            if (!std::isfinite(o.m[q])) return fail(QS_EINVAL, "gate " + std::to_string(j) + ": non-finite matrix");
        o.cls = o.kind == OP_SWAP ? GC_PERM : classify(o.m);
        out.push_back(o);
    }
    return QS_OK;
}

static qs_status check_state(const qs_state* s) {
    if (!s || !s->data) return fail(QS_EINVAL, "state handle is NULL");
    return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

const char* qs_last_error(void) { return g_last_error.c_str(); }

const char* qs_version(void) { return "qs 0.1 (sm_103a)"; }

qs_status qs_wrap(void* dev_ptr, int n, qs_dtype dt, void* stream, qs_state** out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 40) return fail(QS_EINVAL, "n must be in [1, 40]");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EDTYPE, "unknown dtype");
    if (!dev_ptr) return fail(QS_EINVAL, "device pointer is NULL");
    if ((uintptr_t)dev_ptr % amp_bytes(dt) != 0) return fail(QS_EINVAL, "device pointer is not aligned to one amplitude");
    qs_state* s = new (std::nothrow) qs_state();
    if (!s) return fail(QS_ENOMEM, "host allocation failed");
    s->n = n;
    s->dt = dt;
    s->data = dev_ptr;
    s->owned = false;
    s->stream = (cudaStream_t)stream;
    cudaGetDevice(&s->device);
    // Where the runtime can classify the pointer, it must be device (or managed)
    // memory of the current device: the state's kernels launch there.
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, dev_ptr) == cudaSuccess) {
        if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
            delete s;
            return fail(QS_EINVAL, "pointer is not device memory");
        }
        if (attr.type == cudaMemoryTypeDevice && attr.device != s->device) {
            delete s;
            return fail(QS_EINVAL, "pointer belongs to device " + std::to_string(attr.device) +
                                       " but device " + std::to_string(s->device) + " is current");
        }
    } else {
        cudaGetLastError();  // no device or driver here: the pointer cannot be checked
    }
    *out = s;
    return QS_OK;
}

qs_status qs_create(int n, qs_dtype dt, void* stream, qs_state** out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 36) return fail(QS_EINVAL, "n must be in [1, 36]");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EDTYPE, "unknown dtype");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, amp_bytes(dt) << n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, std::string("cudaMalloc of the state failed: ") + cudaGetErrorString(e));
    }
    qs_status st = qs_wrap(p, n, dt, stream, out);
    if (st != QS_OK) {
        cudaFree(p);
        return st;
    }
    (*out)->owned = true;
    st = qs_init_basis(*out, 0);
    if (st != QS_OK) {
        qs_destroy(*out);
        *out = nullptr;
    }
    return st;
}

qs_status qs_destroy(qs_state* s) {
    if (!s) return QS_OK;
    if (s->owned && s->data) cudaFree(s->data);
    if (s->d_partials) cudaFree(s->d_partials);
    if (s->h_result) cudaFreeHost(s->h_result);
    if (s->d_dense) cudaFree(s->d_dense);
    if (s->h_dense) cudaFreeHost(s->h_dense);
    delete s;
    return QS_OK;
}

qs_status qs_set_stream(qs_state* s, void* stream) {
    if (qs_status st = check_state(s)) return st;
    s->stream = (cudaStream_t)stream;
    return QS_OK;
}

qs_status qs_set_arith(qs_state* s, int native_f64) {
    if (qs_status st = check_state(s)) return st;
    s->arith_f64 = native_f64 != 0;
    return QS_OK;
}

qs_status qs_set_lanes(qs_state* s, int mode) {
    if (qs_status st = check_state(s)) return st;
    if (mode != QS_LANES_OFF && mode != QS_LANES_AUTO && mode != QS_LANES_ON)
        return fail(QS_EINVAL, "lane mode must be QS_LANES_OFF, QS_LANES_AUTO or QS_LANES_ON");
    s->lane_mode = mode == QS_LANES_AUTO ? 0 : (mode == QS_LANES_ON ? 1 : -1);
    return QS_OK;
}

qs_status qs_info(const qs_state* s, void** dev_ptr, int* n, qs_dtype* dt) {
    if (!s) return fail(QS_EINVAL, "state handle is NULL");
    if (dev_ptr) *dev_ptr = s->data;
    if (n) *n = s->n;
    if (dt) *dt = s->dt;
    return QS_OK;
}

qs_status qs_init_basis(qs_state* s, uint64_t x) {
    if (qs_status st = check_state(s)) return st;
    const uint64_t N = 1ull << s->n;
    if (x >= N) return fail(QS_EINVAL, "basis index out of range");
    uint64_t blocks = (N + 511) / 512;
    const uint64_t cap = (uint64_t)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (s->dt == QS_C128) k_init_basis_c128<<<(unsigned)blocks, 512, 0, s->stream>>>((double2*)s->data, N, x);
    else k_init_basis_c64<<<(unsigned)blocks, 512, 0, s->stream>>>((float2*)s->data, N, x);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

qs_status qs_copy_out(qs_state* s, uint64_t off, uint64_t cnt, void* host) {
    if (qs_status st = check_state(s)) return st;
    if (!host && cnt) return fail(QS_EINVAL, "host pointer is NULL");
    if (off > (1ull << s->n) || cnt > (1ull << s->n) - off) return fail(QS_EINVAL, "range out of bounds");
    const size_t ab = amp_bytes(s->dt);
    QS_CUDA_TRY(cudaMemcpyAsync(host, (char*)s->data + off * ab, cnt * ab, cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
}

qs_status qs_copy_in(qs_state* s, uint64_t off, uint64_t cnt, const void* host) {
    if (qs_status st = check_state(s)) return st;
    if (!host && cnt) return fail(QS_EINVAL, "host pointer is NULL");
    if (off > (1ull << s->n) || cnt > (1ull << s->n) - off) return fail(QS_EINVAL, "range out of bounds");
    const size_t ab = amp_bytes(s->dt);
    QS_CUDA_TRY(cudaMemcpyAsync((char*)s->data + off * ab, host, cnt * ab, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
}

// ---- host buffers for transfers -------------------------------------------------
// Page-locked host memory of base-size pages (what cudaHostAlloc returns) lost up
// to 8x of its host-to-device rate on the GB300 nodes measured (64 KiB base pages):
// for the first copy after the GPU had been busy or idle for a few seconds, and
// for every copy once other jobs had fragmented host memory.  An anonymous mapping
// backed by transparent huge pages and then registered kept the full rate on every
// copy.  The mapping's size is kept here so that qs_host_free needs only the pointer.
namespace {
std::mutex g_host_mu;
std::map<void*, size_t> g_host_maps;
}  // namespace

// Transparent huge page size of this kernel (2 MiB where it cannot be read).
static size_t thp_size() {
    size_t v = 0;
    if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long x = 0;
        if (std::fscanf(f, "%llu", &x) == 1) v = (size_t)x;
        std::fclose(f);
    }
    return (v >= 4096 && (v & (v - 1)) == 0) ? v : ((size_t)2 << 20);
}

qs_status qs_host_alloc(size_t bytes, void** out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (bytes == 0) return fail(QS_EINVAL, "size is zero");
    // Start and length aligned to the transparent huge page size (the PMD size:
    // 2 MiB with 4 KiB base pages, 512 MiB with 64 KiB ones), so that every page of
    // the buffer can be a huge page: the device then reads it through far fewer
    // translations (a 16 GiB copy: 84-97 ms on huge pages; 310-680 ms with 12 of
    // its 32 pages left at 64 KiB)
    // (buffers smaller than one huge page are aligned to 2 MiB only: rounding
    // them up to 512 MiB would waste memory and the time to populate it)
    const size_t thp = thp_size();
    const size_t align = bytes >= thp ? thp : ((size_t)2 << 20);
    const size_t len = (bytes + align - 1) / align * align;
    void* raw = mmap(nullptr, len + align, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == MAP_FAILED) return fail(QS_ENOMEM, "mmap of the host buffer failed");
    const uintptr_t r = (uintptr_t)raw, a = (r + align - 1) / align * align;
    if (a > r) munmap(raw, a - r);                                // trim to the aligned range
    if (r + align > a) munmap((void*)(a + len), r + align - a);
    void* p = (void*)a;
#ifdef MADV_HUGEPAGE
    madvise(p, len, MADV_HUGEPAGE);  // best effort: the buffer works with base pages too
#endif
    // Populate one huge page at a time (as a huge page where the fault path finds
    // one free).  Where it found none (fragmented memory), ask the kernel to
    // collapse that page now, which compacts memory for it (Linux 6.1+; up to
    // three tries; best effort, an older kernel rejects the advice).
    for (size_t off = 0; off < len; off += align) {
        char* c = (char*)p + off;
        std::memset(c, 0, align);
        for (int tries = 0; tries < 3 && madvise(c, align, 25 /* MADV_COLLAPSE */) != 0; ++tries) {
        }
    }
    cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        munmap(p, len);
        return fail(e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA,
                    std::string("cudaHostRegister of the host buffer failed: ") + cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        g_host_maps[p] = len;
    }
    *out = p;
    return QS_OK;
}

qs_status qs_host_free(void* p) {
    if (!p) return QS_OK;
    size_t len = 0;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_maps.find(p);
        if (it == g_host_maps.end()) return fail(QS_EINVAL, "pointer was not returned by qs_host_alloc");
        len = it->second;
        g_host_maps.erase(it);
    }
    cudaError_t e = cudaHostUnregister(p);
    munmap(p, len);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostUnregister");
    return QS_OK;
}

qs_status qs_apply_1q(qs_state* s, int k, const double U[8]) {
    if (qs_status st = check_state(s)) return st;
    if (!U) return fail(QS_EINVAL, "matrix is NULL");
    qs_gate g{};
    g.kind = QS_G_U1; g.t = k; g.c = -1; g.param = -1;
    std::memcpy(g.m, U, sizeof(g.m));
    std::vector<Op> ops;
    if (qs_status st = lower_gates(&g, 1, nullptr, 0, s->n, ops)) return st;
    return launch_op(s, ops[0], s->arith_f64);
}

qs_status qs_apply_ctrl(qs_state* s, int c, int t, const double U[8]) {
    if (qs_status st = check_state(s)) return st;
    if (!U) return fail(QS_EINVAL, "matrix is NULL");
    qs_gate g{};
    g.kind = QS_G_CU; g.t = t; g.c = c; g.param = -1;
    std::memcpy(g.m, U, sizeof(g.m));
    std::vector<Op> ops;
    if (qs_status st = lower_gates(&g, 1, nullptr, 0, s->n, ops)) return st;
    return launch_op(s, ops[0], s->arith_f64);
}

qs_status qs_apply_swap(qs_state* s, int a, int b) {
    if (qs_status st = check_state(s)) return st;
    qs_gate g{};
    g.kind = QS_G_SWAP; g.t = a; g.c = b; g.param = -1;
    std::vector<Op> ops;
    if (qs_status st = lower_gates(&g, 1, nullptr, 0, s->n, ops)) return st;
    return launch_op(s, ops[0], s->arith_f64);
}

}  // extern "C"
