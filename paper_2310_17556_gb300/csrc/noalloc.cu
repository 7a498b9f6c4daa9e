// dfs_fisher_pass_noalloc: the streaming pass of dfs_fisher_pass without a handle and without
// any device-memory allocation.  The paper has no counterpart; this exists for callers that
// cannot allocate device memory around the call, e.g. a caller whose device memory is fully
// reserved by its own pool allocator, or one that cannot afford the implicit device-wide
// synchronisation cudaMalloc and cudaFree may perform.
//
// Scratch (the per-CTA FP64 row partials of R = S U - lambda Y, the per-CTA sums of ||U||^2, and
// the device status word) lives in one file-scope __device__ array of DFS_NOALLOC_SCRATCH_BYTES,
// part of the library's device image.  Its address is looked up once per device, at the first
// call made with that device current, with cudaGetSymbolAddress; that first call also reads the
// device's SM count and shared-memory limit.  A call that would need more scratch than the array
// holds is rejected before anything is launched.
//
// All calls on one device share the one array: two calls whose work overlaps on the device (on
// different streams without ordering between them, or from several host threads) race on it and
// give wrong results.  Order such calls on one stream or with events.
#include <algorithm>
#include <mutex>

#include "kernels.cuh"

namespace dfs {
namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

// Layout: [DevStatus | U2 (2 KQ) | U2part (parts x 2 KQ) | Rpart (parts x n x KQ)], each 256-aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DFS_NOALLOC_SCRATCH_BYTES];

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];
// test hook (dfs_fisher_pass_noalloc_test_fault), per device
int g_test_fault[kMaxDevices] = {};
unsigned long long g_test_wait_ns[kMaxDevices] = {};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int pow2_ceil(int64_t k) {
    int p = 1;
    while (p < k && p < (1 << 20)) p <<= 1;
    return p;
}

size_t elem_bytes(int s_dtype) { return s_dtype == DFS_F64 ? 8 : (s_dtype == DFS_F32 ? 4 : 2); }

struct Layout {
    size_t off_u2, off_u2part, off_rpart, total;
};

Layout layout_for(int grid, int64_t n, int kq, bool with_r) {
    Layout l{};
    l.off_u2 = align_up(sizeof(DevStatus));
    l.off_u2part = l.off_u2 + align_up((size_t)2 * kq * sizeof(double));
    l.off_rpart = l.off_u2part + align_up((size_t)grid * 2 * kq * sizeof(double));
    l.total = l.off_rpart + (with_r ? (size_t)grid * (size_t)n * kq * sizeof(double) : 0);
    return l;
}

// Once per device, with that device current: the scratch address and the launch limits.
dfs_status setup_device(int dev, DeviceSetup* out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& d = g_setup[dev];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return DFS_ERR_CUDA;
        }
        int sms = 0, optin = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            return DFS_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char*>(p);
        d.num_sms = sms;
        d.smem_optin = (size_t)optin;
        d.ready = true;
    }
    *out = d;
    return DFS_OK;
}

}  // namespace
}  // namespace dfs

using namespace dfs;

extern "C" dfs_status dfs_fisher_pass_noalloc(const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds,
                                              const void* V, int64_t k, int64_t ldv, const double* Y, int64_t ldy,
                                              double lambda, void* X, int64_t ldx, double* R, int64_t ldr,
                                              void* stream_, int64_t* scratch_bytes) {
    if (scratch_bytes) *scratch_bytes = 0;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (s_dtype != DFS_F64 && s_dtype != DFS_F32 && s_dtype != DFS_BF16) return DFS_ERR_INVALID_ARG;
    if (!S || n < 1 || m < 1 || lds < m) return DFS_ERR_INVALID_ARG;
    if (n > 65536) return DFS_ERR_UNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(S) % 16 != 0 || (lds * (int64_t)elem_bytes(s_dtype)) % 16 != 0)
        return DFS_ERR_INVALID_ARG;
    if (!std::isfinite(lambda) || !(lambda > 0.0)) return DFS_ERR_INVALID_ARG;
    if (!V || k < 1 || ldv < m) return DFS_ERR_INVALID_ARG;
    if ((X && ldx < m) || (Y && ldy < k) || (R && ldr < k)) return DFS_ERR_INVALID_ARG;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DFS_ERR_CUDA;
    }
    DeviceSetup d;
    dfs_status s = setup_device(dev, &d);
    if (s != DFS_OK) return s;

    const int kmax = pass_max_group((int)n, s_dtype, d.smem_optin);
    if (kmax < 1) return DFS_ERR_UNSUPPORTED;
    // Right-hand sides per pass: as dfs_fisher_pass, halved while the partials do not fit.
    int kq = pow2_ceil(k);
    if (kq > kmax) kq = kmax;
    PassPlan pp = pass_make_plan((int)n, kq, s_dtype, d.num_sms, m, d.smem_optin, X != nullptr);
    Layout lay = layout_for(std::max(pp.nparts, pp.uparts), n, kq, R != nullptr);
    while (lay.total > DFS_NOALLOC_SCRATCH_BYTES && kq > 1) {
        kq >>= 1;
        pp = pass_make_plan((int)n, kq, s_dtype, d.num_sms, m, d.smem_optin, X != nullptr);
        lay = layout_for(std::max(pp.nparts, pp.uparts), n, kq, R != nullptr);
    }
    if (scratch_bytes) *scratch_bytes = (int64_t)lay.total;
    if (lay.total > DFS_NOALLOC_SCRATCH_BYTES) return DFS_ERR_NO_MEMORY;

    DevStatus* st = reinterpret_cast<DevStatus*>(d.scratch);
    double* U2part = reinterpret_cast<double*>(d.scratch + lay.off_u2part);
    double* Rpart = R ? reinterpret_cast<double*>(d.scratch + lay.off_rpart) : nullptr;
    const size_t vs = s_dtype == DFS_F64 ? 8 : 4;
    // The status word must start at zero (the pass kernels skip their work on a non-zero
    // status); the partials need no clearing: every CTA writes all of its own.
    if (launch_status_reset(st, stream, g_test_wait_ns[dev], g_test_fault[dev]) != cudaSuccess) return DFS_ERR_CUDA;
    for (int64_t q0 = 0; q0 < k; q0 += kq) {
        const int kg = (int)((k - q0) < kq ? (k - q0) : kq);
        const void* Vg = static_cast<const char*>(V) + q0 * ldv * vs;
        void* Xg = X ? static_cast<char*>(X) + q0 * ldx * vs : nullptr;
        const double* Yg = Y ? Y + q0 : nullptr;
        if (launch_pass(pp, s_dtype, kq, S, (int)n, m, lds, Vg, ldv, kg, Yg, Y ? ldy : kq, lambda, Xg, ldx, Rpart,
                        U2part, 0, st, 0, stream) != cudaSuccess)
            return DFS_ERR_CUDA;
        if (R && launch_pass_reduce(0, Rpart, pp.nparts, (int)n, (int)n, kq, kg, Yg, ldy, lambda, R + q0, ldr, nullptr,
                                    nullptr, nullptr, st, 0, stream) != cudaSuccess)
            return DFS_ERR_CUDA;
    }
    return DFS_OK;
}

extern "C" dfs_status dfs_fisher_pass_noalloc_status(int* status_out, void* stream_) {
    if (!status_out) return DFS_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DFS_ERR_CUDA;
    }
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (g_setup[dev].ready) scratch = g_setup[dev].scratch;
    }
    if (!scratch) return DFS_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    int v = 0;
    // the status word is the first member of the DevStatus at the start of the scratch
    if (cudaMemcpyAsync(&v, scratch, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return DFS_ERR_CUDA;
    }
    *status_out = v;
    return DFS_OK;
}

extern "C" dfs_status dfs_fisher_pass_noalloc_test_fault(int fault, int64_t wait_limit_ns) {
    if (fault < DFS_TEST_FAULT_NONE || fault > DFS_TEST_FAULT_FUSED_GRAM) return DFS_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DFS_ERR_CUDA;
    }
    g_test_fault[dev] = fault;
    g_test_wait_ns[dev] = wait_limit_ns > 0 ? (unsigned long long)wait_limit_ns : 0ull;
    return DFS_OK;
}
