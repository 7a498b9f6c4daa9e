// Shared device/host helpers of libdfs (internal header, not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/dfs.h"

namespace dfs {

constexpr int kNumSmsGB300 = 152;

// Number of kernels this library has launched in the process (reported by dfs_kernel_launches).
std::atomic<long long>& launch_counter();
inline void count_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }

// Device-side status word layout (int32 array in the handle's workspace).
//   [0] status (dfs_status), [1] failed pivot (int, -1 none), [2] converged flag,
//   [3] refinement passes done, [4] stop flag (set once converged or diverged)
struct DevStatus {
    int status;
    int failed_pivot;
    int converged;
    int iters;
    int stop;
    int passes;  // full passes over S run by the refinement (a tile correction does not count)
    int fault;   // test hook: DFS_TEST_FAULT_* of the call (0 normally), set by the status reset
    int bounds_site;  // debug build: site of the first failed index check (file id * 100000 + line)
    double rel_correction;
    double rel_residual;
    double prev_correction;
    unsigned long long wait_ns;  // limit of every bounded device wait of the call (ns)
};

constexpr unsigned long long kDefaultWaitNs = 2000000000ull;  // 2 s

// The limit of the bounded waits of the call that owns `st` (the default if it was never set).
__device__ __forceinline__ unsigned long long wait_limit(const DevStatus* st) {
    const unsigned long long w = *reinterpret_cast<const volatile unsigned long long*>(&st->wait_ns);
    return w ? w : kDefaultWaitNs;
}
__device__ __forceinline__ int test_fault(const DevStatus* st) {
    return *reinterpret_cast<const volatile int*>(&st->fault);
}

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return (float)x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T>
struct Vec16;  // 16-byte vector load of storage type T, unpacked to the accumulate type
template <>
struct Vec16<float> {
    static constexpr int N = 4;
};
template <>
struct Vec16<double> {
    static constexpr int N = 2;
};
template <>
struct Vec16<__nv_bfloat16> {
    static constexpr int N = 8;
};

// Load 16 bytes from global memory (read-only path) and unpack to N values of type A.
template <typename T, typename A>
__device__ __forceinline__ void load16(const T* p, A* out);

template <>
__device__ __forceinline__ void load16<float, float>(const float* p, float* o) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load16<float, double>(const float* p, double* o) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load16<double, double>(const double* p, double* o) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
}
template <>
__device__ __forceinline__ void load16<__nv_bfloat16, float>(const __nv_bfloat16* p, float* o) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(w[i] << 16);
        o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// Streaming (evict-first) 16-byte load for data read exactly once.
template <typename T, typename A>
__device__ __forceinline__ void load16_stream(const T* p, A* out);
template <>
__device__ __forceinline__ void load16_stream<float, float>(const float* p, float* o) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load16_stream<double, double>(const double* p, double* o) {
    double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
}
template <>
__device__ __forceinline__ void load16_stream<__nv_bfloat16, float>(const __nv_bfloat16* p, float* o) {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(w[i] << 16);
        o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// 16-byte load from shared memory, unpacked to the accumulate type.
template <typename T, typename A>
__device__ __forceinline__ void load16_smem(const T* p, A* out);
template <>
__device__ __forceinline__ void load16_smem<float, float>(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load16_smem<double, double>(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
}
template <>
__device__ __forceinline__ void load16_smem<__nv_bfloat16, float>(const __nv_bfloat16* p, float* o) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(w[i] << 16);
        o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// Scalar guarded load (tails).
template <typename T, typename A>
__device__ __forceinline__ A load1(const T* p) {
    return (A)(*p);
}
template <>
__device__ __forceinline__ float load1<__nv_bfloat16, float>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ double load1<__nv_bfloat16, double>(const __nv_bfloat16* p) {
    return (double)__bfloat162float(*p);
}

__host__ __device__ constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

__device__ __forceinline__ void set_status(DevStatus* st, int code) {
    atomicCAS(&st->status, 0, code);
}

// ---- index checks of the debug build ----
// Built with -DDFS_DEBUG_BOUNDS (build.py --debug-bounds, a separate libdfs_debug.so),
// DFS_IN_BOUNDS(st, cond) tests the index condition of a global memory access: when it fails,
// the first failure records DFS_ERR_BOUNDS and its site (DFS_SRC_ID * 100000 + line) in the
// device status and the caller skips the access (a copy that others wait for aborts its loop,
// so their bounded waits end).  Nothing traps.  In other builds every check is the constant true.
// A source file defines DFS_SRC_ID before its includes.
#ifndef DFS_SRC_ID
#define DFS_SRC_ID 0
#endif
#ifdef DFS_DEBUG_BOUNDS
static __device__ __noinline__ bool dfs_bounds_fail(const DevStatus* st, int site) {
    if (st != nullptr) {
        DevStatus* s = const_cast<DevStatus*>(st);
        atomicCAS(&s->bounds_site, 0, site);
        atomicCAS(&s->status, 0, (int)DFS_ERR_BOUNDS);
    }
    return false;
}
#define DFS_IN_BOUNDS(st, cond) ((cond) || ::dfs::dfs_bounds_fail((st), DFS_SRC_ID * 100000 + __LINE__))
#else
#define DFS_IN_BOUNDS(st, cond) true
#endif

// Block-uniform early exit: thread 0 reads the device status once (another CTA may change it
// while this one runs), all threads see the same answer.  Contains a __syncthreads().
__device__ __forceinline__ bool block_should_exit(const DevStatus* st, int honor_stop) {
    __shared__ int s_exit;
    if (threadIdx.x == 0) {
        const volatile DevStatus* v = st;
        s_exit = (v->status != 0) || (honor_stop && v->stop);
    }
    __syncthreads();
    return s_exit != 0;
}

}  // namespace dfs
