// Throughput probes for the roofline denominators the SIMT kernels need: FP32 fused multiply-add
// (the plain FP32 path's Gram runs on it) and FP64 fused multiply-add (the FP64 path and the
// optional FP64 Cholesky panel).  Each thread runs kChains independent multiply-add chains (enough
// to cover the pipeline latency) for a fixed count; a grid of several CTAs per SM keeps every SM
// busy.  The result is stored so that the work cannot be dropped.  These kernels change no GPU
// setting; they only measure.
#include "kernels.cuh"

namespace dfs {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
double run_fma_probe(int num_sms, int iters) {
    const int grid = num_sms * 8;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)grid * kThreads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a < 1 keeps the chains bounded: x -> b / (1 - a)
    const T a = (T)0.999, b = (T)1e-3;
    fma_chain_kernel<T><<<grid, kThreads>>>(out, iters > 8 ? iters / 8 : 1, a, b);  // warm-up
    cudaEventRecord(e0);
    fma_chain_kernel<T><<<grid, kThreads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return -1.0;
    const double fmas = (double)grid * kThreads * (double)iters * 16 * kChains;
    return 2.0 * fmas / (ms * 1e-3);  // flop/s (2 per fused multiply-add)
}

}  // namespace

}  // namespace dfs

using namespace dfs;

extern "C" dfs_status dfs_measure_peak(int kind, double* flops_per_s) {
    if (!flops_per_s || (kind != DFS_PEAK_FFMA32 && kind != DFS_PEAK_DFMA64)) return DFS_ERR_INVALID_ARG;
    *flops_per_s = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return DFS_ERR_CUDA;
    }
    // about 0.1-0.3 s of work at the expected rates (~80 TFLOP/s FP32, ~1.2 TFLOP/s FP64 on GB300)
    const double r = kind == DFS_PEAK_FFMA32 ? run_fma_probe<float>(sms, 128) : run_fma_probe<double>(sms, 4);
    if (r <= 0.0) return DFS_ERR_CUDA;
    *flops_per_s = r;
    return DFS_OK;
}
