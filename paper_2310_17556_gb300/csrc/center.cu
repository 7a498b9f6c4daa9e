// Centred score matrices for stochastic reconfiguration (Section 4 of arXiv 2310.17556):
// S = (O - O_bar) / sqrt(n), O_bar the average of O over the n samples (rows).  With the
// centring matrix P = I - 1 1^T / n, S = P O / sqrt(n), so everything Algorithm 1 needs from S
// follows from O and n-space work only; the passes over O are unchanged:
//   W     = S S^T + lambda I = P (O O^T / n) P + lambda I      (Gram of O, then centred here)
//   b     = S v              = P (O v) / sqrt(n)
//   S^T y = O^T (P y / sqrt(n))                               (a pass over O with y_hat = P y / sqrt(n))
//   r     = S u - lambda y   = P (O u) / sqrt(n) - lambda y    (the refinement residual)
// Sums run in FP64 in a fixed order (no atomics), so results do not vary run to run.
#include "kernels.cuh"

namespace dfs {

namespace {

constexpr int CG_THREADS = 256;

__device__ __forceinline__ double block_sum_256(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < CG_THREADS / 32; ++w) t += red[w];
    return t;  // valid in thread 0
}

}  // namespace

// rl[i] = sum_{k <= i} W[i][k] (the row of the stored lower triangle), one CTA per row.
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) center_rowsum_kernel(const T* __restrict__ W, int64_t ld, int n,
                                                                   double* __restrict__ rl) {
    __shared__ double red[CG_THREADS / 32];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k <= i; k += CG_THREADS) s += (double)W[(int64_t)i * ld + k];
    const double t = block_sum_256(s, red);
    if (threadIdx.x == 0) rl[i] = t;
}

// cl[c] = sum_{i > c} W[i][c] (the column below the diagonal), one CTA per 32 columns: thread
// (c = tid % 32, g = tid / 32) takes rows c0 + 1 + g, + 8, ... (coalesced 128-byte row pieces).
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) center_colsum_kernel(const T* __restrict__ W, int64_t ld, int n,
                                                                   double* __restrict__ cl) {
    __shared__ double part[CG_THREADS / 32][33];
    const int cc = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cc;
    double s = 0.0;
    for (int i = blockIdx.x * 32 + 1 + g; i < n; i += CG_THREADS / 32)
        if (c < i) s += (double)W[(int64_t)i * ld + c];
    part[g][cc] = s;
    __syncthreads();
    if (g == 0 && c < n) {
        double t = 0.0;
        for (int q = 0; q < CG_THREADS / 32; ++q) t += part[q][cc];
        cl[c] = t;
    }
}

// gm[i] = (rl[i] + cl[i]) / n, the mean of row i of the symmetric G; gm[n] = mean of all of G.
__global__ void __launch_bounds__(CG_THREADS) center_means_kernel(const double* __restrict__ rl,
                                                                  const double* __restrict__ cl, int n,
                                                                  double* __restrict__ gm) {
    __shared__ double red[CG_THREADS / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += CG_THREADS) {
        const double r = (rl[i] + cl[i]) / (double)n;
        gm[i] = r;
        s += r;
    }
    const double t = block_sum_256(s, red);
    if (threadIdx.x == 0) gm[n] = t / (double)n;
}

// W[i][k] <- (G_ik - gm_i - gm_k + gm_n) / n + lambda [i == k] for k <= i < n (P G P / n + lambda I).
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) center_apply_kernel(T* __restrict__ W, int64_t ld, int n,
                                                                  const double* __restrict__ gm, double lambda) {
    const int i = blockIdx.x;
    const double gi = gm[i], gb = gm[n], inv_n = 1.0 / (double)n;
    for (int k = threadIdx.x; k <= i; k += CG_THREADS) {
        T* w = W + (int64_t)i * ld + k;
        *w = (T)(((double)*w - gi - gm[k] + gb) * inv_n + (i == k ? lambda : 0.0));
    }
}

// n-space vectors (n_pad x KQ row-major, FP64), one CTA of 1024 threads.
//   mode 0: R <- P R / sqrt(n) - lambda Y (no lambda term when Y is null), Z <- R (solve type T);
//   mode 1: Yc <- P Y / sqrt(n).
// Rows in [n, n_pad) and columns q >= k are set to zero.  Skips its work once the device status
// is set, or (honor_stop) once refinement has stopped.
template <typename T>
__global__ void __launch_bounds__(1024) center_vec_kernel(int mode, int n, int n_pad, int KQ, int k,
                                                          double* __restrict__ R, const double* __restrict__ Y,
                                                          double lambda, T* __restrict__ Z, double* __restrict__ Yc,
                                                          const DevStatus* st, int honor_stop) {
    __shared__ double red[32][8];
    __shared__ double mean[8];
    if (st->status != 0 || (honor_stop && st->stop)) return;
    const double* src = mode == 0 ? R : Y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int q = 0; q < KQ; ++q) {
        double s = 0.0;
        if (q < k)
            for (int i = tid; i < n; i += 1024) s += src[(int64_t)i * KQ + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][q] = s;
    }
    __syncthreads();
    if (tid < KQ) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += red[w][tid];
        mean[tid] = t / (double)n;
    }
    __syncthreads();
    const double rsn = 1.0 / sqrt((double)n);
    for (int64_t e = tid; e < (int64_t)n_pad * KQ; e += 1024) {
        const int i = (int)(e / KQ), q = (int)(e % KQ);
        const bool live = i < n && q < k;
        if (mode == 0) {
            double t = live ? (R[e] - mean[q]) * rsn : 0.0;
            if (live && Y != nullptr) t -= lambda * Y[e];
            R[e] = t;
            Z[e] = (T)t;
        } else {
            Yc[e] = live ? (Y[e] - mean[q]) * rsn : 0.0;
        }
    }
}

cudaError_t launch_center_gram(int f64, void* W, int64_t ld, int n, double* scratch, double lambda,
                               cudaStream_t stream) {
    double* rl = scratch;
    double* cl = scratch + n;
    double* gm = scratch + 2 * (int64_t)n;  // n + 1 entries
    const int cblocks = (n + 31) / 32;
    if (f64) {
        center_rowsum_kernel<double><<<n, CG_THREADS, 0, stream>>>(static_cast<const double*>(W), ld, n, rl);
        center_colsum_kernel<double><<<cblocks, CG_THREADS, 0, stream>>>(static_cast<const double*>(W), ld, n, cl);
    } else {
        center_rowsum_kernel<float><<<n, CG_THREADS, 0, stream>>>(static_cast<const float*>(W), ld, n, rl);
        center_colsum_kernel<float><<<cblocks, CG_THREADS, 0, stream>>>(static_cast<const float*>(W), ld, n, cl);
    }
    center_means_kernel<<<1, CG_THREADS, 0, stream>>>(rl, cl, n, gm);
    if (f64)
        center_apply_kernel<double><<<n, CG_THREADS, 0, stream>>>(static_cast<double*>(W), ld, n, gm, lambda);
    else
        center_apply_kernel<float><<<n, CG_THREADS, 0, stream>>>(static_cast<float*>(W), ld, n, gm, lambda);
    for (int l = 0; l < 4; ++l) count_launch();
    return cudaGetLastError();
}

size_t center_gram_scratch_doubles(int64_t n) { return 3 * (size_t)n + 1; }

cudaError_t launch_center_vec(int f64, int mode, int n, int n_pad, int KQ, int k, double* R, const double* Y,
                              double lambda, void* Z, double* Yc, const DevStatus* st, int honor_stop,
                              cudaStream_t stream) {
    if (KQ > 8) return cudaErrorInvalidValue;
    if (f64)
        center_vec_kernel<double><<<1, 1024, 0, stream>>>(mode, n, n_pad, KQ, k, R, Y, lambda,
                                                          static_cast<double*>(Z), Yc, st, honor_stop);
    else
        center_vec_kernel<float><<<1, 1024, 0, stream>>>(mode, n, n_pad, KQ, k, R, Y, lambda, static_cast<float*>(Z),
                                                         Yc, st, honor_stop);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dfs
