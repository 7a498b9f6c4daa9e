// Small data-movement kernels used at the C-ABI boundary (padding, layout changes).
#include "kernels.cuh"

namespace dfs {

// dst (n_pad x n_pad, ld n_pad) = lower triangle of src (n x n, ld lds), identity on the padding.
template <typename T>
__global__ void pad_copy_in_kernel(const T* src, int64_t lds, int64_t n, T* dst, int64_t n_pad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pad * n_pad) return;
    const int64_t i = e / n_pad, j = e % n_pad;
    if (j > i) return;
    T v;
    if (i < n && j < n) v = src[i * lds + j];
    else v = (i == j) ? (T)1 : (T)0;
    dst[e] = v;
}

template <typename T>
__global__ void copy_lower_out_kernel(const T* src, int64_t n_pad, T* dst, int64_t ldd, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e % n;
    if (j > i) return;
    dst[i * ldd + j] = src[i * n_pad + j];
}

// n-space vectors: caller layout (n rows, stride lds, k used) <-> internal (n_pad rows x KQ).
template <typename T>
__global__ void copy_rhs_in_kernel(const T* src, int64_t lds, int64_t n, int k, T* dst, int KQ, int64_t n_pad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pad * KQ) return;
    const int64_t i = e / KQ;
    const int q = (int)(e % KQ);
    dst[e] = (i < n && q < k) ? src[i * lds + q] : (T)0;
}

template <typename T>
__global__ void copy_rhs_out_kernel(const T* src, int KQ, int64_t n, int k, T* dst, int64_t ldd) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    const int64_t i = e / k;
    const int q = (int)(e % k);
    dst[i * ldd + q] = src[i * KQ + q];
}

__global__ void status_save_kernel(const DevStatus* st, int* dst) {
    if (threadIdx.x == 0) *dst = st->status;
}

__global__ void group_reset_kernel(DevStatus* st) {
    if (threadIdx.x == 0) {
        st->stop = 0;
        st->converged = 0;
        st->prev_correction = 0.0;
    }
}

static inline int blocks_for(int64_t total) { return (int)ceil_div(total, 256); }

cudaError_t launch_pad_copy_in(int f64, const void* src, int64_t lds, int64_t n, void* dst, int64_t n_pad,
                               cudaStream_t stream) {
    if (f64)
        {
            pad_copy_in_kernel<double><<<blocks_for(n_pad * n_pad), 256, 0, stream>>>(
                static_cast<const double*>(src), lds, n, static_cast<double*>(dst), n_pad);
            count_launch();
        }
    else
        {
            pad_copy_in_kernel<float><<<blocks_for(n_pad * n_pad), 256, 0, stream>>>(
                static_cast<const float*>(src), lds, n, static_cast<float*>(dst), n_pad);
            count_launch();
        }
    return cudaGetLastError();
}

cudaError_t launch_copy_lower_out(int f64, const void* src, int64_t n_pad, void* dst, int64_t ldd, int64_t n,
                                  cudaStream_t stream) {
    if (f64)
        {
            copy_lower_out_kernel<double><<<blocks_for(n * n), 256, 0, stream>>>(
                static_cast<const double*>(src), n_pad, static_cast<double*>(dst), ldd, n);
            count_launch();
        }
    else
        {
            copy_lower_out_kernel<float><<<blocks_for(n * n), 256, 0, stream>>>(
                static_cast<const float*>(src), n_pad, static_cast<float*>(dst), ldd, n);
            count_launch();
        }
    return cudaGetLastError();
}

cudaError_t launch_copy_rhs_in(int f64, const void* src, int64_t lds, int64_t n, int k, void* dst, int KQ,
                               int64_t n_pad, cudaStream_t stream) {
    if (f64)
        {
            copy_rhs_in_kernel<double><<<blocks_for(n_pad * KQ), 256, 0, stream>>>(
                static_cast<const double*>(src), lds, n, k, static_cast<double*>(dst), KQ, n_pad);
            count_launch();
        }
    else
        {
            copy_rhs_in_kernel<float><<<blocks_for(n_pad * KQ), 256, 0, stream>>>(
                static_cast<const float*>(src), lds, n, k, static_cast<float*>(dst), KQ, n_pad);
            count_launch();
        }
    return cudaGetLastError();
}

cudaError_t launch_copy_rhs_out(int f64, const void* src, int KQ, int64_t n, int k, void* dst, int64_t ldd,
                                cudaStream_t stream) {
    if (f64)
        {
            copy_rhs_out_kernel<double><<<blocks_for(n * k), 256, 0, stream>>>(
                static_cast<const double*>(src), KQ, n, k, static_cast<double*>(dst), ldd);
            count_launch();
        }
    else
        {
            copy_rhs_out_kernel<float><<<blocks_for(n * k), 256, 0, stream>>>(
                static_cast<const float*>(src), KQ, n, k, static_cast<float*>(dst), ldd);
            count_launch();
        }
    return cudaGetLastError();
}

cudaError_t launch_status_save(const DevStatus* st, int* dst, cudaStream_t stream) {
    {
        status_save_kernel<<<1, 32, 0, stream>>>(st, dst);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_group_reset(DevStatus* st, cudaStream_t stream) {
    {
        group_reset_kernel<<<1, 32, 0, stream>>>(st);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace dfs
