// Complex score matrices (Section 4 of arXiv 2310.17556, complex SR with F = S^dagger S): the
// real 2n x 2m representation of S = A + iB,
//   R(S) = [[A, -B],
//           [B,  A]],
// satisfies R(S)^T R(S) = R(S^dagger S) and R(S) [Re x; Im x] = [Re(S x); Im(S x)], so
// (S^dagger S + lambda I) x = v is the real Eq. 1 for R(S), [Re x; Im x] and [Re v; Im v].
// This kernel writes R(S) from the two planes; the real solver does the rest.
#include "kernels.cuh"

namespace dfs {

template <typename T>
__device__ __forceinline__ T negate(T x) {
    return -x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 negate<__nv_bfloat16>(__nv_bfloat16 x) {
    return __hneg(x);
}

// One CTA row per source row i (blockIdx.y), threads over columns: R[i][j] = A, R[i][m + j] = -B,
// R[n + i][j] = B, R[n + i][m + j] = A.  ldr >= 2m.
template <typename T>
__global__ void __launch_bounds__(256) complex_embed_kernel(const T* __restrict__ A, const T* __restrict__ B,
                                                            int64_t n, int64_t m, int64_t lds, T* __restrict__ R,
                                                            int64_t ldr) {
    const int64_t i = blockIdx.y;
    const T* a = A + i * lds;
    const T* b = B + i * lds;
    T* top = R + i * ldr;
    T* bot = R + (n + i) * ldr;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const T x = a[j], y = b[j];
        top[j] = x;
        top[m + j] = negate(y);
        bot[j] = y;
        bot[m + j] = x;
    }
}

cudaError_t launch_complex_embed(int s_dtype, const void* A, const void* B, int64_t n, int64_t m, int64_t lds, void* R,
                                 int64_t ldr, cudaStream_t stream) {
    if (n > 65535) return cudaErrorInvalidValue;
    const int64_t want = (m + 255) / 256;
    const dim3 grid((unsigned)(want < 64 ? want : 64), (unsigned)n);
    switch (s_dtype) {
        case DFS_F32:
            complex_embed_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float*>(A),
                                                                  static_cast<const float*>(B), n, m, lds,
                                                                  static_cast<float*>(R), ldr);
            break;
        case DFS_F64:
            complex_embed_kernel<double><<<grid, 256, 0, stream>>>(static_cast<const double*>(A),
                                                                   static_cast<const double*>(B), n, m, lds,
                                                                   static_cast<double*>(R), ldr);
            break;
        case DFS_BF16:
            complex_embed_kernel<__nv_bfloat16><<<grid, 256, 0, stream>>>(
                static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), n, m, lds,
                static_cast<__nv_bfloat16*>(R), ldr);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace dfs
