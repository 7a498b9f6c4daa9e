// The two triangular solves of Section 2 (Q inlined): A = L^{-1} B, then Y = L^{-T} A.
//
// One CTA of 1024 threads (32 warps) walks the 32-row diagonal blocks of the padded factor L.
// The RHS block lives in shared memory for the whole solve (n_pad x KQ values).  Each block
// step is two warp-level GEMV pieces:
//   forward  t = B_i - L[i, <i] A_<i   (warp w owns row w of the block, lanes walk columns)
//            A_i = Linv_i t              (Linv_i = inverse of the 32 x 32 diagonal block)
//   backward t = A_i - L[>i, i]^T Y_>i  (lanes own the block's columns, warps walk rows)
//            Y_i = Linv_i^T t
// Products and sums are in the storage type of L (FP32 on the FP32/mixed paths, FP64 on the
// FP64 path).  With `stop` set in the device status (refinement already converged) the
// kernels return at once.
#include "kernels.cuh"

namespace dfs {

constexpr int TB = 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int KQ>
__global__ void __launch_bounds__(1024)
trsv_lower_kernel(const T* __restrict__ L, int64_t ld, int n_pad, const T* __restrict__ Linv,
                  T* __restrict__ B, int64_t ldb, int k, const DevStatus* st, int honor_stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* x = reinterpret_cast<T*>(smem);  // n_pad x KQ
    T* t = x + (int64_t)n_pad * KQ;     // TB x KQ
    if (block_should_exit(st, honor_stop)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < n_pad * KQ; e += blockDim.x) {
        const int i = e / KQ, q = e % KQ;
        x[e] = (q < k) ? B[(int64_t)i * ldb + q] : (T)0;
    }
    __syncthreads();
    const int nblk = n_pad / TB;
    for (int ib = 0; ib < nblk; ++ib) {
        const int r = ib * TB + warp;
        T acc[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q] = 0;
        const T* Lr = L + (int64_t)r * ld;
        const int cend = ib * TB;
#pragma unroll 4
        for (int c = lane; c < cend; c += 32) {
            const T l = Lr[c];
#pragma unroll
            for (int q = 0; q < KQ; ++q) acc[q] = fma(l, x[c * KQ + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < KQ; ++q) t[warp * KQ + q] = x[r * KQ + q] - acc[q];
        }
        __syncthreads();
        const T li = Linv[(int64_t)ib * TB * TB + warp * TB + lane];
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q] = warp_sum(li * t[lane * KQ + q]);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < KQ; ++q) x[r * KQ + q] = acc[q];
        }
        __syncthreads();
    }
    for (int e = tid; e < n_pad * KQ; e += blockDim.x) {
        const int i = e / KQ, q = e % KQ;
        if (q < k) B[(int64_t)i * ldb + q] = x[e];
    }
}

template <typename T, int KQ>
__global__ void __launch_bounds__(1024)
trsv_upper_t_kernel(const T* __restrict__ L, int64_t ld, int n_pad, const T* __restrict__ Linv,
                    T* __restrict__ B, int64_t ldb, int k, const DevStatus* st, int honor_stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* y = reinterpret_cast<T*>(smem);       // n_pad x KQ
    T* t = y + (int64_t)n_pad * KQ;          // TB x KQ
    T* red = t + TB * KQ;                    // 32 warps x TB x KQ
    if (block_should_exit(st, honor_stop)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < n_pad * KQ; e += blockDim.x) {
        const int i = e / KQ, q = e % KQ;
        y[e] = (q < k) ? B[(int64_t)i * ldb + q] : (T)0;
    }
    __syncthreads();
    const int nblk = n_pad / TB;
    for (int ib = nblk - 1; ib >= 0; --ib) {
        const int c = ib * TB + lane;
        T acc[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q] = 0;
#pragma unroll 4
        for (int r = (ib + 1) * TB + warp; r < n_pad; r += 32) {
            const T l = L[(int64_t)r * ld + c];
#pragma unroll
            for (int q = 0; q < KQ; ++q) acc[q] = fma(l, y[r * KQ + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < KQ; ++q) red[(warp * TB + lane) * KQ + q] = acc[q];
        __syncthreads();
        if (tid < TB * KQ) {
            const int cl = tid / KQ, q = tid % KQ;
            T s = 0;
            for (int w = 0; w < 32; ++w) s += red[(w * TB + cl) * KQ + q];
            t[cl * KQ + q] = y[(ib * TB + cl) * KQ + q] - s;
        }
        __syncthreads();
        // Y_i[w] = sum_p Linv[p][w] t[p]
        const T li = Linv[(int64_t)ib * TB * TB + lane * TB + warp];
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q] = warp_sum(li * t[lane * KQ + q]);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < KQ; ++q) y[(ib * TB + warp) * KQ + q] = acc[q];
        }
        __syncthreads();
    }
    for (int e = tid; e < n_pad * KQ; e += blockDim.x) {
        const int i = e / KQ, q = e % KQ;
        if (q < k) B[(int64_t)i * ldb + q] = y[e];
    }
}

size_t trsv_smem_bytes(int n_pad, int KQ, int elem) {
    return ((size_t)n_pad * KQ + TB * KQ + 32 * TB * KQ) * elem;
}

template <typename T, int KQ>
static cudaError_t launch_trsv_t(int trans, const void* L, int64_t ld, int n_pad, const void* Linv,
                                 void* B, int64_t ldb, int k, const DevStatus* st, int honor_stop,
                                 cudaStream_t stream) {
    const size_t smem = trsv_smem_bytes(n_pad, KQ, sizeof(T));
    if (trans) {
        auto kern = trsv_upper_t_kernel<T, KQ>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
            kern<<<1, 1024, smem, stream>>>(static_cast<const T*>(L), ld, n_pad, static_cast<const T*>(Linv),
                                            static_cast<T*>(B), ldb, k, st, honor_stop);
            count_launch();
        }
    } else {
        auto kern = trsv_lower_kernel<T, KQ>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
            kern<<<1, 1024, smem, stream>>>(static_cast<const T*>(L), ld, n_pad, static_cast<const T*>(Linv),
                                            static_cast<T*>(B), ldb, k, st, honor_stop);
            count_launch();
        }
    }
    return cudaGetLastError();
}

// Largest RHS group (1, 2, 4 or 8) whose shared-memory footprint fits.
int trsv_max_group(int n_pad, int elem, size_t smem_limit) {
    for (int kq = 8; kq >= 1; kq >>= 1)
        if (trsv_smem_bytes(n_pad, kq, elem) <= smem_limit) return kq;
    return 0;
}

cudaError_t launch_trsv(int f64, int trans, const void* L, int64_t ld, int n_pad, const void* Linv,
                        void* B, int64_t ldb, int k, int kq, const DevStatus* st, int honor_stop,
                        cudaStream_t stream) {
#define DFS_TRSV_CASE(KQ)                                                                              \
    case KQ:                                                                                           \
        return f64 ? launch_trsv_t<double, KQ>(trans, L, ld, n_pad, Linv, B, ldb, k, st, honor_stop, stream) \
                   : launch_trsv_t<float, KQ>(trans, L, ld, n_pad, Linv, B, ldb, k, st, honor_stop, stream);
    switch (kq) {
        DFS_TRSV_CASE(1)
        DFS_TRSV_CASE(2)
        DFS_TRSV_CASE(4)
        DFS_TRSV_CASE(8)
        default:
            return cudaErrorInvalidValue;
    }
#undef DFS_TRSV_CASE
}

}  // namespace dfs
