// Streaming passes over S (HBM-bound): Algorithm 1 step 4 with Q inlined, plus the n-space
// residual used by iterative refinement, both in ONE read of S.
//
//   U = V - S^T Y                 (S^T y: the leftmost product of S^T L^{-T} L^{-1} S v)
//   X = U / lambda                (Algorithm 1 step 4)
//   R = S U - lambda Y            (= S v - (S S^T + lambda I~) y, Appendix A's identity)
//
// S is n x m row-major.  A CTA owns a strip of 128 bytes of columns (W = 8 * VEC columns) over
// all n rows: 8 lanes cover one row segment with 16-byte loads, a warp covers 4 rows, 16 warps
// cover 64 rows per sweep.  Phase 1 reduces S^T Y over the rows of the strip (FP32 products,
// per-thread FP32 partials, cross-warp sum in FP64); phase 2 re-reads the strip (L1/L2 hits)
// and adds the strip's contribution S U into a per-CTA FP64 accumulator R_s in shared memory.
// The grid is persistent (strips round-robin over CTAs); each CTA finally writes its R_s and
// its sum of U^2 (for ||X||) to a partial buffer that pass_reduce sums in a fixed order.
#include "kernels.cuh"

namespace dfs {

constexpr int PASS_THREADS = 512;
constexpr int PASS_WARPS = PASS_THREADS / 32;
constexpr int PASS_ROWS = PASS_WARPS * 4;  // rows per sweep

template <typename TS>
struct PassTypes {
    using TA = float;  // accumulate / V / X type
};
template <>
struct PassTypes<double> {
    using TA = double;
};

template <typename TS, int KQ>
__global__ void __launch_bounds__(PASS_THREADS)
fisher_pass_kernel(const TS* __restrict__ S, int n, int64_t m, int64_t lds,
                   const typename PassTypes<TS>::TA* __restrict__ V, int64_t ldv, int k,
                   const double* __restrict__ Y, int64_t ldy, double lambda,
                   typename PassTypes<TS>::TA* __restrict__ X, int64_t ldx,
                   double* __restrict__ Rpart, double* __restrict__ U2part,
                   const DevStatus* st, int honor_stop) {
    using TA = typename PassTypes<TS>::TA;
    constexpr int VEC = Vec16<TS>::N;
    constexpr int W = 8 * VEC;
    extern __shared__ __align__(16) unsigned char smem[];
    double* Rs = reinterpret_cast<double*>(smem);                 // n x KQ
    TA* Ys = reinterpret_cast<TA*>(Rs + (int64_t)n * KQ);         // n x KQ
    TA* ured = Ys + (int64_t)n * KQ;                              // PASS_WARPS x W x KQ
    TA* us = ured + PASS_WARPS * W * KQ;                          // W x KQ
    if (st->status != 0 || (honor_stop && st->stop)) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rr = lane >> 3, cq = lane & 7;
    const bool haveY = (Y != nullptr);
    const bool wantR = (Rpart != nullptr);
    for (int e = tid; e < n * KQ; e += PASS_THREADS) {
        const int i = e / KQ, q = e % KQ;
        Rs[e] = 0.0;
        Ys[e] = (haveY && q < k) ? (TA)Y[(int64_t)i * ldy + q] : (TA)0;
    }
    double u2[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) u2[q] = 0.0;
    __syncthreads();

    const int64_t nstrips = ceil_div(m, W);
    for (int64_t s = blockIdx.x; s < nstrips; s += gridDim.x) {
        const int64_t j0 = s * W;
        const int64_t jc = j0 + cq * VEC;
        const bool full = (j0 + W <= m);
        // ---- phase 1: column sums of S^T Y over the strip -------------------------------
        if (haveY) {
            TA acc[KQ][VEC];
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc[q][e] = 0;
            int i = warp * 4 + rr;
            for (; i + 3 * PASS_ROWS < n; i += 4 * PASS_ROWS) {
                TA sv[4][VEC];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const TS* p = S + (int64_t)(i + u * PASS_ROWS) * lds + jc;
                    if (full) {
                        load16<TS, TA>(p, sv[u]);
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e) sv[u][e] = (jc + e < m) ? load1<TS, TA>(p + e) : (TA)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        const TA yv = Ys[(i + u * PASS_ROWS) * KQ + q];
#pragma unroll
                        for (int e = 0; e < VEC; ++e) acc[q][e] = fma(sv[u][e], yv, acc[q][e]);
                    }
            }
            for (; i < n; i += PASS_ROWS) {
                TA sv[VEC];
                const TS* p = S + (int64_t)i * lds + jc;
                if (full) {
                    load16<TS, TA>(p, sv);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) sv[e] = (jc + e < m) ? load1<TS, TA>(p + e) : (TA)0;
                }
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    const TA yv = Ys[i * KQ + q];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) acc[q][e] = fma(sv[e], yv, acc[q][e]);
                }
            }
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    TA v = acc[q][e];
                    v += __shfl_xor_sync(0xffffffffu, v, 8);
                    v += __shfl_xor_sync(0xffffffffu, v, 16);
                    acc[q][e] = v;
                }
            if (rr == 0) {
#pragma unroll
                for (int q = 0; q < KQ; ++q)
#pragma unroll
                    for (int e = 0; e < VEC; ++e) ured[(warp * W + cq * VEC + e) * KQ + q] = acc[q][e];
            }
        }
        __syncthreads();
        // ---- U = V - S^T Y, X = U / lambda --------------------------------------------------
        if (tid < W * KQ) {
            const int c = tid / KQ, q = tid % KQ;
            const int64_t j = j0 + c;
            double sum = 0.0;
            if (haveY)
                for (int w = 0; w < PASS_WARPS; ++w) sum += (double)ured[(w * W + c) * KQ + q];
            const bool valid = (j < m) && (q < k);
            const double v = valid ? (double)V[(int64_t)q * ldv + j] : 0.0;
            const double u = valid ? v - sum : 0.0;
            us[c * KQ + q] = (TA)u;
            if (valid) {
                if (X != nullptr) X[(int64_t)q * ldx + j] = (TA)(u / lambda);
                u2[q] += u * u;
            }
        }
        __syncthreads();
        // ---- phase 2: R_s += S_strip U_strip ------------------------------------------------
        if (wantR) {
            TA uu[KQ][VEC];
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) uu[q][e] = us[(cq * VEC + e) * KQ + q];
            // The row loop is warp-uniform (the shuffles below need all 32 lanes); rows past n
            // are predicated off.
            for (int ib = warp * 4; ib < n; ib += PASS_ROWS) {
                const int i = ib + rr;
                const bool ok = i < n;
                TA sv[VEC];
                const TS* p = S + (int64_t)i * lds + jc;
                if (ok && full) {
                    load16<TS, TA>(p, sv);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) sv[e] = (ok && jc + e < m) ? load1<TS, TA>(p + e) : (TA)0;
                }
                TA pr[KQ];
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    TA a = 0;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) a = fma(sv[e], uu[q][e], a);
                    a += __shfl_xor_sync(0xffffffffu, a, 1);
                    a += __shfl_xor_sync(0xffffffffu, a, 2);
                    a += __shfl_xor_sync(0xffffffffu, a, 4);
                    pr[q] = a;
                }
                if (ok && cq == 0) {
#pragma unroll
                    for (int q = 0; q < KQ; ++q) Rs[i * KQ + q] += (double)pr[q];
                }
            }
        }
    }
    __syncthreads();
    if (wantR) {
        double* dst = Rpart + (int64_t)blockIdx.x * n * KQ;
        for (int e = tid; e < n * KQ; e += PASS_THREADS) dst[e] = Rs[e];
    }
    // sum of U^2 per RHS: threads tid < W*KQ hold disjoint columns; reduce through smem
    __shared__ double u2s[PASS_THREADS / 32][8];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        double v = u2[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) u2s[warp][q] = v;
    }
    __syncthreads();
    if (tid < KQ) {
        double v = 0.0;
        for (int w = 0; w < PASS_WARPS; ++w) v += u2s[w][tid];
        U2part[(int64_t)blockIdx.x * KQ + tid] = v;
    }
}

// R = sum_b Rpart[b] - lambda Y (FP64, fixed order), rows [0, n_out) with stride ldr (rows >= n
// are zero), an optional copy Rt (n_out x KQ, solve type T) for the triangular solves, and the
// summed ||U||^2 per RHS.
template <typename T>
__global__ void __launch_bounds__(256)
pass_reduce_kernel(const double* __restrict__ Rpart, int nparts, int n, int n_out, int KQ, int k,
                   const double* __restrict__ Y, int64_t ldy, double lambda, double* __restrict__ R, int64_t ldr,
                   T* __restrict__ Rt, const double* __restrict__ U2part, double* __restrict__ U2,
                   const DevStatus* st, int honor_stop) {
    if (st->status != 0 || (honor_stop && st->stop)) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)n_out * KQ) {
        const int i = (int)(e / KQ), q = (int)(e % KQ);
        double v = 0.0;
        if (i < n && q < k) {
            for (int b = 0; b < nparts; ++b) v += Rpart[(int64_t)b * n * KQ + e];
            if (Y != nullptr) v -= lambda * Y[(int64_t)i * ldy + q];
        }
        if (R != nullptr && q < k) R[(int64_t)i * ldr + q] = v;
        if (Rt != nullptr) Rt[e] = (T)v;
    }
    if (U2 != nullptr && blockIdx.x == 0 && threadIdx.x < KQ) {
        double v = 0.0;
        for (int b = 0; b < nparts; ++b) v += U2part[(int64_t)b * KQ + threadIdx.x];
        U2[threadIdx.x] = v;
    }
}

size_t pass_smem_bytes(int n, int KQ, int s_dtype) {
    const int ta = (s_dtype == DFS_F64) ? 8 : 4;
    const int vec = (s_dtype == DFS_F64) ? 2 : (s_dtype == DFS_F32 ? 4 : 8);
    const int W = 8 * vec;
    return (size_t)n * KQ * 8 + (size_t)n * KQ * ta + (size_t)PASS_WARPS * W * KQ * ta + (size_t)W * KQ * ta;
}

int pass_max_group(int n, int s_dtype, size_t smem_limit) {
    for (int kq = 8; kq >= 1; kq >>= 1)
        if (pass_smem_bytes(n, kq, s_dtype) <= smem_limit) return kq;
    return 0;
}

template <typename TS, int KQ>
static cudaError_t launch_pass_t(const void* S, int n, int64_t m, int64_t lds, const void* V, int64_t ldv,
                                 int k, const double* Y, int64_t ldy, double lambda, void* X, int64_t ldx,
                                 double* Rpart, double* U2part, int grid, const DevStatus* st, int honor_stop,
                                 cudaStream_t stream, int s_dtype) {
    using TA = typename PassTypes<TS>::TA;
    const size_t smem = pass_smem_bytes(n, KQ, s_dtype);
    auto kern = fisher_pass_kernel<TS, KQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, PASS_THREADS, smem, stream>>>(static_cast<const TS*>(S), n, m, lds, static_cast<const TA*>(V),
                                               ldv, k, Y, ldy, lambda, static_cast<TA*>(X), ldx, Rpart, U2part,
                                               st, honor_stop);
    return cudaGetLastError();
}

int pass_grid(int n, int KQ, int s_dtype, int num_sms, int64_t m) {
    const size_t smem = pass_smem_bytes(n, KQ, s_dtype);
    int per_sm = (int)((200u * 1024u) / (smem + 1024));
    if (per_sm > 4) per_sm = 4;  // 4 x 512 threads = 2048 = SM thread limit
    if (per_sm < 1) per_sm = 1;
    const int vec = (s_dtype == DFS_F64) ? 2 : (s_dtype == DFS_F32 ? 4 : 8);
    const int64_t nstrips = ceil_div(m, 8 * vec);
    int64_t g = (int64_t)num_sms * per_sm;
    if (g > nstrips) g = nstrips;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_pass(int s_dtype, int kq, const void* S, int n, int64_t m, int64_t lds, const void* V,
                        int64_t ldv, int k, const double* Y, int64_t ldy, double lambda, void* X, int64_t ldx,
                        double* Rpart, double* U2part, int grid, const DevStatus* st, int honor_stop,
                        cudaStream_t stream) {
#define DFS_PASS_CASE(KQ)                                                                                     \
    case KQ:                                                                                                  \
        if (s_dtype == DFS_F32)                                                                               \
            return launch_pass_t<float, KQ>(S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart, U2part,   \
                                            grid, st, honor_stop, stream, s_dtype);                           \
        if (s_dtype == DFS_BF16)                                                                              \
            return launch_pass_t<__nv_bfloat16, KQ>(S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart,   \
                                                    U2part, grid, st, honor_stop, stream, s_dtype);           \
        if (s_dtype == DFS_F64)                                                                               \
            return launch_pass_t<double, KQ>(S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart, U2part,  \
                                             grid, st, honor_stop, stream, s_dtype);                          \
        return cudaErrorInvalidValue;
    switch (kq) {
        DFS_PASS_CASE(1)
        DFS_PASS_CASE(2)
        DFS_PASS_CASE(4)
        DFS_PASS_CASE(8)
        default:
            return cudaErrorInvalidValue;
    }
#undef DFS_PASS_CASE
}

cudaError_t launch_pass_reduce(int f64, const double* Rpart, int nparts, int n, int n_out, int KQ, int k,
                               const double* Y, int64_t ldy, double lambda, double* R, int64_t ldr, void* Rt,
                               const double* U2part, double* U2, const DevStatus* st, int honor_stop,
                               cudaStream_t stream) {
    const int64_t total = (int64_t)n_out * KQ;
    const int blocks = (int)ceil_div(total, 256);
    if (f64)
        pass_reduce_kernel<double><<<blocks, 256, 0, stream>>>(Rpart, nparts, n, n_out, KQ, k, Y, ldy, lambda, R, ldr,
                                                               static_cast<double*>(Rt), U2part, U2, st, honor_stop);
    else
        pass_reduce_kernel<float><<<blocks, 256, 0, stream>>>(Rpart, nparts, n, n_out, KQ, k, Y, ldy, lambda, R, ldr,
                                                              static_cast<float*>(Rt), U2part, U2, st, honor_stop);
    return cudaGetLastError();
}

}  // namespace dfs
