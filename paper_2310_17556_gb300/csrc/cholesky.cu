// Algorithm 1 step 2: L = Chol(W), W = L L^T, L lower triangular with a positive diagonal.
//
// Blocked right-looking factorisation of the padded n_pad x n_pad matrix W (row-major, lower
// triangle), with NB = 32 diagonal blocks:
//   step kb:  for every trailing tile (I, J) (TU x TU, I >= J) below/right of block kb,
//               P_r = A[r, kb] Linv_kb^T,  P_q = A[q, kb] Linv_kb^T     (panel TRSM, recomputed)
//               A[r, q] -= P_r P_q^T                                     (SYRK/GEMM update)
//             and the CTA owning the next diagonal block factors it right after its update.
//   each diagonal block is factored in FP64 (whatever the storage type) and its inverse
//   Linv_kb is kept for the panel TRSM and for the triangular solves.
//   after the last step, one kernel scales every panel: L[i, kb] = A[i, kb] Linv_kb^T.
// The panels are left unscaled while the steps run, so no CTA ever reads a value another CTA
// of the same launch writes.  A pivot <= 0 (or NaN/Inf) sets DFS_ERR_NOT_SPD and the pivot
// index in the device status; later steps see the status and return without work.
#include "kernels.cuh"

namespace dfs {

constexpr int NB = 32;
constexpr int TU = 64;

// Inverse of a lower-triangular NB x NB block held in shared memory (FP64), one column per
// thread by forward substitution; written to dst (NB x NB row-major, zeros above the diagonal).
template <typename T>
__device__ void invert_lower_block(const double (*a)[NB + 1], double (*inv)[NB + 1], T* dst) {
    const int tid = threadIdx.x;
    if (tid < NB) {
        const int c = tid;
        for (int i = 0; i < c; ++i) inv[i][c] = 0.0;
        inv[c][c] = 1.0 / a[c][c];
        for (int i = c + 1; i < NB; ++i) {
            double s = 0.0;
            for (int p = c; p < i; ++p) s = fma(a[i][p], inv[p][c], s);
            inv[i][c] = -s / a[i][i];
        }
    }
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) dst[e] = (T)inv[e / NB][e % NB];
    __syncthreads();
}

// Factor diagonal block kb in FP64 and write L_kb (storage type T) plus its inverse.
// Needs blockDim.x >= 32 and `scratch` >= 2 * NB * (NB + 1) doubles of shared memory.
template <typename T>
__device__ void factor_diag_block(T* W, int64_t ld, int kb, T* Linv, DevStatus* st, double* scratch) {
    double(*a)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(scratch);
    double(*inv)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(scratch + NB * (NB + 1));
    __shared__ int fail;
    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    const int64_t o = (int64_t)kb * NB;
    for (int e = tid; e < NB * NB; e += nth) {
        const int i = e / NB, j = e % NB;
        a[i][j] = (j <= i) ? (double)W[(o + i) * ld + o + j] : 0.0;
    }
    if (tid == 0) fail = -1;
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        const double d = a[j][j];
        // d is the same in every thread, so the exit is uniform.
        if (!(d > 0.0) || !isfinite(d)) {
            if (tid == 0) fail = isfinite(d) ? j : -2 - j;  // -2 - j encodes a NaN/Inf pivot
            break;
        }
        const double ljj = sqrt(d);
        __syncthreads();
        if (tid == 0) a[j][j] = ljj;
        for (int i = j + 1 + tid; i < NB; i += nth) a[i][j] /= ljj;
        __syncthreads();
        const int rem = NB - 1 - j;
        for (int e = tid; e < rem * rem; e += nth) {
            const int i = j + 1 + e / rem, p = j + 1 + e % rem;
            if (p <= i) a[i][p] = fma(-a[i][j], a[p][j], a[i][p]);
        }
        __syncthreads();
    }
    __syncthreads();
    if (fail != -1) {
        if (tid == 0) {
            const int j = fail >= 0 ? fail : -2 - fail;
            set_status(st, fail >= 0 ? DFS_ERR_NOT_SPD : DFS_ERR_NONFINITE);
            atomicCAS(&st->failed_pivot, -1, (int)(o + j));
        }
        return;
    }
    for (int e = tid; e < NB * NB; e += nth) {
        const int i = e / NB, j = e % NB;
        if (j <= i) W[(o + i) * ld + o + j] = (T)a[i][j];
    }
    invert_lower_block<T>(a, inv, Linv + (int64_t)kb * NB * NB);
}

template <typename T>
__global__ void __launch_bounds__(256) chol_first_kernel(T* W, int64_t ld, T* Linv, DevStatus* st) {
    __shared__ double scratch[2 * NB * (NB + 1)];
    if (st->status != 0) return;
    factor_diag_block<T>(W, ld, 0, Linv, st, scratch);
}

__device__ __forceinline__ void tri_ij(int t, int& I, int& J) {
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    I = i;
    J = t - i * (i + 1) / 2;
}

// Load a rows x NB panel block into smem and replace it by P = A Linv^T (rows beyond `rows`
// are zero).  Linv is lower triangular, so P[i][j] = sum_{p <= j} A[i][p] Linv[j][p].
template <typename T>
__device__ __forceinline__ void panel_times_linv_t(const T* W, int64_t ld, int64_t r0, int rows,
                                                   int64_t col0, const T (*sL)[NB + 1], T (*sA)[NB + 1]) {
    const int tid = threadIdx.x;
    for (int e = tid; e < TU * NB; e += blockDim.x) {
        const int i = e / NB, p = e % NB;
        sA[i][p] = (i < rows) ? W[(r0 + i) * ld + col0 + p] : (T)0;
    }
    __syncthreads();
    T out[TU * NB / 256];
#pragma unroll
    for (int u = 0; u < TU * NB / 256; ++u) {
        const int e = tid + u * 256;
        const int i = e / NB, j = e % NB;
        T s = 0;
        for (int p = 0; p <= j; ++p) s = fma(sA[i][p], sL[j][p], s);
        out[u] = s;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TU * NB / 256; ++u) {
        const int e = tid + u * 256;
        sA[e / NB][e % NB] = out[u];
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256)
chol_step_kernel(T* W, int64_t ld, int64_t n_pad, int kb, T* Linv, DevStatus* st) {
    constexpr int kPanelBytes = 2 * TU * (NB + 1) * (int)sizeof(T);
    constexpr int kFactorBytes = 2 * NB * (NB + 1) * (int)sizeof(double);
    __shared__ __align__(16) T sL[NB][NB + 1];
    // The two panel buffers and the FP64 factor scratch are never live at the same time.
    __shared__ __align__(16) unsigned char raw[kPanelBytes > kFactorBytes ? kPanelBytes : kFactorBytes];
    T(*sR)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(raw);
    T(*sQ)[NB + 1] = sR + TU;
    double* scratch = reinterpret_cast<double*>(raw);
    if (st->status != 0) return;
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)(kb + 1) * NB;
    const int64_t rem = n_pad - c0;
    int I, J;
    tri_ij(blockIdx.x, I, J);
    const int64_t r0 = c0 + (int64_t)I * TU, q0 = c0 + (int64_t)J * TU;
    const int rows_r = (int)min((int64_t)TU, rem - (int64_t)I * TU);
    const int rows_q = (int)min((int64_t)TU, rem - (int64_t)J * TU);
    const int64_t kc = (int64_t)kb * NB;

    const T* Lk = Linv + (int64_t)kb * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) sL[e / NB][e % NB] = Lk[e];
    __syncthreads();
    panel_times_linv_t<T>(W, ld, r0, rows_r, kc, sL, sR);
    if (I != J) panel_times_linv_t<T>(W, ld, q0, rows_q, kc, sL, sQ);
    const T(*pq)[NB + 1] = (I != J) ? sQ : sR;

    // C[i][j] -= sum_p P_r[i][p] P_q[j][p]; thread owns rows ty + 16 a, cols tx + 16 b.
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
#pragma unroll 8
    for (int p = 0; p < NB; ++p) {
        T ra[4], rb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) ra[a] = sR[ty + 16 * a][p];
#pragma unroll
        for (int b = 0; b < 4; ++b) rb[b] = pq[tx + 16 * b][p];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(ra[a], rb[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = ty + 16 * a;
        if (i >= rows_r) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = tx + 16 * b;
            if (j >= rows_q) continue;
            const int64_t gi = r0 + i, gj = q0 + j;
            if (gj > gi) continue;
            T* p = W + gi * ld + gj;
            *p = *p - acc[a][b];
        }
    }
    if (I == 0 && J == 0 && c0 < n_pad) {
        __threadfence_block();
        __syncthreads();  // all reads of sR/sQ are done before the factor scratch reuses them
        factor_diag_block<T>(W, ld, kb + 1, Linv, st, scratch);
    }
}

// Final panel scaling: L[i, kb] = A[i, kb] Linv_kb^T for all rows below diagonal block kb.
template <typename T>
__global__ void __launch_bounds__(256) chol_scale_kernel(T* W, int64_t ld, int64_t n_pad, T* Linv, DevStatus* st) {
    __shared__ __align__(16) T sL[NB][NB + 1];
    __shared__ __align__(16) T sA[TU][NB + 1];
    if (st->status != 0) return;
    const int kb = blockIdx.y;
    const int64_t c0 = (int64_t)(kb + 1) * NB;
    const int64_t r0 = c0 + (int64_t)blockIdx.x * TU;
    if (r0 >= n_pad) return;
    const int rows = (int)min((int64_t)TU, n_pad - r0);
    const T* Lk = Linv + (int64_t)kb * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) sL[e / NB][e % NB] = Lk[e];
    __syncthreads();
    panel_times_linv_t<T>(W, ld, r0, rows, (int64_t)kb * NB, sL, sA);
    for (int e = threadIdx.x; e < rows * NB; e += blockDim.x) {
        const int i = e / NB, p = e % NB;
        W[(r0 + i) * ld + (int64_t)kb * NB + p] = sA[i][p];
    }
}

// Inverses of all diagonal blocks of an existing factor L (for triangular solves with a
// caller-supplied L).  A zero or non-finite diagonal entry sets DFS_ERR_INVALID_ARG.
template <typename T>
__global__ void __launch_bounds__(256) diag_inverse_kernel(const T* L, int64_t ld, T* Linv, DevStatus* st) {
    __shared__ double a[NB][NB + 1];
    __shared__ double inv[NB][NB + 1];
    __shared__ int bad;
    const int kb = blockIdx.x;
    const int64_t o = (int64_t)kb * NB;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        const double v = (j <= i) ? (double)L[(o + i) * ld + o + j] : 0.0;
        a[i][j] = v;
        if (i == j && (!(v != 0.0) || !isfinite(v))) atomicExch(&bad, 1);
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) set_status(st, DFS_ERR_INVALID_ARG);
        return;
    }
    invert_lower_block<T>(a, inv, Linv + (int64_t)kb * NB * NB);
}

cudaError_t launch_diag_inverse(int w_f64, const void* L, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                                cudaStream_t stream) {
    const int nblk = (int)(n_pad / NB);
    if (w_f64)
        diag_inverse_kernel<double><<<nblk, 256, 0, stream>>>(static_cast<const double*>(L), ld,
                                                               static_cast<double*>(Linv), st);
    else
        diag_inverse_kernel<float><<<nblk, 256, 0, stream>>>(static_cast<const float*>(L), ld,
                                                              static_cast<float*>(Linv), st);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_cholesky_t(void* W_, int64_t ld, int64_t n_pad, void* Linv_, DevStatus* st,
                                     cudaStream_t stream) {
    T* W = static_cast<T*>(W_);
    T* Linv = static_cast<T*>(Linv_);
    const int nblk = (int)(n_pad / NB);
    chol_first_kernel<T><<<1, 256, 0, stream>>>(W, ld, Linv, st);
    for (int kb = 0; kb + 1 < nblk; ++kb) {
        const int64_t rem = n_pad - (int64_t)(kb + 1) * NB;
        const int Tn = (int)ceil_div(rem, TU);
        chol_step_kernel<T><<<Tn * (Tn + 1) / 2, 256, 0, stream>>>(W, ld, n_pad, kb, Linv, st);
    }
    if (nblk > 1) {
        dim3 grid((unsigned)ceil_div(n_pad, TU), nblk - 1);
        chol_scale_kernel<T><<<grid, 256, 0, stream>>>(W, ld, n_pad, Linv, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_cholesky(int w_f64, void* W, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                            cudaStream_t stream) {
    if (n_pad % NB != 0) return cudaErrorInvalidValue;
    return w_f64 ? launch_cholesky_t<double>(W, ld, n_pad, Linv, st, stream)
                 : launch_cholesky_t<float>(W, ld, n_pad, Linv, st, stream);
}

}  // namespace dfs
