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

// Inverse of the lower-triangular NB x NB factor l (shared memory, compute type CT), in the
// storage precision T.  One warp per column c (columns c = warp, warp + 8, ...; needs 256
// threads), lane i holds x_i of L x = e_c: for p = c..NB-1, lane p finalises x_p = x_p / L_pp,
// broadcasts it, and lanes i > p subtract L_ip x_p.  Written to dst (NB x NB row-major, zeros
// above the diagonal).
template <typename T, typename CT>
__device__ void invert_lower_block(const CT (*l)[NB + 1], T* dst) {
    __shared__ T rd[NB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < NB) rd[tid] = (T)1 / (T)l[tid][tid];
    __syncthreads();
    for (int c = warp; c < NB; c += (int)(blockDim.x >> 5)) {
        T x = (lane == c) ? (T)1 : (T)0;
        for (int p = c; p < NB; ++p) {
            if (lane == p) x *= rd[p];
            const T xp = __shfl_sync(0xffffffffu, x, p);
            if (lane > p) x = fma(-(T)l[lane][p], xp, x);
        }
        dst[lane * NB + c] = (lane >= c) ? x : (T)0;
    }
    __syncthreads();
}

// 1/sqrt(d): FP32 hardware estimate, then (FP64) two Newton steps r <- r (3 - d r^2) / 2, each
// doubling the correct bits (~2^-22 -> 2^-44 -> below FP64 rounding).  A short dependent chain:
// the pivots of the diagonal factor are the critical path of the whole Cholesky.
__device__ __forceinline__ double rsqrt_ct(double d) {
    if (!(d > 1e-30 && d < 1e30)) return rsqrt(d);  // outside the FP32 estimate's safe range
    double r = (double)rsqrtf((float)d);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double h = 0.5 * d * r;
        r = fma(-h, r * r, 1.5 * r);  // r (1.5 - 0.5 d r^2)
    }
    return r;
}
__device__ __forceinline__ float rsqrt_ct(float d) { return rsqrtf(d); }

// Factor diagonal block kb in the compute type CT (double: the FP64 diagonal panel; float: the
// fast variant) and write L_kb (storage type T) plus its inverse.
// Column j: d = a[j][j]; r = 1/sqrt(d) (one thread); L[j][j] = d r, L[i][j] = a[i][j] r (one
// thread per row); then a[i][p] -= L[i][j] L[p][j] for j < p <= i (one FMA per element).  The
// elements of the trailing triangle are enumerated by a table sorted by column descending, so
// the trailing triangle of step j is exactly the first (31-j)(32-j)/2 table entries.
// Needs 256 threads and `scratch` >= 2 * NB * (NB + 1) CT values of shared memory.
template <typename T, typename CT>
__device__ void factor_diag_block(T* W, int64_t ld, int kb, T* Linv, DevStatus* st, CT* scratch) {
    CT(*a)[NB + 1] = reinterpret_cast<CT(*)[NB + 1]>(scratch);
    CT(*l)[NB + 1] = reinterpret_cast<CT(*)[NB + 1]>(scratch + NB * (NB + 1));
    __shared__ int fail;
    __shared__ CT rcol;
    __shared__ unsigned short tab[NB * (NB + 1) / 2];
    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    const int64_t o = (int64_t)kb * NB;
    for (int e = tid; e < NB * NB; e += nth) {
        const int i = e / NB, j = e % NB;
        a[i][j] = (j <= i) ? (CT)W[(o + i) * ld + o + j] : (CT)0;
        l[i][j] = (CT)0;
    }
    // tab[e] = (i << 8) | p over the lower triangle, p descending, i ascending within p
    for (int e = tid; e < NB * (NB + 1) / 2; e += nth) {
        int p = NB - 1, rem = e;
        while (rem >= NB - p) {
            rem -= NB - p;
            --p;
        }
        tab[e] = (unsigned short)(((p + rem) << 8) | p);
    }
    if (tid == 0) fail = -1;
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        if (tid == 0) {
            const CT d = a[j][j];
            if (!(d > (CT)0) || !isfinite(d)) {
                fail = isfinite(d) ? j : -2 - j;  // -2 - j encodes a NaN/Inf pivot
            } else {
                const CT r = rsqrt_ct(d);
                rcol = r;
                l[j][j] = d * r;
            }
        }
        __syncthreads();
        if (fail != -1) break;  // uniform: read after the barrier
        // column j of L and the rank-1 update, both from the unscaled column a[][j] and r (one
        // barrier per column): a[i][p] -= (a[i][j] r) (a[p][j] r)
        const CT r = rcol;
        if (tid > j && tid < NB) l[tid][j] = a[tid][j] * r;
        const int cnt = (NB - 1 - j) * (NB - j) / 2;
        for (int e = tid; e < cnt; e += nth) {
            const int ip = tab[e];
            const int i = ip >> 8, p = ip & 0xff;
            a[i][p] = fma(-(a[i][j] * r), a[p][j] * r, a[i][p]);
        }
        __syncthreads();
    }
    if (fail != -1) {
        if (tid == 0) {
            const int j = fail >= 0 ? fail : -2 - fail;
            set_status(st, fail >= 0 ? DFS_ERR_NOT_SPD : DFS_ERR_NONFINITE);
            atomicCAS(&st->failed_pivot, -1, (int)(o + j));
        }
        __syncthreads();
        return;
    }
    for (int e = tid; e < NB * NB; e += nth) {
        const int i = e / NB, j = e % NB;
        if (j <= i) W[(o + i) * ld + o + j] = (T)l[i][j];
    }
    invert_lower_block<T, CT>(l, Linv + (int64_t)kb * NB * NB);
}

template <typename T, typename CT>
__global__ void __launch_bounds__(256) chol_first_kernel(T* W, int64_t ld, T* Linv, DevStatus* st) {
    __shared__ CT scratch[2 * NB * (NB + 1)];
    if (block_should_exit(st, 0)) return;
    factor_diag_block<T, CT>(W, ld, 0, Linv, st, scratch);
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

template <typename T, typename CT>
__global__ void __launch_bounds__(256)
chol_step_kernel(T* W, int64_t ld, int64_t n_pad, int kb, T* Linv, DevStatus* st) {
    constexpr int kPanelBytes = 2 * TU * (NB + 1) * (int)sizeof(T);
    constexpr int kFactorBytes = 2 * NB * (NB + 1) * (int)sizeof(CT);
    __shared__ __align__(16) T sL[NB][NB + 1];
    // The two panel buffers and the FP64 factor scratch are never live at the same time.
    __shared__ __align__(16) unsigned char raw[kPanelBytes > kFactorBytes ? kPanelBytes : kFactorBytes];
    T(*sR)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(raw);
    T(*sQ)[NB + 1] = sR + TU;
    CT* scratch = reinterpret_cast<CT*>(raw);
    if (block_should_exit(st, 0)) return;
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
        factor_diag_block<T, CT>(W, ld, kb + 1, Linv, st, scratch);
    }
}

// Final panel scaling: L[i, kb] = A[i, kb] Linv_kb^T for all rows below diagonal block kb.
template <typename T>
__global__ void __launch_bounds__(256) chol_scale_kernel(T* W, int64_t ld, int64_t n_pad, T* Linv, DevStatus* st) {
    __shared__ __align__(16) T sL[NB][NB + 1];
    __shared__ __align__(16) T sA[TU][NB + 1];
    if (block_should_exit(st, 0)) return;
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
    invert_lower_block<T, double>(a, Linv + (int64_t)kb * NB * NB);
}

cudaError_t launch_diag_inverse(int w_f64, const void* L, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                                cudaStream_t stream) {
    const int nblk = (int)(n_pad / NB);
    if (w_f64)
        {
            diag_inverse_kernel<double><<<nblk, 256, 0, stream>>>(static_cast<const double*>(L), ld,
                                                                   static_cast<double*>(Linv), st);
            count_launch();
        }
    else
        {
            diag_inverse_kernel<float><<<nblk, 256, 0, stream>>>(static_cast<const float*>(L), ld,
                                                                  static_cast<float*>(Linv), st);
            count_launch();
        }
    return cudaGetLastError();
}

template <typename T, typename CT>
static cudaError_t launch_cholesky_t(void* W_, int64_t ld, int64_t n_pad, void* Linv_, DevStatus* st,
                                     cudaStream_t stream) {
    T* W = static_cast<T*>(W_);
    T* Linv = static_cast<T*>(Linv_);
    const int nblk = (int)(n_pad / NB);
    {
        chol_first_kernel<T, CT><<<1, 256, 0, stream>>>(W, ld, Linv, st);
        count_launch();
    }
    for (int kb = 0; kb + 1 < nblk; ++kb) {
        const int64_t rem = n_pad - (int64_t)(kb + 1) * NB;
        const int Tn = (int)ceil_div(rem, TU);
        {
            chol_step_kernel<T, CT><<<Tn * (Tn + 1) / 2, 256, 0, stream>>>(W, ld, n_pad, kb, Linv, st);
            count_launch();
        }
    }
    if (nblk > 1) {
        dim3 grid((unsigned)ceil_div(n_pad, TU), nblk - 1);
        {
            chol_scale_kernel<T><<<grid, 256, 0, stream>>>(W, ld, n_pad, Linv, st);
            count_launch();
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_cholesky(int w_f64, void* W, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                            cudaStream_t stream, int fp64_panel) {
    if (n_pad % NB != 0) return cudaErrorInvalidValue;
    if (w_f64) return launch_cholesky_t<double, double>(W, ld, n_pad, Linv, st, stream);
    return fp64_panel ? launch_cholesky_t<float, double>(W, ld, n_pad, Linv, st, stream)
                      : launch_cholesky_t<float, float>(W, ld, n_pad, Linv, st, stream);
}

}  // namespace dfs
