// Algorithm 1's Gram on the SIMT pipes: W = S S^T (lower triangle), FP32 FFMA or FP64 DFMA.
//
// This is the plain-precision Gram of arXiv 2310.17556, Algorithm 1's Gram (the O(n^2 m)
// contraction that Section 2 names as the dominant cost).  S is n x m row-major, so both
// operands of S S^T are K-major (K = m contiguous).  The lower triangle is cut into BM x BM
// tiles (I >= J) and the contraction dimension m into `nsplit` chunks; each CTA computes one
// (tile, chunk) partial product and writes it to a partial buffer.  gram_finalize sums the
// chunks in a fixed order (deterministic), adds lambda to the diagonal and writes the padded
// n_pad x n_pad matrix used by the Cholesky step (rows/cols >= n get the identity).
#include "kernels.cuh"

namespace dfs {

__device__ __forceinline__ void lower_tile_ij(int t, int& I, int& J) {
    // t = I (I + 1) / 2 + J, 0 <= J <= I
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    I = i;
    J = t - i * (i + 1) / 2;
}

// Smem layout: operand tile transposed to [BK][BM] so that a thread reads its TM/2-element row
// groups as 16-byte vectors.  The row index is XOR-swizzled with a multiple of G = TM/2 that
// depends on k, which keeps the transposed 4-byte stores free of bank conflicts while every
// aligned G-group stays contiguous.
template <typename TS, typename TA, int BM, int BK, int TM>
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
gram_simt_kernel(const TS* __restrict__ S, int64_t n, int64_t m, int64_t lds, int64_t chunk,
                 int ntiles, TA* __restrict__ P) {
    constexpr int TD = BM / TM;
    constexpr int NT = TD * TD;
    constexpr int VEC = Vec16<TS>::N;
    constexpr int VPR = BK / VEC;
    constexpr int NV = BM * VPR / NT;
    constexpr int G = TM / 2;
    static_assert((BM * VPR) % NT == 0, "tile load must split evenly");
    static_assert(G * 8 <= BM / 2, "swizzle must stay inside a half tile");

    __shared__ __align__(16) TA As[BK][BM];
    __shared__ __align__(16) TA Bs[BK][BM];

    const int tid = threadIdx.x;
    const int tx = tid % TD, ty = tid / TD;
    int I, J;
    lower_tile_ij(blockIdx.x, I, J);
    const bool diag = (I == J);
    const int64_t rowA = (int64_t)I * BM, rowB = (int64_t)J * BM;
    const int64_t k0 = (int64_t)blockIdx.y * chunk;
    const int64_t k1 = min(m, k0 + chunk);
    const int64_t nk = (k1 > k0) ? ceil_div(k1 - k0, BK) : 0;

    TA acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = (TA)0;

    TA ra[NV][VEC], rb[NV][VEC];

    auto gload = [&](int64_t kt, TA (&r)[NV][VEC], int64_t row0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int idx = tid + v * NT;
            const int row = idx / VPR, cv = idx % VPR;
            const int64_t grow = row0 + row;
            const int64_t gk = kt + (int64_t)cv * VEC;
            if (grow < n && gk + VEC <= k1) {
                load16<TS, TA>(S + grow * lds + gk, r[v]);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    r[v][e] = (grow < n && gk + e < k1) ? load1<TS, TA>(S + grow * lds + gk + e) : (TA)0;
            }
        }
    };
    auto sstore = [&](TA (&r)[NV][VEC], TA (*sm)[BM]) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int idx = tid + v * NT;
            const int row = idx / VPR, cv = idx % VPR;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int kk = cv * VEC + e;
                const int sw = ((kk / VEC) & 7) * G;
                sm[kk][row ^ sw] = r[v][e];
            }
        }
    };

    if (nk > 0) {
        gload(k0, ra, rowA);
        if (!diag) gload(k0, rb, rowB);
    }
    for (int64_t it = 0; it < nk; ++it) {
        __syncthreads();
        sstore(ra, As);
        if (!diag) sstore(rb, Bs);
        __syncthreads();
        if (it + 1 < nk) {
            gload(k0 + (it + 1) * BK, ra, rowA);
            if (!diag) gload(k0 + (it + 1) * BK, rb, rowB);
        }
        const TA(*Bsrc)[BM] = diag ? As : Bs;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const int sw = ((kk / VEC) & 7) * G;
            TA a[TM], b[TM];
            const int ia0 = (ty * G) ^ sw, ia1 = (BM / 2 + ty * G) ^ sw;
            const int ib0 = (tx * G) ^ sw, ib1 = (BM / 2 + tx * G) ^ sw;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                a[g] = As[kk][ia0 + g];
                a[G + g] = As[kk][ia1 + g];
                b[g] = Bsrc[kk][ib0 + g];
                b[G + g] = Bsrc[kk][ib1 + g];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }

    TA* out = P + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (int64_t)(BM * BM);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = (i < G) ? (ty * G + i) : (BM / 2 + ty * G + (i - G));
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int c = (j < G) ? (tx * G + j) : (BM / 2 + tx * G + (j - G));
            out[r * BM + c] = acc[i][j];
        }
    }
}

// Sum the split-m partials in a fixed order (FP64), add lambda on the diagonal, and write the
// lower triangle of W.  Rows/cols in [n, n_out) get the identity (padding for the blocked
// Cholesky); upper-triangle entries are not written.
template <typename TA, typename TW, int BM>
__global__ void __launch_bounds__(256)
gram_finalize_kernel(const TA* __restrict__ P, int nsplit, int ntiles, int64_t n, int64_t n_out,
                     double lambda, TW* __restrict__ W, int64_t ldw) {
    int I, J;
    lower_tile_ij(blockIdx.x, I, J);
    const TA* base = P + (int64_t)blockIdx.x * (BM * BM);
    const int64_t tstride = (int64_t)ntiles * BM * BM;
    for (int e = threadIdx.x; e < BM * BM; e += blockDim.x) {
        const int r = e / BM, c = e % BM;
        const int64_t gi = (int64_t)I * BM + r, gj = (int64_t)J * BM + c;
        if (gi >= n_out || gj > gi) continue;
        double v;
        if (gi >= n || gj >= n) {
            v = (gi == gj) ? 1.0 : 0.0;
        } else {
            v = 0.0;
            for (int s = 0; s < nsplit; ++s) v += (double)base[s * tstride + e];
            if (gi == gj) v += lambda;
        }
        W[gi * ldw + gj] = (TW)v;
    }
}

// ---- host launchers ---------------------------------------------------------------------

template <typename TS, typename TA, int BM, int BK, int TM>
static cudaError_t launch_gram_simt_t(const void* S, int64_t n, int64_t m, int64_t lds,
                                      int nsplit, int64_t chunk, void* P, cudaStream_t stream) {
    const int T = (int)ceil_div(n, BM);
    const int ntiles = T * (T + 1) / 2;
    dim3 grid(ntiles, nsplit);
    {
        gram_simt_kernel<TS, TA, BM, BK, TM><<<grid, (BM / TM) * (BM / TM), 0, stream>>>(
            static_cast<const TS*>(S), n, m, lds, chunk, ntiles, static_cast<TA*>(P));
        count_launch();
    }
    return cudaGetLastError();
}

int gram_simt_tile(int acc_f64) { return acc_f64 ? 64 : 128; }

void gram_simt_plan(int64_t n, int64_t m, int acc_f64, int num_sms, int* nsplit, int64_t* chunk) {
    const int BM = gram_simt_tile(acc_f64);
    const int BK = acc_f64 ? 16 : 32;
    const int T = (int)ceil_div(n, BM);
    const int ntiles = T * (T + 1) / 2;
    // About two waves of 2 CTAs per SM; each chunk at least 16 k-steps.
    int64_t want = ceil_div(4LL * num_sms, ntiles);
    int64_t maxs = ceil_div(m, 16LL * BK);
    int64_t s = want < maxs ? want : maxs;
    if (s < 1) s = 1;
    if (s > 4096) s = 4096;
    int64_t c = round_up(ceil_div(m, s), BK);
    s = ceil_div(m, c);
    *nsplit = (int)s;
    *chunk = c;
}

size_t gram_simt_partial_bytes(int64_t n, int acc_f64, int nsplit) {
    const int BM = gram_simt_tile(acc_f64);
    const int64_t T = ceil_div(n, BM);
    return (size_t)nsplit * (size_t)(T * (T + 1) / 2) * BM * BM * (acc_f64 ? 8 : 4);
}

cudaError_t launch_gram_simt(int s_dtype, int acc_f64, const void* S, int64_t n, int64_t m,
                             int64_t lds, int nsplit, int64_t chunk, void* P, cudaStream_t stream) {
    if (acc_f64) {
        if (s_dtype == DFS_F64) return launch_gram_simt_t<double, double, 64, 16, 4>(S, n, m, lds, nsplit, chunk, P, stream);
        return cudaErrorInvalidValue;
    }
    if (s_dtype == DFS_F32) return launch_gram_simt_t<float, float, 128, 32, 8>(S, n, m, lds, nsplit, chunk, P, stream);
    if (s_dtype == DFS_BF16) return launch_gram_simt_t<__nv_bfloat16, float, 128, 32, 8>(S, n, m, lds, nsplit, chunk, P, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_gram_finalize(int acc_f64, int w_f64, int BM, const void* P, int nsplit,
                                 int64_t n, int64_t n_out, double lambda, void* W, int64_t ldw,
                                 cudaStream_t stream) {
    const int T = (int)ceil_div(n_out, BM);
    const int ntiles_out = T * (T + 1) / 2;
    const int Tn = (int)ceil_div(n, BM);
    const int ntiles = Tn * (Tn + 1) / 2;
    // Tiles beyond the computed ones (padding only) read no partials: n_out >= n, and a tile
    // index past ntiles only ever covers rows >= n, where the kernel writes the identity.
    if (acc_f64) {
        if (!w_f64 || BM != 64) return cudaErrorInvalidValue;
        {
            gram_finalize_kernel<double, double, 64><<<ntiles_out, 256, 0, stream>>>(
                static_cast<const double*>(P), nsplit, ntiles, n, n_out, lambda, static_cast<double*>(W), ldw);
            count_launch();
        }
    } else {
        if (BM != 128) return cudaErrorInvalidValue;
        if (w_f64)
            {
                gram_finalize_kernel<float, double, 128><<<ntiles_out, 256, 0, stream>>>(
                    static_cast<const float*>(P), nsplit, ntiles, n, n_out, lambda, static_cast<double*>(W), ldw);
                count_launch();
            }
        else
            {
                gram_finalize_kernel<float, float, 128><<<ntiles_out, 256, 0, stream>>>(
                    static_cast<const float*>(P), nsplit, ntiles, n, n_out, lambda, static_cast<float*>(W), ldw);
                count_launch();
            }
    }
    return cudaGetLastError();
}

}  // namespace dfs
