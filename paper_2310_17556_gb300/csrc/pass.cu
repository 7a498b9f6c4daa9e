// Streaming passes over S (HBM-bound), the inlined-Q part of Algorithm 1 (Section 2):
//
//   sv_pack_kernel       R = S V                 (b = S v, the rightmost product of
//                                                 S^T L^{-T} L^{-1} S v), optionally writing S
//                                                 again as packed tensor-core tiles (below)
//   fisher_pass_kernel   U = V - S^T Y           (S^T y, the leftmost product)
//                        X = U / lambda          (Algorithm 1's update of x)
//                        R = S U - lambda Y      (= S v - (S S^T + lambda I~) y, Appendix A's
//                                                 identity; the refinement residual)
//
// S is n x m row-major.  A CTA owns a column strip of W = LPR * VEC columns (LPR lanes of 16-byte
// loads per row) across all n rows; strips are dealt round-robin to a persistent grid.
//
// fisher_pass_kernel: 512 threads, 8 lanes per row (128-byte row segments), 64 rows per sweep.
// For n <= 64 * RPT each thread keeps its RPT row segments of the strip in registers between the
// two phases, so S crosses HBM and L2 exactly once (RPT = 0: phase 2 re-reads from L2).
//   phase 1  FP32 partials of S^T Y over rows -> shuffle over the row lanes -> shared memory ->
//            sum over the 16 warps -> U for the strip's columns (v and the previous x are loaded
//            before phase 1 so their latency is hidden); X written, sums of U^2 and of the x
//            change kept for the refinement's stopping rule;
//   phase 2  per-row dot products of the strip with U, reduced across the 8 lanes of the row,
//            added by one owner thread per row into an FP32 per-row sum that is folded into
//            FP64 every kFold strips.
// sv_pack_kernel: no cross-warp step at all (rows are owned by warps): per-row dot products of the
// strip with V as in phase 2.  With packing it also writes each 128-row x 128-byte block of S
// (one tensor-core k-block of a 128-row tile) as a contiguous 16 KB tile in the 128-byte-swizzled
// K-major layout the tcgen05 Gram consumes: BF16 (round to nearest even) or TF32 (FP32 rounded to
// nearest, ties away), or a plain re-layout of BF16 S.  Tiles of rows >= n and columns >= m
// are zero.  Tile (I, kb) sits at byte offset (kb * T + I) * 16384 (T = row tiles): the tiles of
// one k-block are contiguous, so the Gram's working set (a few k-blocks, all row tiles) is one
// contiguous region of L2.
// Each CTA finally writes its FP64 row sums (and the two per-RHS sums) to partial buffers that
// pass_reduce adds in a fixed order.
#include <cuda_fp8.h>

#define DFS_SRC_ID 2
#include "kernels.cuh"

namespace dfs {

constexpr int PASS_THREADS = 512;
constexpr int PASS_WARPS = PASS_THREADS / 32;
constexpr int kFold = 32;

template <typename TS>
struct PassTypes {
    using TA = float;  // accumulate / V / X type
};
template <>
struct PassTypes<double> {
    using TA = double;
};

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// H = bf16(x) and L = bf16(x - H) (both round to nearest even) of four consecutive floats, as
// two 8-byte groups of BF16 pairs; x - H is exact in FP32.
__device__ __forceinline__ void split_bf16x4(float x0, float x1, float x2, float x3, uint2& wh, uint2& wl) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(x0, x1), h23 = __floats2bfloat162_rn(x2, x3);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(x0 - f01.x, x1 - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(x2 - f23.x, x3 - f23.y);
    wh.x = *reinterpret_cast<const uint32_t*>(&h01);
    wh.y = *reinterpret_cast<const uint32_t*>(&h23);
    wl.x = *reinterpret_cast<const uint32_t*>(&l01);
    wl.y = *reinterpret_cast<const uint32_t*>(&l23);
}

// Four floats -> four e4m3 bytes (round to nearest even, saturating), lowest column first.
__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return (lo & 0xffffu) | (hi << 16);
}
// Byte offset, within a 128-row x 128-byte swizzled tile, of `bytes_per_lane` e4m3 values of row
// r that start at column `col` (a multiple of bytes_per_lane) of the tile's 128 columns.
__device__ __forceinline__ int fp8_tile_offset(int r, int col) {
    return r * 128 + ((((col >> 4) ^ (r & 7))) << 4) + (col & 15);
}

// Fold the FP32 per-row sums of the rows this thread owns into FP64.
template <typename TA, int KQ>
__device__ __forceinline__ void fold_rows(double* Rs64, TA* Rs32, int first, int step, int n) {
    for (int i = first; i < n; i += step)
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            Rs64[i * KQ + q] += (double)Rs32[i * KQ + q];
            Rs32[i * KQ + q] = (TA)0;
        }
}

// ------------------------------------------------------------------------------------------
// Per-row power-of-two scales of the FP8 Gram operand: r_i = 2^e, the smallest power of two with
// max_j |s_ij| <= 448 r_i (448 is the largest finite e4m3 value), so s_ij / r_i is exact and never
// saturates; r_i = 1 for a row of zeros and for the padding rows [n, n_pad); r_i = NaN for a row
// holding Inf or NaN, so the NaN reaches the Cholesky's check through the Gram.
// rs[0, n_pad) = r_i, rs[n_pad, 2 n_pad) = 1 / r_i.  One CTA of 256 threads per row.
template <typename TS>
__global__ void __launch_bounds__(256)
row_scale_kernel(const TS* __restrict__ S, int n, int n_pad, int64_t m, int64_t lds, float* __restrict__ rs,
                 const DevStatus* st) {
    constexpr int VEC = Vec16<TS>::N;
    __shared__ float s_max[8];
    __shared__ int s_bad[8];
    if (block_should_exit(st, 0)) return;
    const int i = blockIdx.x, tid = threadIdx.x;
    if (i >= n) {
        if (tid == 0) rs[i] = rs[n_pad + i] = 1.f;
        return;
    }
    const TS* row = S + (int64_t)i * lds;
    float amax = 0.f;
    int bad = 0;
    for (int64_t j = (int64_t)tid * VEC; j < m; j += 256 * VEC) {
        float v[VEC];
        if (j + VEC <= m) {
            load16_stream<TS, float>(row + j, v);
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) v[e] = (j + e < m) ? load1<TS, float>(row + j + e) : 0.f;
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const float a = fabsf(v[e]);
            bad |= !(a <= 3.4028235e38f);
            amax = fmaxf(amax, a);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((tid & 31) == 0) {
        s_max[tid >> 5] = amax;
        s_bad[tid >> 5] = bad;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < 8; ++w) {
            amax = fmaxf(amax, s_max[w]);
            bad |= s_bad[w];
        }
        float r = 1.f;
        if (bad) {
            r = __int_as_float(0x7fc00000);
        } else if (amax > 0.f) {
            int e;
            const float f = frexpf(amax / 448.f, &e);  // amax / 448 = f 2^e, f in [0.5, 1)
            if (f == 0.5f) --e;
            r = ldexpf(1.f, e < -126 ? -126 : e);
        }
        rs[i] = r;
        rs[n_pad + i] = 1.f / r;
    }
}

cudaError_t launch_row_scale(int s_dtype, const void* S, int n, int n_pad, int64_t m, int64_t lds, float* rs,
                             const DevStatus* st, cudaStream_t stream) {
    if (s_dtype == DFS_F32)
        row_scale_kernel<float><<<n_pad, 256, 0, stream>>>(static_cast<const float*>(S), n, n_pad, m, lds, rs, st);
    else if (s_dtype == DFS_BF16)
        row_scale_kernel<__nv_bfloat16>
            <<<n_pad, 256, 0, stream>>>(static_cast<const __nv_bfloat16*>(S), n, n_pad, m, lds, rs, st);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// R = S V, optionally packing S into tensor-core tiles.
//   PACK 0: none; 1: BF16 tiles (64-column k-blocks); 2: TF32 tiles (32-column k-blocks);
//   3 (FP32 S): BF16 H = bf16(s) in row block I and L = bf16(s - H) in row block n_rows / 128 + I,
//   2 n_rows / 128 tiles per k-block (the stacked operand of the BF16x3 Gram);
//   4: e4m3(s / r_i) with the row's power-of-two scale (rinv[i] = 1 / r_i), 128-column k-blocks:
//   a 64-column strip s fills half (s mod 2) of k-block s / 2, and the strip count is rounded up
//   to whole k-blocks so the tail half is written with zeros.
template <typename TS, int KQ, int PACK>
__global__ void __launch_bounds__(PASS_THREADS)
sv_pack_kernel(const TS* __restrict__ S, int n, int n_rows, int64_t m, int64_t lds,
               const typename PassTypes<TS>::TA* __restrict__ V, int64_t ldv, int k, double* __restrict__ Rpart,
               unsigned char* __restrict__ Sp, int64_t nkb, const DevStatus* st, const float* __restrict__ rinv) {
    using TA = typename PassTypes<TS>::TA;
    constexpr int VEC = Vec16<TS>::N;
    constexpr int LPR = ((PACK == 1 || PACK == 3 || PACK == 4) && sizeof(TS) == 4) ? 16 : 8;  // lanes per row
    static_assert(PACK != 4 || sizeof(TS) <= 4, "FP8 tiles from FP32 or BF16 S");
    static_assert(PACK != 3 || sizeof(TS) == 4, "the H / L split needs FP32 S");
    constexpr int W = LPR * VEC;
    constexpr int RPW = 32 / LPR;
    constexpr int SWEEP = PASS_WARPS * RPW;
    constexpr int RB = 8;
    extern __shared__ __align__(16) unsigned char smem[];
    double* Rs64 = reinterpret_cast<double*>(smem);
    TA* Rs32 = reinterpret_cast<TA*>(Rs64 + (size_t)n * KQ);
    if (block_should_exit(st, 0)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rr = lane / LPR, cq = lane % LPR;
    for (int e = tid; e < n * KQ; e += PASS_THREADS) {
        Rs64[e] = 0.0;
        Rs32[e] = (TA)0;
    }
    __syncthreads();
    const int64_t nstrips = PACK == 4 ? 2 * ceil_div(m, 2 * W) : ceil_div(m, W);
    int since_fold = 0;
    for (int64_t s = blockIdx.x; s < nstrips; s += gridDim.x) {
        const int64_t j0 = s * W;
        const int64_t jc = j0 + cq * VEC;
        const bool full = (j0 + W <= m);
        TA vv[KQ][VEC];
#pragma unroll
        for (int q = 0; q < KQ; ++q)
#pragma unroll
            for (int e = 0; e < VEC; ++e) vv[q][e] = (q < k && jc + e < m) ? V[(int64_t)q * ldv + jc + e] : (TA)0;
        // warp-uniform row loop (the row reductions below shuffle across lanes)
        for (int base = warp * RPW; base < n_rows; base += RB * SWEEP) {
            TA sv[RB][VEC];
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int i = base + u * SWEEP + rr;
                const TS* p = S + (int64_t)i * lds + jc;
                if (i < n && full) {
                    load16_stream<TS, TA>(p, sv[u]);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) sv[u][e] = (i < n && jc + e < m) ? load1<TS, TA>(p + e) : (TA)0;
                }
            }
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int i = base + u * SWEEP + rr;
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    TA a = 0;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) a = fma(sv[u][e], vv[q][e], a);
#pragma unroll
                    for (int o = 1; o < LPR; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                    if (cq == 0 && i < n) Rs32[i * KQ + q] += a;
                }
                if constexpr (PACK != 0) {
                    if (i < n_rows) {
                        const int r = i & 127;
                        constexpr int NTM = PACK == 3 ? 2 : 1;
                        unsigned char* tile = Sp + (((int64_t)s * (NTM * (n_rows >> 7)) + (i >> 7)) << 14) + r * 128;
                        if constexpr (PACK == 4) {
                            unsigned char* t8 = Sp + (((int64_t)(s >> 1) * (n_rows >> 7) + (i >> 7)) << 14);
                            const float q = i < n ? __ldg(rinv + i) : 0.f;
                            const int col = (int)(s & 1) * 64 + cq * VEC;
                            if constexpr (VEC == 4) {
                                *reinterpret_cast<uint32_t*>(t8 + fp8_tile_offset(r, col)) =
                                    e4m3x4(sv[u][0] * q, sv[u][1] * q, sv[u][2] * q, sv[u][3] * q);
                            } else {
                                uint2 w;
                                w.x = e4m3x4(sv[u][0] * q, sv[u][1] * q, sv[u][2] * q, sv[u][3] * q);
                                w.y = e4m3x4(sv[u][4] * q, sv[u][5] * q, sv[u][6] * q, sv[u][7] * q);
                                *reinterpret_cast<uint2*>(t8 + fp8_tile_offset(r, col)) = w;
                            }
                        } else if constexpr (PACK == 3) {
                            uint2 wh, wl;
                            split_bf16x4(sv[u][0], sv[u][1], sv[u][2], sv[u][3], wh, wl);
                            const int off = (((cq >> 1) ^ (r & 7)) << 4) | ((cq & 1) << 3);
                            *reinterpret_cast<uint2*>(tile + off) = wh;
                            *reinterpret_cast<uint2*>(tile + ((int64_t)(n_rows >> 7) << 14) + off) = wl;
                        } else if constexpr (PACK == 1 && sizeof(TS) == 4) {
                            // 4 floats -> 4 bf16 (8 bytes), half of 16-byte chunk cq / 2
                            if (!DFS_IN_BOUNDS(st, s < nkb)) continue;
                            const __nv_bfloat162 lo = __floats2bfloat162_rn(sv[u][0], sv[u][1]);
                            const __nv_bfloat162 hi = __floats2bfloat162_rn(sv[u][2], sv[u][3]);
                            uint2 w;
                            w.x = *reinterpret_cast<const uint32_t*>(&lo);
                            w.y = *reinterpret_cast<const uint32_t*>(&hi);
                            *reinterpret_cast<uint2*>(tile + ((((cq >> 1) ^ (r & 7)) << 4) | ((cq & 1) << 3))) = w;
                        } else if constexpr (PACK == 1) {
                            // BF16 S: the 16-byte chunk is copied as is
                            const TS* p = S + (int64_t)i * lds + jc;
                            uint4 w = make_uint4(0, 0, 0, 0);
                            if (i < n && full) {
                                w = __ldg(reinterpret_cast<const uint4*>(p));
                            } else if (i < n) {
                                uint32_t h[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    h[e] = (jc + e < m) ? (uint32_t)reinterpret_cast<const unsigned short*>(p)[e] : 0u;
                                w = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16),
                                               h[6] | (h[7] << 16));
                            }
                            *reinterpret_cast<uint4*>(tile + ((cq ^ (r & 7)) << 4)) = w;
                        } else {
                            uint4 w;
                            w.x = tf32_rna(sv[u][0]);
                            w.y = tf32_rna(sv[u][1]);
                            w.z = tf32_rna(sv[u][2]);
                            w.w = tf32_rna(sv[u][3]);
                            *reinterpret_cast<uint4*>(tile + ((cq ^ (r & 7)) << 4)) = w;
                        }
                    }
                }
            }
        }
        if (++since_fold == kFold) {
            since_fold = 0;
            if (cq == 0) fold_rows<TA, KQ>(Rs64, Rs32, warp * RPW + rr, SWEEP, n);
        }
    }
    if (cq == 0) fold_rows<TA, KQ>(Rs64, Rs32, warp * RPW + rr, SWEEP, n);
    __syncthreads();
    double* dst = Rpart + (int64_t)blockIdx.x * n * KQ;
    for (int e = tid; e < n * KQ; e += PASS_THREADS) dst[e] = Rs64[e];
}

// ------------------------------------------------------------------------------------------
// R = S V by blocks of R rows (8; 4 with 8 RHS), optionally packing S into BF16 tiles (PACK 1), for
// S whose rows are far apart (FP32 S with more than 1024 rows, BF16 S).  The CTA's 512 threads
// share its rows: at each step thread t takes the 8-column group base + t of every row, so a CTA
// streams each of its rows as one contiguous front of 4096 columns, and the grid keeps about
// R * num_sms rows open at once.  (One CTA per column strip opens every row of S at once, one per
// 128 rows 128 * num_sms rows; rows megabytes apart each sit in pages of their own, and that many
// open pages hold those forms to address-translation speed, well below HBM bandwidth.)  A
// thread's V values serve all R rows.  Sums in FP32 per thread, folded every 32 steps into FP64
// per warp (fixed shuffle order), the warps then added in order; part c of Rpart holds column
// chunk c's sums of every row, times scale (lambda when V is the pass's X = U / lambda).
constexpr int SVB_THREADS = 512;
constexpr int SVB_WARPS = SVB_THREADS / 32;
constexpr int SVB_FOLD = 32;

template <int KQ>
struct SvbRows {
    static constexpr int R = KQ >= 8 ? 4 : 8;
};

// 8 consecutive elements of S as raw 16-byte vectors (two for FP32, one for BF16), and back
template <typename TS>
__device__ __forceinline__ void svb_pack_raw(const float* f, uint4* raw);
template <>
__device__ __forceinline__ void svb_pack_raw<float>(const float* f, uint4* raw) {
    raw[0] = make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]), __float_as_uint(f[3]));
    raw[1] = make_uint4(__float_as_uint(f[4]), __float_as_uint(f[5]), __float_as_uint(f[6]), __float_as_uint(f[7]));
}
__device__ __forceinline__ uint32_t svb_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <>
__device__ __forceinline__ void svb_pack_raw<__nv_bfloat16>(const float* f, uint4* raw) {
    // f holds BF16 values: the conversion is exact
    raw[0] = make_uint4(svb_bf16x2(f[0], f[1]), svb_bf16x2(f[2], f[3]), svb_bf16x2(f[4], f[5]), svb_bf16x2(f[6], f[7]));
}
template <typename TS>
__device__ __forceinline__ void svb_unpack_raw(const uint4* raw, float* f);
template <>
__device__ __forceinline__ void svb_unpack_raw<float>(const uint4* raw, float* f) {
    f[0] = __uint_as_float(raw[0].x), f[1] = __uint_as_float(raw[0].y);
    f[2] = __uint_as_float(raw[0].z), f[3] = __uint_as_float(raw[0].w);
    f[4] = __uint_as_float(raw[1].x), f[5] = __uint_as_float(raw[1].y);
    f[6] = __uint_as_float(raw[1].z), f[7] = __uint_as_float(raw[1].w);
}
template <>
__device__ __forceinline__ void svb_unpack_raw<__nv_bfloat16>(const uint4* raw, float* f) {
    const uint32_t w[4] = {raw[0].x, raw[0].y, raw[0].z, raw[0].w};
#pragma unroll
    for (int e = 0; e < 4; ++e) f[2 * e] = __uint_as_float(w[e] << 16), f[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
}
// the BF16 tile chunk of the 8 elements: S's own bits for BF16 S, round-to-nearest for FP32 S
template <typename TS>
__device__ __forceinline__ uint4 svb_bf16_chunk(const uint4* raw);
template <>
__device__ __forceinline__ uint4 svb_bf16_chunk<__nv_bfloat16>(const uint4* raw) {
    return raw[0];
}
template <>
__device__ __forceinline__ uint4 svb_bf16_chunk<float>(const uint4* raw) {
    float f[8];
    svb_unpack_raw<float>(raw, f);
    return make_uint4(svb_bf16x2(f[0], f[1]), svb_bf16x2(f[2], f[3]), svb_bf16x2(f[4], f[5]), svb_bf16x2(f[6], f[7]));
}

template <typename TS, int KQ, int PACK>
__global__ void __launch_bounds__(SVB_THREADS, 1)
sv_rows_kernel(const TS* __restrict__ S, int n, int n_rows, int64_t m, int64_t lds, const float* __restrict__ V,
               int64_t ldv, int k, double* __restrict__ Rpart, unsigned char* __restrict__ Sp, int nchunks,
               const DevStatus* st, double scale, int honor_stop, const float* __restrict__ rinv) {
    constexpr int R = SvbRows<KQ>::R;
    constexpr int VEC = Vec16<TS>::N;  // elements per 16-byte load: 4 (FP32) or 8 (BF16)
    constexpr int LPG = 8 / VEC;       // 16-byte loads per row and 8-column group
    // steps in flight: 2 for BF16 S with one RHS (256 bytes per thread, as FP32 S keeps with one step);
    // more RHS leave no registers for it
    constexpr int U = (LPG == 1 && KQ == 1) ? 2 : 1;
    __shared__ double s_acc[SVB_WARPS][R * KQ];
    if (block_should_exit(st, honor_stop)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nrb = n_rows / R;
    const int rb = blockIdx.x % nrb, chunk = blockIdx.x / nrb;
    const int i0 = rb * R;
    // 64-column units of the columns the tiles cover (FP8 tiles: 128 columns, two units, so that
    // every tile column is written, zeros past m)
    const int64_t nkb_all = PACK == 4 ? 2 * ceil_div(m, 128) : ceil_div(m, 64);
    const int64_t per = ceil_div(nkb_all, nchunks);
    const int64_t g0 = (int64_t)chunk * per * 8;  // this CTA's 8-column groups [g0, g1)
    const int64_t g1 = g0 + per * 8 < nkb_all * 8 ? g0 + per * 8 : nkb_all * 8;
    // V's rows need not be 16-byte aligned (ldv is any value >= m): vector loads only when they are
    const bool v_vec = ((reinterpret_cast<uintptr_t>(V) | (uintptr_t)(ldv * 4)) & 15) == 0;
    for (int e = tid; e < SVB_WARPS * R * KQ; e += SVB_THREADS) (&s_acc[0][0])[e] = 0.0;
    __syncthreads();
    float acc[R][KQ];
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[j][q] = 0.f;
    // FP32 row sums -> the warp's FP64 sums: each (row, RHS) value is added over the warp's lanes
    // in FP32 (a butterfly: every lane ends with the total), then lane j KQ + q adds value (j, q)
    // to FP64, so that a fold costs each warp two FP64 instructions (on GB300 an FP64 warp
    // instruction occupies its sub-partition's FP64 unit for about 64 cycles, whatever the lanes).
    static_assert(R * KQ <= 32, "one lane per (row, RHS) value");
    auto fold = [&]() {
        float mine = 0.f;
#pragma unroll
        for (int j = 0; j < R; ++j)
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                if (q >= k) break;
                float a = acc[j][q];
                acc[j][q] = 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == j * KQ + q) mine = a;
            }
        if (lane < R * KQ) s_acc[warp][lane] += (double)mine;
    };
    int since = 0;
    for (int64_t base = g0; base < g1; base += (int64_t)U * SVB_THREADS) {
        // all loads of the step first (raw 16-byte vectors: R * U * LPG in flight per thread)
        uint4 raw[U][R][LPG];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = base + u * SVB_THREADS + tid;
            const bool gin = g < g1;
            const int64_t col = g * 8;
            const bool full = gin && col + 8 <= m;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const bool rin = i0 + j < n;
                const TS* p = S + (int64_t)(rin ? i0 + j : 0) * lds + (gin ? col : 0);
                if (rin && full) {
#pragma unroll
                    for (int l = 0; l < LPG; ++l) raw[u][j][l] = __ldcs(reinterpret_cast<const uint4*>(p + l * VEC));
                } else {
                    float f[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) f[e] = (rin && gin && col + e < m) ? load1<TS, float>(p + e) : 0.f;
                    svb_pack_raw<TS>(f, raw[u][j]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = base + u * SVB_THREADS + tid;
            const bool gin = g < g1;
            const int64_t col = g * 8;
            const bool full = gin && col + 8 <= m;
            // V's 8 values per RHS; BF16 S with up to 4 RHS (small raw vectors) holds all of them and
            // unpacks each row once, otherwise one RHS at a time
            constexpr bool ROW_OUTER = LPG == 1 && KQ <= 4;
            constexpr int WQ = ROW_OUTER ? KQ : 1;
            float w[WQ][8];
            auto load_w = [&](int q, float* wq) {
                const float* vq = V + (int64_t)q * ldv + (gin ? col : 0);
                if (v_vec && full) {
                    const float4 w0 = __ldg(reinterpret_cast<const float4*>(vq));
                    const float4 w1 = __ldg(reinterpret_cast<const float4*>(vq + 4));
                    wq[0] = w0.x, wq[1] = w0.y, wq[2] = w0.z, wq[3] = w0.w;
                    wq[4] = w1.x, wq[5] = w1.y, wq[6] = w1.z, wq[7] = w1.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) wq[e] = (gin && col + e < m) ? __ldg(vq + e) : 0.f;
                }
            };
            if constexpr (ROW_OUTER) {
#pragma unroll
                for (int q = 0; q < KQ; ++q)
                    if (q < k) load_w(q, w[q]);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    float sv[8];
                    svb_unpack_raw<TS>(raw[u][j], sv);
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        if (q >= k) break;
                        float a = acc[j][q];
#pragma unroll
                        for (int e = 0; e < 8; ++e) a = fmaf(sv[e], w[q][e], a);
                        acc[j][q] = a;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    if (q >= k) break;
                    load_w(q, w[0]);
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float sv[8];
                        svb_unpack_raw<TS>(raw[u][j], sv);
                        float a = acc[j][q];
#pragma unroll
                        for (int e = 0; e < 8; ++e) a = fmaf(sv[e], w[0][e], a);
                        acc[j][q] = a;
                    }
                }
            }
            if constexpr (PACK == 4) {
                if (gin) {
                    // 8 e4m3 bytes (row i scaled by rinv[i], round to nearest even, saturating) at
                    // columns (g & 15) * 8 of FP8 k-block g >> 4, in tile row i & 127
                    const int nblk = n_rows >> 7, col = (int)(g & 15) * 8;
                    unsigned char* tk = Sp + (((g >> 4) * (int64_t)nblk) << 14);
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const int i = i0 + j;
                        const float q = i < n ? __ldg(rinv + i) : 0.f;
                        float f[8];
                        svb_unpack_raw<TS>(raw[u][j], f);
                        uint2 w8;
                        w8.x = e4m3x4(f[0] * q, f[1] * q, f[2] * q, f[3] * q);
                        w8.y = e4m3x4(f[4] * q, f[5] * q, f[6] * q, f[7] * q);
                        *reinterpret_cast<uint2*>(tk + ((int64_t)(i >> 7) << 14) + fp8_tile_offset(i & 127, col)) = w8;
                    }
                }
            }
            if constexpr (PACK == 1) {
                if (gin) {
                    // 16-byte chunk c = g & 7 of k-block g >> 3 in tile row i & 127 (128-byte swizzle)
                    const int nblk = n_rows >> 7, c = (int)(g & 7);
                    unsigned char* tk = Sp + (((g >> 3) * (int64_t)nblk) << 14);
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const int i = i0 + j, r = i & 127;
                        *reinterpret_cast<uint4*>(tk + ((int64_t)(i >> 7) << 14) + r * 128 + ((c ^ (r & 7)) << 4)) =
                            svb_bf16_chunk<TS>(raw[u][j]);
                    }
                }
            }
        }
        if (++since == SVB_FOLD / U) {
            since = 0;
            fold();
        }
    }
    fold();
    __syncthreads();
    for (int t = tid; t < R * KQ; t += SVB_THREADS) {
        const int i = i0 + t / KQ;
        double a = 0.0;
        for (int w = 0; w < SVB_WARPS; ++w) a += s_acc[w][t];
        if (i < n) Rpart[((int64_t)chunk * n + i) * KQ + t % KQ] = scale * a;
    }
}

// column chunks of sv_rows_kernel (at most num_sms: the partial rows of R).  One 512-thread CTA
// fills an SM's registers, so the nrb * c equal CTAs run in waves of num_sms: take the smallest
// c >= num_sms / nrb whose last wave is at least 95 % full (the fullest found otherwise).
static int sv_rows_chunks(int nrb, int64_t m, int num_sms) {
    const int64_t nkb = ceil_div(m, 64);
    int64_t cmax = num_sms < nkb ? num_sms : nkb;
    if (cmax < 1) cmax = 1;
    int64_t c0 = ceil_div((int64_t)num_sms, (int64_t)nrb);
    if (c0 > cmax) c0 = cmax;
    int best = (int)c0;
    double best_eff = 0.0;
    for (int64_t c = c0; c <= cmax; ++c) {
        const int64_t ctas = (int64_t)nrb * c, waves = ceil_div(ctas, (int64_t)num_sms);
        const double eff = (double)ctas / (double)(waves * num_sms);
        if (eff > best_eff + 1e-9) best_eff = eff, best = (int)c;
        if (eff >= 0.95) break;
    }
    return best;
}

template <typename TS, int KQ, int PACK>
static cudaError_t launch_sv_rows_t(int nchunks, const void* S, int n, int n_rows, int64_t m, int64_t lds,
                                    const void* V, int64_t ldv, int k, double* Rpart, void* Sp, const DevStatus* st,
                                    cudaStream_t stream, double scale = 1.0, int honor_stop = 0,
                                    const float* rinv = nullptr) {
    const int64_t grid = (int64_t)nchunks * (n_rows / SvbRows<KQ>::R);
    sv_rows_kernel<TS, KQ, PACK><<<(unsigned)grid, SVB_THREADS, 0, stream>>>(
        static_cast<const TS*>(S), n, n_rows, m, lds, static_cast<const float*>(V), ldv, k, Rpart,
        static_cast<unsigned char*>(Sp), nchunks, st, scale, honor_stop, rinv);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// X = (V - S^T Y) / lambda for S whose rows are far apart (n > 2048): the first kernel of the
// refinement pass as two (the second, R = S U - lambda Y, is sv_rows_kernel on X with scale
// lambda).  fisher_pass_kernel's strips span all n rows at once; here a CTA takes 4096-column
// chunks (round-robin over a one-CTA-per-SM grid) down all n rows, its 512 threads sharing each
// row, so the grid keeps about RB rows per SM open.  Thread t holds 8 columns of the chunk: 8
// contiguous BF16, or two runs of 4 FP32 128 columns apart, so that every warp load is 512
// contiguous bytes.  Column sums in FP32 over panels of 256 rows, the panels added in FP64 in
// shared memory (a thread owns its columns outright: no cross-thread step; its registers keep 256
// bytes of S in flight); then, as fisher_pass_kernel, U = V - S^T Y, X = U / lambda and the sums
// of U^2 and of the change of X (dmode).
constexpr int STY_COLS = SVB_THREADS * 8;

template <typename TS, int KQ>
struct StyRows {  // rows in flight per thread: up to 256 bytes of S, as the KQ accumulators allow
    static constexpr int R = sizeof(TS) == 2 ? (KQ == 1 ? 16 : (KQ == 2 ? 10 : 12)) : (KQ <= 2 ? 8 : 6);
};
// dynamic shared memory of sty_cols_kernel: a thread's FP64 column sums (8 columns x KQ), then its
// FP64 sums of U^2 and dX^2 (KQ each)
constexpr size_t sty_smem_bytes(int KQ) { return (size_t)KQ * 10 * SVB_THREADS * sizeof(double); }

template <typename TS, int KQ>
__global__ void __launch_bounds__(SVB_THREADS, 1)
sty_cols_kernel(const TS* __restrict__ S, int n, int64_t m, int64_t lds, const float* __restrict__ V, int64_t ldv,
                int k, const double* __restrict__ Y, int64_t ldy, double lambda, float* __restrict__ X,
                int64_t ldx, double* __restrict__ U2part, int dmode, const DevStatus* st, int honor_stop) {
    constexpr int VEC = Vec16<TS>::N;  // 4 (FP32) or 8 (BF16)
    constexpr int LPG = 8 / VEC;       // 16-byte loads per row: 2 (FP32) or 1 (BF16)
    constexpr int RB = StyRows<TS, KQ>::R;
    constexpr int PANEL = 256;
    // y in FP32, YB rows at a time (a multiple of the rows of a step), converted once per CTA and
    // read from shared memory: converting it from FP64 in the row loop (KQ conversions a row and
    // thread) made the loop FP64-bound with several right-hand sides, as FP64 instructions are
    // slow on this GPU.  The values are the same FP32 roundings of y as before.
    constexpr int YB = RB * ((PANEL + RB - 1) / RB);
    __shared__ __align__(16) float ys[YB * KQ];
    extern __shared__ double tot[];  // [(q * 8 + e) * SVB_THREADS + tid]
    double* uds = tot + KQ * 8 * SVB_THREADS;  // [q * SVB_THREADS + tid]: U^2, then dX^2 at + KQ
    __shared__ double red[SVB_WARPS][16];
    if (block_should_exit(st, honor_stop)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float inv_lambda = (float)(1.0 / lambda);
    const int64_t nchunks = ceil_div(m, (int64_t)STY_COLS);
#pragma unroll
    for (int q = 0; q < 2 * KQ; ++q) uds[q * SVB_THREADS + tid] = 0.0;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        // column of element e: cb + (e / VEC) * (256 / LPG) + e % VEC
        const int64_t cb = c * STY_COLS + warp * 256 + lane * VEC;
#pragma unroll
        for (int qe = 0; qe < KQ * 8; ++qe) tot[qe * SVB_THREADS + tid] = 0.0;
        if (Y != nullptr) {
            float acc[KQ][8];
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < 8; ++e) acc[q][e] = 0.f;
            int rows = 0, yb0 = 0;
            for (int i0 = 0; i0 < n; i0 += RB) {
                if (i0 % YB == 0) {
                    __syncthreads();  // every thread is done with the previous block of y
                    yb0 = i0;
                    for (int e = tid; e < YB * KQ; e += SVB_THREADS) {
                        const int i = i0 + e / KQ, q = e % KQ;
                        ys[e] = (i < n && q < k) ? (float)Y[(int64_t)i * ldy + q] : 0.f;
                    }
                    __syncthreads();
                }
                uint4 raw[RB][LPG];
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    const int i = i0 + j;
                    const TS* row = S + (int64_t)(i < n ? i : 0) * lds;
#pragma unroll
                    for (int l = 0; l < LPG; ++l) {
                        const int64_t cl = cb + l * (256 / LPG);
                        if (i < n && cl + VEC <= m) {
                            raw[j][l] = __ldcs(reinterpret_cast<const uint4*>(row + cl));
                        } else {
                            float f[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) f[e] = 0.f;
#pragma unroll
                            for (int e = 0; e < VEC; ++e)
                                if (i < n && cl + e < m) f[e] = load1<TS, float>(row + cl + e);
                            uint4 two[2];
                            svb_pack_raw<TS>(f, two);
                            raw[j][l] = two[0];
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    float yv[KQ];
                    const float* yr = ys + (i0 - yb0 + j) * KQ;
                    if constexpr (KQ == 4) {
                        const float4 t = *reinterpret_cast<const float4*>(yr);
                        yv[0] = t.x, yv[1] = t.y, yv[2] = t.z, yv[3] = t.w;
                    } else if constexpr (KQ == 2) {
                        const float2 t = *reinterpret_cast<const float2*>(yr);
                        yv[0] = t.x, yv[1] = t.y;
                    } else {
#pragma unroll
                        for (int q = 0; q < KQ; ++q) yv[q] = yr[q];
                    }
                    float sv[8];
                    svb_unpack_raw<TS>(raw[j], sv);
#pragma unroll
                    for (int q = 0; q < KQ; ++q)
#pragma unroll
                        for (int e = 0; e < 8; ++e) acc[q][e] = fmaf(sv[e], yv[q], acc[q][e]);
                }
                if ((rows += RB) >= PANEL || i0 + RB >= n) {
                    rows = 0;
#pragma unroll
                    for (int q = 0; q < KQ; ++q)
#pragma unroll
                        for (int e = 0; e < 8; ++e) tot[(q * 8 + e) * SVB_THREADS + tid] += (double)acc[q][e], acc[q][e] = 0.f;
                }
            }
        }
        // U = V - S^T Y, X = U / lambda, and the stopping rule's sums
        float u2f[KQ], d2f[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) u2f[q] = d2f[q] = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t col = cb + (e / VEC) * (256 / LPG) + e % VEC;
            if (col >= m) continue;
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                if (q >= k) break;
                const float v = V[(int64_t)q * ldv + col];
                const float u = (float)((double)v - tot[(q * 8 + e) * SVB_THREADS + tid]);
                const float xn = u * inv_lambda;
                float dx = 0.f;
                if (dmode == 1) dx = xn - X[(int64_t)q * ldx + col];
                else if (dmode == 2) dx = (u - v) * inv_lambda;
                X[(int64_t)q * ldx + col] = xn;
                u2f[q] += u * u;
                d2f[q] += dx * dx;
            }
        }
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            uds[q * SVB_THREADS + tid] += (double)u2f[q];
            uds[(KQ + q) * SVB_THREADS + tid] += (double)d2f[q];
        }
    }
    // per-RHS sums over the CTA, in a fixed order (the U2part layout of fisher_pass_kernel)
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        double v = uds[q * SVB_THREADS + tid], w = uds[(KQ + q) * SVB_THREADS + tid];
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (lane == 0) red[warp][q] = v, red[warp][8 + q] = w;
    }
    __syncthreads();
    if (tid < KQ) {
        double v = 0.0, w = 0.0;
        for (int wp = 0; wp < SVB_WARPS; ++wp) v += red[wp][tid], w += red[wp][8 + tid];
        U2part[(int64_t)blockIdx.x * 2 * KQ + tid] = v;
        U2part[(int64_t)blockIdx.x * 2 * KQ + KQ + tid] = w;
    }
}

// ------------------------------------------------------------------------------------------
// R = S V for FP32 S with at most 1024 rows, optionally packing S into BF16 tiles (PACK 1): a
// streaming form of sv_pack_kernel.  A thread owns rows warp * 2 + rr + 32 t (t < 32) and 16 bytes
// of every 64-column strip; its row segments stream through a cp.async ring of 4-row sub-stages
// (6 slots, ~160 KB in flight per SM, each slot refilled by the thread that read it, so no
// barrier), the per-row partial dot products stay in registers across strips and are reduced over
// the 16 lanes of a row (shuffles) and folded into FP64 every 32 strips, and the next strip's V is
// prefetched.  Each 16-byte segment is converted (round to nearest even) and stored as 8 bytes of
// its swizzled BF16 tile row as it passes.
constexpr int SVR_TPS = 4;       // rows per thread and sub-stage
constexpr int SVR_SLOTS = 6;
constexpr int SVR_MAXNR = 32;    // rows per thread (n_rows <= 1024)

template <int KQ, int PACK>
__global__ void __launch_bounds__(PASS_THREADS, 1)
sv_ring_kernel(const float* __restrict__ S, int n, int n_rows, int64_t m, int64_t lds, const float* __restrict__ V,
               int64_t ldv, int k, double* __restrict__ Rpart, unsigned char* __restrict__ Sp, int64_t nkb,
               const DevStatus* st, const float* __restrict__ rinv) {
    constexpr int LPR = 16, W = 64, SWEEP = PASS_THREADS / LPR, NSUBMAX = SVR_MAXNR / SVR_TPS;
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* ring = reinterpret_cast<uint4*>(smem);
    double* Rs64 = reinterpret_cast<double*>(smem + (size_t)SVR_SLOTS * SVR_TPS * PASS_THREADS * 16);  // n x KQ
    if (block_should_exit(st, 0)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rr = lane / LPR, cq = lane % LPR;
    const int row0 = warp * 2 + rr;
    const int NR = (n_rows + SWEEP - 1) / SWEEP;
    const int nsub = (NR + SVR_TPS - 1) / SVR_TPS;
    for (int e = tid; e < n * KQ; e += PASS_THREADS) Rs64[e] = 0.0;
    const int64_t nstrips = PACK == 4 ? 2 * ceil_div(m, 2 * W) : ceil_div(m, W);  // FP8: whole k-blocks
    const int64_t my_strips = (int64_t)blockIdx.x < nstrips ? (nstrips - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nitems = my_strips * nsub;
    auto issue = [&](int64_t g) {
        if (g < nitems) {
            const int64_t s = blockIdx.x + (g / nsub) * gridDim.x;
            const int j = (int)(g % nsub);
            const int64_t jn = s * W + cq * 4;
            const int64_t rem = m - jn;
            const int bytes_col = rem >= 4 ? 16 : (rem > 0 ? (int)rem * 4 : 0);
            uint4* slot = ring + (size_t)(g % SVR_SLOTS) * SVR_TPS * PASS_THREADS;
#pragma unroll
            for (int tt = 0; tt < SVR_TPS; ++tt) {
                const int t = j * SVR_TPS + tt;
                const int i = row0 + t * SWEEP;
                const int bytes = (i < n && t < NR) ? bytes_col : 0;
                const float* src = bytes ? S + (int64_t)i * lds + jn : S;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                 static_cast<uint32_t>(__cvta_generic_to_shared(&slot[tt * PASS_THREADS + tid]))),
                             "l"(src), "r"(bytes)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto load_v = [&](int64_t s, float (&vv)[KQ][4]) {
        const int64_t jc = s * W + cq * 4;
#pragma unroll
        for (int q = 0; q < KQ; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) vv[q][e] = (s < nstrips && q < k && jc + e < m) ? V[(int64_t)q * ldv + jc + e] : 0.f;
    };
    float acc[KQ][SVR_MAXNR];
#pragma unroll
    for (int q = 0; q < KQ; ++q)
#pragma unroll
        for (int t = 0; t < SVR_MAXNR; ++t) acc[q][t] = 0.f;
    auto fold = [&]() {
#pragma unroll
        for (int t = 0; t < SVR_MAXNR; ++t) {
            const int i = row0 + t * SWEEP;
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                float a = acc[q][t];
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                a += __shfl_xor_sync(0xffffffffu, a, 4);
                a += __shfl_xor_sync(0xffffffffu, a, 8);
                if (cq == 0 && i < n) Rs64[i * KQ + q] += (double)a;
                acc[q][t] = 0.f;
            }
        }
    };
    for (int g = 0; g < SVR_SLOTS - 1; ++g) issue(g);
    float vv[KQ][4], vn[KQ][4];
    load_v(blockIdx.x, vn);
    __syncthreads();  // Rs64 zeroed
    int64_t g = 0;
    int since_fold = 0;
    for (int64_t ls = 0; ls < my_strips; ++ls) {
        const int64_t s = blockIdx.x + ls * gridDim.x;
#pragma unroll
        for (int q = 0; q < KQ; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) vv[q][e] = vn[q][e];
        load_v(s + gridDim.x, vn);
#pragma unroll
        for (int j = 0; j < NSUBMAX; ++j) {
            if (j < nsub) {
                asm volatile("cp.async.wait_group %0;" ::"n"(SVR_SLOTS - 2) : "memory");
                const uint4* slot = ring + (size_t)(g % SVR_SLOTS) * SVR_TPS * PASS_THREADS;
#pragma unroll
                for (int tt = 0; tt < SVR_TPS; ++tt) {
                    const int t = j * SVR_TPS + tt;
                    const uint4 w = slot[tt * PASS_THREADS + tid];
                    const float x0 = __uint_as_float(w.x), x1 = __uint_as_float(w.y), x2 = __uint_as_float(w.z),
                                x3 = __uint_as_float(w.w);
#pragma unroll
                    for (int q = 0; q < KQ; ++q)
                        acc[q][t] = fmaf(x3, vv[q][3], fmaf(x2, vv[q][2], fmaf(x1, vv[q][1], fmaf(x0, vv[q][0], acc[q][t]))));
                    if constexpr (PACK == 4) {
                        const int i = row0 + t * SWEEP;
                        if (i < n_rows) {
                            unsigned char* t8 = Sp + (((int64_t)(s >> 1) * (n_rows >> 7) + (i >> 7)) << 14);
                            const float q = i < n ? __ldg(rinv + i) : 0.f;
                            *reinterpret_cast<uint32_t*>(t8 + fp8_tile_offset(i & 127, (int)(s & 1) * 64 + cq * 4)) =
                                e4m3x4(x0 * q, x1 * q, x2 * q, x3 * q);
                        }
                    } else if constexpr (PACK == 3) {
                        const int i = row0 + t * SWEEP;
                        if (i < n_rows) {
                            const int r = i & 127;
                            unsigned char* tile = Sp + (((int64_t)s * (2 * (n_rows >> 7)) + (i >> 7)) << 14) + r * 128;
                            uint2 wh, wl;
                            split_bf16x4(x0, x1, x2, x3, wh, wl);
                            const int off = (((cq >> 1) ^ (r & 7)) << 4) | ((cq & 1) << 3);
                            *reinterpret_cast<uint2*>(tile + off) = wh;
                            *reinterpret_cast<uint2*>(tile + ((int64_t)(n_rows >> 7) << 14) + off) = wl;
                        }
                    } else if constexpr (PACK == 1) {
                        const int i = row0 + t * SWEEP;
                        if (i < n_rows && DFS_IN_BOUNDS(st, s < nkb)) {
                            const int r = i & 127;
                            unsigned char* tile = Sp + (((int64_t)s * (n_rows >> 7) + (i >> 7)) << 14) + r * 128;
                            const __nv_bfloat162 lo = __floats2bfloat162_rn(x0, x1);
                            const __nv_bfloat162 hi = __floats2bfloat162_rn(x2, x3);
                            uint2 o;
                            o.x = *reinterpret_cast<const uint32_t*>(&lo);
                            o.y = *reinterpret_cast<const uint32_t*>(&hi);
                            *reinterpret_cast<uint2*>(tile + ((((cq >> 1) ^ (r & 7)) << 4) | ((cq & 1) << 3))) = o;
                        }
                    }
                }
                issue(g + SVR_SLOTS - 1);
                ++g;
            }
        }
        if (++since_fold == kFold) {
            since_fold = 0;
            fold();
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    fold();
    __syncthreads();
    double* dst = Rpart + (int64_t)blockIdx.x * n * KQ;
    for (int e = tid; e < n * KQ; e += PASS_THREADS) dst[e] = Rs64[e];
}

// ------------------------------------------------------------------------------------------
// The refinement's last correction read from the packed BF16 tiles instead of S:
//   x <- x - S_bf16^T dy / lambda
// (n_rows x 64-column tiles, 128-byte swizzled rows, k-block major as written by the S v pass),
// and per CTA the sums of the passes' stopping statistics: lambda^2 ||x_new||^2 and
// ||x_new - x_old||^2 per RHS (U2part, 2 KQ doubles per CTA).  Each warp owns whole k-blocks (64
// columns): lane (chunk c = lane % 8, row group lane / 8) reads the 16-byte logical chunk c (8
// columns) of rows lane / 8, + 4, + 8, ... (the four rows of a step are whole 128-byte lines), 8
// steps in flight (16 with 4 right-hand sides); with 8 right-hand sides 16 lanes of 8 bytes cover a
// row, a warp has two row groups and 32 steps in flight.  dy sits in shared memory, each value twice, so that one 16-byte load gives the
// operands of two right-hand sides' paired multiply-adds (each lane of a pair an IEEE fmaf, as in
// scalar code); the row groups are added with shuffles and the lanes of row group 0 update their
// columns of x in place.
constexpr int TC_CORR_THREADS = 512;
constexpr int TC_CORR_ROWS = 64;  // n_rows is a multiple of the rows a warp has in flight

template <int KQ>
__global__ void __launch_bounds__(TC_CORR_THREADS)
tile_correct_kernel(const unsigned char* __restrict__ Sp, int n, int n_rows, int64_t m, int64_t nkb,
                    const float* __restrict__ Z, int k, double lambda, float* __restrict__ X, int64_t ldx,
                    double* __restrict__ U2part, const DevStatus* st) {
    // columns per lane: 8 (a 16-byte chunk), or 4 (half a chunk) with 8 right-hand sides, whose
    // accumulators would not fit otherwise
    constexpr int CPL = KQ >= 8 ? 4 : 8;
    constexpr int LPRC = 64 / CPL;  // lanes per row
    constexpr int RG = 32 / LPRC;   // row groups of a warp
    // rows in flight per thread: 128 bytes, or 256 with 4 or more right-hand sides, whose
    // accumulators leave room for one CTA per SM only (the bytes in flight then come from the rows)
    constexpr int UNROLL = CPL == 4 ? 32 : (KQ >= 4 ? 16 : 8);
    static_assert(RG * UNROLL <= TC_CORR_ROWS && TC_CORR_ROWS % (RG * UNROLL) == 0, "row step");
    // dy twice per entry, [row][q][2]: the pair operand of the paired multiply-adds
    extern __shared__ float sdy[];  // n_rows x KQ x 2
    __shared__ double red[TC_CORR_THREADS / 32][2 * KQ];
    if (block_should_exit(st, 1)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < n_rows * KQ; e += TC_CORR_THREADS) {
        const float d = (e / KQ < n && e % KQ < k) ? Z[e] : 0.f;
        sdy[2 * e] = d;
        sdy[2 * e + 1] = d;
    }
    const int wpb = TC_CORR_THREADS / 32;
    // the warp's sums of ||x_new||^2 and ||x_new - x_old||^2 per RHS (added by its lane 0)
    for (int e = tid; e < wpb * 2 * KQ; e += TC_CORR_THREADS) red[e / (2 * KQ)][e % (2 * KQ)] = 0.0;
    __syncthreads();
    const int c = lane % LPRC, rg = lane / LPRC;
    const int T = n_rows >> 7;
    const float inv_l = (float)(1.0 / lambda);
    for (int64_t kb = (int64_t)blockIdx.x * wpb + warp; kb < nkb; kb += (int64_t)gridDim.x * wpb) {
        const unsigned char* base = Sp + ((kb * T) << 14);
        float2 acc[KQ][CPL / 2];  // the lane's columns in pairs (0, 1), (2, 3), ...
#pragma unroll
        for (int q = 0; q < KQ; ++q)
#pragma unroll
            for (int e = 0; e < CPL / 2; ++e) acc[q][e] = make_float2(0.f, 0.f);
        for (int r0 = 0; r0 < n_rows; r0 += RG * UNROLL) {
            uint32_t w[UNROLL][CPL / 2];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int r = r0 + RG * u + rg;
                const unsigned char* row = base + ((r >> 7) << 14) + (r & 127) * 128;
                if (!DFS_IN_BOUNDS(st, r < n_rows && kb < nkb)) {
#pragma unroll
                    for (int e = 0; e < CPL / 2; ++e) w[u][e] = 0u;
                    continue;
                }
                if constexpr (CPL == 8) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + ((c ^ (r & 7)) << 4)));
                    w[u][0] = v.x, w[u][1] = v.y, w[u][2] = v.z, w[u][3] = v.w;
                } else {
                    const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + ((((c >> 1) ^ (r & 7)) << 4) | ((c & 1) << 3))));
                    w[u][0] = v.x, w[u][1] = v.y;
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int r = r0 + RG * u + rg;
                float2 f[CPL / 2];  // the BF16 pair of word e, widened exactly
#pragma unroll
                for (int e = 0; e < CPL / 2; ++e)
                    f[e] = make_float2(__uint_as_float(w[u][e] << 16), __uint_as_float(w[u][e] & 0xffff0000u));
                if constexpr (KQ >= 2) {
#pragma unroll
                    for (int q = 0; q < KQ; q += 2) {
                        const float4 d4 = *reinterpret_cast<const float4*>(&sdy[(r * KQ + q) * 2]);
                        const float2 da = make_float2(d4.x, d4.y), db = make_float2(d4.z, d4.w);
#pragma unroll
                        for (int e = 0; e < CPL / 2; ++e) {
                            acc[q][e] = __ffma2_rn(f[e], da, acc[q][e]);
                            acc[q + 1][e] = __ffma2_rn(f[e], db, acc[q + 1][e]);
                        }
                    }
                } else {
                    const float2 da = *reinterpret_cast<const float2*>(&sdy[r * 2]);
#pragma unroll
                    for (int e = 0; e < CPL / 2; ++e) acc[0][e] = __ffma2_rn(f[e], da, acc[0][e]);
                }
            }
        }
        // the row groups, in a fixed order
#pragma unroll
        for (int q = 0; q < KQ; ++q)
#pragma unroll
            for (int e = 0; e < CPL / 2; ++e)
#pragma unroll
                for (int o = LPRC; o < 32; o <<= 1) {
                    acc[q][e].x += __shfl_xor_sync(0xffffffffu, acc[q][e].x, o);
                    acc[q][e].y += __shfl_xor_sync(0xffffffffu, acc[q][e].y, o);
                }
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            if (q >= k) continue;
            float px = 0.f, pd = 0.f;
            if (rg == 0) {
                const int64_t j0 = kb * 64 + c * CPL;
                float* xr = X + (int64_t)q * ldx;
#pragma unroll
                for (int e = 0; e < CPL; ++e) {
                    if (j0 + e < m && DFS_IN_BOUNDS(st, j0 + e < ldx)) {
                        const float du = ((e & 1) ? acc[q][e >> 1].y : acc[q][e >> 1].x) * inv_l;
                        const float xn = xr[j0 + e] - du;
                        xr[j0 + e] = xn;
                        px = fmaf(xn, xn, px);
                        pd = fmaf(du, du, pd);
                    }
                }
            }
            // the lanes of a row in a fixed order, then into the warp's FP64 sums
#pragma unroll
            for (int o = 1; o < LPRC; o <<= 1) {
                px += __shfl_xor_sync(0xffffffffu, px, o);
                pd += __shfl_xor_sync(0xffffffffu, pd, o);
            }
            if (lane == 0) {
                red[warp][q] += (double)px;
                red[warp][KQ + q] += (double)pd;
            }
        }
    }
    // per-CTA sums: the warps in order
    __syncthreads();
    if (tid < 2 * KQ) {
        double t = 0.0;
        for (int w = 0; w < wpb; ++w) t += red[w][tid];
        U2part[(int64_t)blockIdx.x * 2 * KQ + tid] = tid < KQ ? t * lambda * lambda : t;
    }
}

// grid: the SM count (the launch multiplies it by the resident CTAs per SM); U2part needs
// tile_correct_parts(num_sms) x 2 kq doubles.
int tile_correct_parts(int num_sms) { return 4 * num_sms; }

// Whether dy (n_rows x kq, stored twice) fits in the shared memory of one CTA.
bool tile_correct_fits(int n_rows, int kq, size_t smem_limit) {
    return (size_t)n_rows * kq * 2 * sizeof(float) + 4096 <= smem_limit;
}

cudaError_t launch_tile_correct(int kq, const void* Sp, int n, int n_rows, int64_t m, int64_t nkb, const float* Z,
                                int k, double lambda, float* X, int64_t ldx, double* U2part, const DevStatus* st,
                                int grid, cudaStream_t stream, int* parts) {
    if (n_rows % TC_CORR_ROWS != 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)n_rows * kq * 2 * sizeof(float);
    const unsigned char* sp = static_cast<const unsigned char*>(Sp);
    // one wave of resident CTAs (grid = num_sms x CTAs per SM): the k-blocks are dealt statically
#define DFS_TCC(KQ)                                                                                           \
    {                                                                                                         \
        auto kern = tile_correct_kernel<KQ>;                                                                  \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        if (e != cudaSuccess) return e;                                                                       \
        int per_sm = 0;                                                                                       \
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_CORR_THREADS, smem)) !=      \
            cudaSuccess)                                                                                      \
            return e;                                                                                         \
        int g = grid * (per_sm > 0 ? per_sm : 1);                                                             \
        if (g > 4 * grid) g = 4 * grid;                                                                       \
        *parts = g;                                                                                           \
        kern<<<g, TC_CORR_THREADS, smem, stream>>>(sp, n, n_rows, m, nkb, Z, k, lambda, X, ldx, U2part, st);  \
        count_launch();                                                                                       \
        return cudaGetLastError();                                                                            \
    }
    switch (kq) {
        case 1: DFS_TCC(1)
        case 2: DFS_TCC(2)
        case 4: DFS_TCC(4)
        case 8: DFS_TCC(8)
        default: return cudaErrorInvalidValue;
    }
#undef DFS_TCC
}

// ------------------------------------------------------------------------------------------
// X = (V - S^T Y) / lambda and R = S (V - S^T Y) - lambda Y in one read of S.
template <typename TS, int KQ, int RPT>
__global__ void __launch_bounds__(PASS_THREADS)
fisher_pass_kernel(const TS* __restrict__ S, int n, int64_t m, int64_t lds,
                   const typename PassTypes<TS>::TA* __restrict__ V, int64_t ldv, int k,
                   const double* __restrict__ Y, int64_t ldy, double lambda,
                   typename PassTypes<TS>::TA* __restrict__ X, int64_t ldx,
                   double* __restrict__ Rpart, double* __restrict__ U2part, int dmode,
                   const DevStatus* st, int honor_stop) {
    using TA = typename PassTypes<TS>::TA;
    constexpr int VEC = Vec16<TS>::N;
    constexpr int LPR = 8;
    constexpr int W = LPR * VEC;
    constexpr int RPW = 4;
    constexpr int SWEEP = PASS_WARPS * RPW;  // 64 rows
    constexpr int RB = 8;                    // re-read mode: rows in flight per thread
    extern __shared__ __align__(16) unsigned char smem[];
    // register-resident mode: the next strip lands here (cp.async) while this one is processed
    uint4* stage = reinterpret_cast<uint4*>(smem);               // RPT x PASS_THREADS x 16 bytes
    double* Rs64 = reinterpret_cast<double*>(smem + (size_t)RPT * PASS_THREADS * 16);  // n x KQ
    TA* Rs32 = reinterpret_cast<TA*>(Rs64 + (size_t)n * KQ);     // n x KQ
    TA* Ys = Rs32 + (size_t)n * KQ;                              // n x KQ
    TA* ured = Ys + (size_t)n * KQ;                              // PASS_WARPS x W x KQ
    TA* us = ured + PASS_WARPS * W * KQ;                         // W x KQ
    if (block_should_exit(st, honor_stop)) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rr = lane / LPR, cq = lane % LPR;
    const bool haveY = (Y != nullptr);
    const bool wantR = (Rpart != nullptr);
    const TA inv_lambda = (TA)(1.0 / lambda);
    for (int e = tid; e < n * KQ; e += PASS_THREADS) {
        const int i = e / KQ, q = e % KQ;
        Rs64[e] = 0.0;
        Rs32[e] = (TA)0;
        Ys[e] = (haveY && q < k) ? (TA)Y[(int64_t)i * ldy + q] : (TA)0;
    }
    TA u2f[KQ], d2f[KQ];
    double u2[KQ], d2[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) u2f[q] = d2f[q] = (TA)0, u2[q] = d2[q] = 0.0;
    __syncthreads();

    const int64_t nstrips = ceil_div(m, W);
    const int row0 = warp * RPW + rr;
    const bool u_thread = tid < W * KQ;
    const int uc = tid / KQ, uq = tid % KQ;
    // This thread's RPT row segments of strip sidx -> stage (zero-filled past row n / column m).
    // Each thread later reads back exactly the slots it filled, so no barrier is involved.
    auto issue_strip = [&](int64_t sidx) {
        const int64_t jn = sidx * W + cq * VEC;
        const int64_t rem = m - jn;
        const int bytes_col = rem >= VEC ? 16 : (rem > 0 ? (int)rem * (int)sizeof(TS) : 0);
#pragma unroll
        for (int t = 0; t < (RPT > 0 ? RPT : 1); ++t) {
            const int i = row0 + t * SWEEP;
            const int bytes = i < n ? bytes_col : 0;
            const TS* src = bytes ? S + (int64_t)i * lds + jn : S;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             static_cast<uint32_t>(__cvta_generic_to_shared(&stage[t * PASS_THREADS + tid]))),
                         "l"(src), "r"(bytes)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if constexpr (RPT > 0) {
        if (blockIdx.x < nstrips) issue_strip(blockIdx.x);
    }
    int since_fold = 0;
    for (int64_t s = blockIdx.x; s < nstrips; s += gridDim.x) {
        const int64_t j0 = s * W;
        const int64_t jc = j0 + cq * VEC;
        const bool full = (j0 + W <= m);
        // the U step's global reads, issued before phase 1 so their latency is hidden
        TA v_pre = 0, x_pre = 0;
        const bool u_valid = u_thread && (j0 + uc < m) && (uq < k);
        if (u_valid) {
            v_pre = V[(int64_t)uq * ldv + j0 + uc];
            if (X != nullptr && dmode == 1) x_pre = X[(int64_t)uq * ldx + j0 + uc];
        }
        TA sv[RPT > 0 ? RPT : 1][VEC];
        if constexpr (RPT > 0) {
            asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
            for (int t = 0; t < RPT; ++t)
                load16_smem<TS, TA>(reinterpret_cast<const TS*>(&stage[t * PASS_THREADS + tid]), sv[t]);
            if (s + gridDim.x < nstrips) issue_strip(s + gridDim.x);
        }
        // ---- phase 1: column sums of S^T Y over the strip ----
        if (haveY) {
            TA acc[KQ][VEC];
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc[q][e] = 0;
            if constexpr (RPT > 0) {
#pragma unroll
                for (int t = 0; t < RPT; ++t) {
                    const int i = row0 + t * SWEEP;
                    if (i < n) {
#pragma unroll
                        for (int q = 0; q < KQ; ++q) {
                            const TA yv = Ys[i * KQ + q];
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[q][e] = fma(sv[t][e], yv, acc[q][e]);
                        }
                    }
                }
            } else {
                for (int ib = row0; ib < n; ib += RB * SWEEP) {
                    TA rv[RB][VEC];
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int i = ib + u * SWEEP;
                        const TS* p = S + (int64_t)i * lds + jc;
                        if (i < n && full) {
                            load16<TS, TA>(p, rv[u]);
                        } else {
#pragma unroll
                            for (int e = 0; e < VEC; ++e)
                                rv[u][e] = (i < n && jc + e < m) ? load1<TS, TA>(p + e) : (TA)0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int i = ib + u * SWEEP;
#pragma unroll
                        for (int q = 0; q < KQ; ++q) {
                            const TA yv = (i < n) ? Ys[i * KQ + q] : (TA)0;
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[q][e] = fma(rv[u][e], yv, acc[q][e]);
                        }
                    }
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
        // ---- U = V - S^T Y, X = U / lambda ----
        if (u_thread) {
            TA sum = 0;
            if (haveY)
                for (int w = 0; w < PASS_WARPS; ++w) sum += ured[(w * W + uc) * KQ + uq];
            const TA u = u_valid ? v_pre - sum : (TA)0;
            us[uc * KQ + uq] = u;
            if (u_valid) {
                if (X != nullptr) {
                    const TA xn = u * inv_lambda;
                    TA dx = 0;
                    if (dmode == 1) dx = xn - x_pre;
                    else if (dmode == 2) dx = (u - v_pre) * inv_lambda;
                    d2f[uq] += dx * dx;
                    X[(int64_t)uq * ldx + j0 + uc] = xn;
                }
                u2f[uq] += u * u;
            }
        }
        __syncthreads();
        // ---- phase 2: R_s += S_strip U_strip ----
        if (wantR) {
            TA uu[KQ][VEC];
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < VEC; ++e) uu[q][e] = us[(cq * VEC + e) * KQ + q];
            if constexpr (RPT > 0) {
#pragma unroll
                for (int t = 0; t < RPT; ++t) {
                    const int i = row0 + t * SWEEP;
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        TA a = 0;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) a = fma(sv[t][e], uu[q][e], a);
                        a += __shfl_xor_sync(0xffffffffu, a, 1);
                        a += __shfl_xor_sync(0xffffffffu, a, 2);
                        a += __shfl_xor_sync(0xffffffffu, a, 4);
                        if (cq == 0 && i < n) Rs32[i * KQ + q] += a;
                    }
                }
            } else {
                // warp-uniform row loop (the shuffles need all 32 lanes)
                for (int base = warp * RPW; base < n; base += RB * SWEEP) {
                    TA rv[RB][VEC];
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int i = base + u * SWEEP + rr;
                        const TS* p = S + (int64_t)i * lds + jc;
                        if (i < n && full) {
                            load16<TS, TA>(p, rv[u]);
                        } else {
#pragma unroll
                            for (int e = 0; e < VEC; ++e)
                                rv[u][e] = (i < n && jc + e < m) ? load1<TS, TA>(p + e) : (TA)0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int i = base + u * SWEEP + rr;
#pragma unroll
                        for (int q = 0; q < KQ; ++q) {
                            TA a = 0;
#pragma unroll
                            for (int e = 0; e < VEC; ++e) a = fma(rv[u][e], uu[q][e], a);
                            a += __shfl_xor_sync(0xffffffffu, a, 1);
                            a += __shfl_xor_sync(0xffffffffu, a, 2);
                            a += __shfl_xor_sync(0xffffffffu, a, 4);
                            if (cq == 0 && i < n) Rs32[i * KQ + q] += a;
                        }
                    }
                }
            }
        }
        if (++since_fold == kFold) {
            since_fold = 0;
            if (wantR && cq == 0) fold_rows<TA, KQ>(Rs64, Rs32, row0, SWEEP, n);
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                u2[q] += (double)u2f[q];
                d2[q] += (double)d2f[q];
                u2f[q] = d2f[q] = (TA)0;
            }
        }
    }
    if (wantR && cq == 0) fold_rows<TA, KQ>(Rs64, Rs32, row0, SWEEP, n);
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        u2[q] += (double)u2f[q];
        d2[q] += (double)d2f[q];
    }
    __syncthreads();
    if (wantR) {
        double* dst = Rpart + (int64_t)blockIdx.x * n * KQ;
        for (int e = tid; e < n * KQ; e += PASS_THREADS) dst[e] = Rs64[e];
    }
    // per-RHS sums of U^2 and (X_new - X_old)^2 (threads tid < W*KQ hold disjoint columns)
    __shared__ double u2s[PASS_WARPS][16];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        double v = u2[q], w = d2[q];
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (lane == 0) {
            u2s[warp][q] = v;
            u2s[warp][8 + q] = w;
        }
    }
    __syncthreads();
    if (tid < KQ) {
        double v = 0.0, w = 0.0;
        for (int wp = 0; wp < PASS_WARPS; ++wp) {
            v += u2s[wp][tid];
            w += u2s[wp][8 + tid];
        }
        U2part[(int64_t)blockIdx.x * 2 * KQ + tid] = v;
        U2part[(int64_t)blockIdx.x * 2 * KQ + KQ + tid] = w;
    }
}

// R = sum_b Rpart[b] - lambda Y (FP64, fixed order), rows [0, n_out) with stride ldr (rows >= n
// are zero), an optional copy Rt (n_out x KQ, solve type T) for the triangular solves, and the
// summed ||U||^2 and ||X_new - X_old||^2 per RHS (U2[0..KQ) and U2[KQ..2KQ)).
// A CTA owns 32 consecutive outputs e; its 16 thread groups walk the parts b = g, g + 16, ...
// (each load a coalesced 256-byte row segment), then group sums are added in group order.
constexpr int RED_GROUPS = 16;

template <typename T>
__global__ void __launch_bounds__(RED_GROUPS * 32)
pass_reduce_kernel(const double* __restrict__ Rpart, int nparts, int n, int n_out, int KQ, int k,
                   const double* __restrict__ Y, int64_t ldy, double lambda, double* __restrict__ R, int64_t ldr,
                   T* __restrict__ Rt, const double* __restrict__ U2part, double* __restrict__ U2,
                   const DevStatus* st, int honor_stop) {
    __shared__ double red[RED_GROUPS][33];
    if (st->status != 0 || (honor_stop && st->stop)) return;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    const int64_t nin = (int64_t)n * KQ;
    double v = 0.0;
    if (e < nin) {
        const double* p = Rpart + e;
#pragma unroll 4
        for (int b = grp; b < nparts; b += RED_GROUPS) v += p[(int64_t)b * nin];
    }
    red[grp][lane] = v;
    __syncthreads();
    if (grp == 0 && e < (int64_t)n_out * KQ) {
        double t = 0.0;
#pragma unroll
        for (int g = 0; g < RED_GROUPS; ++g) t += red[g][lane];
        const int i = (int)(e / KQ), q = (int)(e % KQ);
        if (!(i < n && q < k)) t = 0.0;
        if (i < n && q < k && Y != nullptr) t -= lambda * Y[(int64_t)i * ldy + q];
        if (R != nullptr && q < k) R[(int64_t)i * ldr + q] = t;
        if (Rt != nullptr) Rt[e] = (T)t;
    }
    if (U2 != nullptr && U2part != nullptr && blockIdx.x == 0 && threadIdx.x < 2 * KQ) {
        double u = 0.0;
        for (int b = 0; b < nparts; ++b) u += U2part[(int64_t)b * 2 * KQ + threadIdx.x];
        U2[threadIdx.x] = u;
    }
}

// ---- host side ------------------------------------------------------------------------------

static int vec_of(int s_dtype) { return s_dtype == DFS_F64 ? 2 : (s_dtype == DFS_F32 ? 4 : 8); }
static int ta_of(int s_dtype) { return s_dtype == DFS_F64 ? 8 : 4; }

static int pass_rpt(int n, int KQ, int s_dtype);

// Dynamic shared memory of fisher_pass_kernel, including the strip stage of the
// register-resident mode.
size_t pass_smem_bytes(int n, int KQ, int s_dtype) {
    const int ta = ta_of(s_dtype);
    const int W = 8 * vec_of(s_dtype);
    const size_t stage = (size_t)pass_rpt(n, KQ, s_dtype) * PASS_THREADS * 16;
    return stage + (size_t)n * KQ * (8 + 2 * ta) + (size_t)PASS_WARPS * W * KQ * ta + (size_t)W * KQ * ta;
}

static size_t sv_smem_bytes(int n, int KQ, int s_dtype) { return (size_t)n * KQ * (8 + ta_of(s_dtype)); }

int pass_max_group(int n, int s_dtype, size_t smem_limit) {
    for (int kq = 8; kq >= 1; kq >>= 1)
        if (pass_smem_bytes(n, kq, s_dtype) <= smem_limit) return kq;
    return 0;
}

// Rows per thread kept in registers by fisher_pass_kernel (0: phase 2 re-reads the strip).
static int pass_rpt(int n, int KQ, int s_dtype) {
    const int vec = vec_of(s_dtype);
    int rpt = 2;
    while (rpt * 64 < n) rpt *= 2;
    if (rpt * vec > 64 || KQ * vec > 16 || rpt > 16) return 0;
    return rpt;
}

PassPlan pass_make_plan(int n, int KQ, int s_dtype, int num_sms, int64_t m, size_t smem_limit, int allow_two) {
    PassPlan p{};
    p.rpt = pass_rpt(n, KQ, s_dtype);
    // register-resident strips: one 512-thread CTA per SM; otherwise up to four
    const size_t smem = pass_smem_bytes(n, KQ, s_dtype);
    int per_sm = p.rpt > 0 ? 1 : (int)((200u * 1024u) / (smem + 1024));
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
    const int64_t nstrips = ceil_div(m, 8 * vec_of(s_dtype));
    int64_t g = (int64_t)num_sms * per_sm;
    if (g > nstrips) g = nstrips;
    p.grid = (int)(g < 1 ? 1 : g);
    // the S v pass: one wave of one CTA per SM (its 512 threads x 80 registers fill an SM), so
    // that the n-space step has num_sms partial rows to add
    int64_t gs = (int64_t)num_sms;
    if (gs > nstrips) gs = nstrips;
    p.sv_grid = (int)(gs < 1 ? 1 : gs);
    // FP32 S with n <= 4096: clusters sharing 256-byte-wide strips (pass_cluster.cu)
    p.ncl = smem_limit ? pass_cluster_plan(s_dtype, n, KQ, num_sms, m, smem_limit, &p.cs, &p.crpt) : 0;
    if (p.ncl == 0) p.cs = p.crpt = 0;
    p.nparts = p.cs > 0 ? p.ncl : p.grid;
    p.uparts = p.nparts;
    p.two = 0;
    // n > 2048 rows (FP32 or BF16 S, up to 4 RHS) with a 4096-column chunk for every SM: the pass
    // as sty_cols_kernel then sv_rows_kernel, two reads of S by rows shared across each CTA, in
    // place of one read by strips that span all n rows (which address translation holds to a
    // fraction of HBM bandwidth at this n)
    if (allow_two && (s_dtype == DFS_F32 || s_dtype == DFS_BF16) && KQ <= 4 && n > 2048 &&
        ceil_div(m, (int64_t)STY_COLS) >= num_sms) {
        p.two = 1;
        p.uparts = num_sms;
        p.nparts = sv_rows_chunks((int)round_up(n, 8) / SvbRows<1>::R, m, p.sv_grid);
    }
    return p;
}

int pass_grid(int n, int KQ, int s_dtype, int num_sms, int64_t m) {
    return pass_make_plan(n, KQ, s_dtype, num_sms, m, 0).grid;
}

int pass_partial_rows(const PassPlan& p) { return p.grid > p.sv_grid ? p.grid : p.sv_grid; }

template <typename TS, int KQ, int RPT>
static cudaError_t launch_pass_t(const void* S, int n, int64_t m, int64_t lds, const void* V, int64_t ldv, int k,
                                 const double* Y, int64_t ldy, double lambda, void* X, int64_t ldx, double* Rpart,
                                 double* U2part, int dmode, int grid, const DevStatus* st, int honor_stop,
                                 cudaStream_t stream, int s_dtype) {
    using TA = typename PassTypes<TS>::TA;
    const size_t smem = pass_smem_bytes(n, KQ, s_dtype);
    auto kern = fisher_pass_kernel<TS, KQ, RPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, PASS_THREADS, smem, stream>>>(static_cast<const TS*>(S), n, m, lds, static_cast<const TA*>(V), ldv,
                                               k, Y, ldy, lambda, static_cast<TA*>(X), ldx, Rpart, U2part, dmode, st,
                                               honor_stop);
    count_launch();
    return cudaGetLastError();
}

template <typename TS, int KQ>
static cudaError_t launch_pass_rpt(int rpt, const void* S, int n, int64_t m, int64_t lds, const void* V, int64_t ldv,
                                   int k, const double* Y, int64_t ldy, double lambda, void* X, int64_t ldx,
                                   double* Rpart, double* U2part, int dmode, int grid, const DevStatus* st,
                                   int honor_stop, cudaStream_t stream, int s_dtype) {
#define DFS_RPT(R)                                                                                             \
    case R:                                                                                                    \
        return launch_pass_t<TS, KQ, R>(S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart, U2part, dmode, \
                                        grid, st, honor_stop, stream, s_dtype);
    switch (rpt) {
        DFS_RPT(0)
        DFS_RPT(2)
        DFS_RPT(4)
        DFS_RPT(8)
        DFS_RPT(16)
        default:
            return cudaErrorInvalidValue;
    }
#undef DFS_RPT
}

cudaError_t launch_pass(const PassPlan& plan, int s_dtype, int kq, const void* S, int n, int64_t m, int64_t lds,
                        const void* V, int64_t ldv, int k, const double* Y, int64_t ldy, double lambda, void* X,
                        int64_t ldx, double* Rpart, double* U2part, int dmode, const DevStatus* st, int honor_stop,
                        cudaStream_t stream) {
    if (plan.two && X != nullptr && (s_dtype == DFS_F32 || s_dtype == DFS_BF16) && kq <= 4) {
        // X = (V - S^T Y) / lambda, then the partial rows of R = S U (the reduce subtracts lambda Y)
        cudaError_t e = cudaSuccess;
#define DFS_STY(TS, KQ)                                                                                          \
    if ((e = cudaFuncSetAttribute(sty_cols_kernel<TS, KQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                  (int)sty_smem_bytes(KQ))) != cudaSuccess)                                        \
        return e;                                                                                                 \
    sty_cols_kernel<TS, KQ><<<plan.uparts, SVB_THREADS, sty_smem_bytes(KQ), stream>>>(                           \
        static_cast<const TS*>(S), n, m, lds, static_cast<const float*>(V), ldv, k, Y, ldy, lambda,               \
        static_cast<float*>(X), ldx, U2part, dmode, st, honor_stop)
#define DFS_STY_KQ(TS)                  \
    switch (kq) {                       \
        case 1: DFS_STY(TS, 1); break;  \
        case 2: DFS_STY(TS, 2); break;  \
        default: DFS_STY(TS, 4); break; \
    }
        if (s_dtype == DFS_F32) {
            DFS_STY_KQ(float)
        } else {
            DFS_STY_KQ(__nv_bfloat16)
        }
#undef DFS_STY_KQ
#undef DFS_STY
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess || Rpart == nullptr) return e;
        // X = U * fl(1 / lambda) in FP32, so U = X / fl(1 / lambda) up to X's own rounding
        const int n_rows = (int)round_up(n, 8);
        const double scale = 1.0 / (double)(float)(1.0 / lambda);
#define DFS_SVR2(TS, KQ)                                                                                         \
    launch_sv_rows_t<TS, KQ, 0>(plan.nparts, S, n, n_rows, m, lds, X, ldx, k, Rpart, nullptr, st, stream, scale, \
                                honor_stop)
        if (s_dtype == DFS_F32) {
            switch (kq) {
                case 1: return DFS_SVR2(float, 1);
                case 2: return DFS_SVR2(float, 2);
                default: return DFS_SVR2(float, 4);
            }
        }
        switch (kq) {
            case 1: return DFS_SVR2(__nv_bfloat16, 1);
            case 2: return DFS_SVR2(__nv_bfloat16, 2);
            default: return DFS_SVR2(__nv_bfloat16, 4);
        }
#undef DFS_SVR2
    }
    if (plan.cs > 0 && s_dtype == DFS_F32)
        return launch_pass_cluster(plan.ncl, plan.cs, plan.crpt, kq, S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx,
                                   Rpart, U2part, dmode, st, honor_stop, stream);
#define DFS_PASS_CASE(KQ)                                                                                         \
    case KQ:                                                                                                      \
        if (s_dtype == DFS_F32)                                                                                   \
            return launch_pass_rpt<float, KQ>(plan.rpt, S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart,   \
                                              U2part, dmode, plan.grid, st, honor_stop, stream, s_dtype);         \
        if (s_dtype == DFS_BF16)                                                                                  \
            return launch_pass_rpt<__nv_bfloat16, KQ>(plan.rpt, S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx,  \
                                                      Rpart, U2part, dmode, plan.grid, st, honor_stop, stream,    \
                                                      s_dtype);                                                   \
        if (s_dtype == DFS_F64)                                                                                   \
            return launch_pass_rpt<double, KQ>(plan.rpt, S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart,  \
                                               U2part, dmode, plan.grid, st, honor_stop, stream, s_dtype);        \
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

template <typename TS, int KQ, int PACK>
static cudaError_t launch_sv_t(int grid, const void* S, int n, int n_rows, int64_t m, int64_t lds, const void* V,
                               int64_t ldv, int k, double* Rpart, void* Sp, int64_t nkb, const DevStatus* st,
                               cudaStream_t stream, int s_dtype, const float* rinv) {
    using TA = typename PassTypes<TS>::TA;
    const size_t smem = sv_smem_bytes(n, KQ, s_dtype);
    auto kern = sv_pack_kernel<TS, KQ, PACK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, PASS_THREADS, smem, stream>>>(static_cast<const TS*>(S), n, n_rows, m, lds, static_cast<const TA*>(V),
                                               ldv, k, Rpart, static_cast<unsigned char*>(Sp), nkb, st, rinv);
    count_launch();
    return cudaGetLastError();
}

// S v launches for KQ right-hand sides: every (S dtype, packing) pair that exists
template <int KQ>
static cudaError_t launch_sv_kq(int grid, int s_dtype, int pack, const void* S, int n, int n_rows, int64_t m,
                                int64_t lds, const void* V, int64_t ldv, int k, double* Rpart, void* Sp, int64_t nkb,
                                const DevStatus* st, cudaStream_t stream, const float* rinv) {
#define DFS_SV(TS, PK) \
    launch_sv_t<TS, KQ, PK>(grid, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st, stream, s_dtype, rinv)
    if (s_dtype == DFS_F32) {
        switch (pack) {
            case 0: return DFS_SV(float, 0);
            case 1: return DFS_SV(float, 1);
            case 2: return DFS_SV(float, 2);
            case 3: return DFS_SV(float, 3);
            case 4: return DFS_SV(float, 4);
            default: return cudaErrorInvalidValue;
        }
    }
    if (s_dtype == DFS_BF16) {
        switch (pack) {
            case 0: return DFS_SV(__nv_bfloat16, 0);
            case 1: return DFS_SV(__nv_bfloat16, 1);
            case 4: return DFS_SV(__nv_bfloat16, 4);
            default: return cudaErrorInvalidValue;
        }
    }
    if (s_dtype == DFS_F64 && pack == 0) return DFS_SV(double, 0);
#undef DFS_SV
    return cudaErrorInvalidValue;
}

int64_t pack_kblocks(int s_dtype, int pack, int64_t m) {
    const int width = (pack == 2) ? 32 : (pack == 4 ? 128 : 64);  // elements per 128-byte tile row
    (void)s_dtype;
    return ceil_div(m, width);
}

// 128-row tiles per k-block: T rounded up to even, twice that for the stacked H / L operand
static int64_t pack_tiles_per_kblock(int pack, int64_t n) {
    const int64_t T = round_up(ceil_div(n, 128), 2);
    return pack == 3 ? 2 * T : T;
}

size_t pack_bytes(int s_dtype, int pack, int64_t n, int64_t m) {
    if (pack == 0) return 0;
    return (size_t)pack_tiles_per_kblock(pack, n) * (size_t)pack_kblocks(s_dtype, pack, m) * 16384;
}

template <int KQ, int PACK>
static cudaError_t launch_sv_ring_t(int grid, const void* S, int n, int n_rows, int64_t m, int64_t lds, const void* V,
                                    int64_t ldv, int k, double* Rpart, void* Sp, int64_t nkb, const DevStatus* st,
                                    cudaStream_t stream, const float* rinv) {
    const size_t smem = (size_t)SVR_SLOTS * SVR_TPS * PASS_THREADS * 16 + (size_t)n * KQ * 8;
    auto kern = sv_ring_kernel<KQ, PACK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, PASS_THREADS, smem, stream>>>(static_cast<const float*>(S), n, n_rows, m, lds,
                                               static_cast<const float*>(V), ldv, k, Rpart,
                                               static_cast<unsigned char*>(Sp), nkb, st, rinv);
    count_launch();
    return cudaGetLastError();
}

template <typename TS, int KQ>
static cudaError_t launch_sv_rows_kq(int pack, int nchunks, const void* S, int n, int n_rows, int64_t m, int64_t lds,
                                     const void* V, int64_t ldv, int k, double* Rpart, void* Sp, const DevStatus* st,
                                     cudaStream_t stream, const float* rinv) {
    if (pack == 4)
        return launch_sv_rows_t<TS, KQ, 4>(nchunks, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, st, stream, 1.0, 0,
                                           rinv);
    return pack ? launch_sv_rows_t<TS, KQ, 1>(nchunks, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, st, stream)
                : launch_sv_rows_t<TS, KQ, 0>(nchunks, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, st, stream);
}

cudaError_t launch_sv_pack(const PassPlan& plan, int s_dtype, int kq, int pack, const void* S, int n, int64_t m,
                           int64_t lds, const void* V, int64_t ldv, int k, double* Rpart, void* Sp,
                           const DevStatus* st, cudaStream_t stream, const float* rinv, int* parts) {
    if (parts) *parts = plan.sv_grid;
    // rows far apart (FP32 S beyond the streaming form's 1024 rows, or BF16 S), BF16 or row-scaled
    // e4m3 tiles or none: the row-blocked form
    if ((pack <= 1 || (pack == 4 && rinv != nullptr)) &&
        (s_dtype == DFS_BF16 || (s_dtype == DFS_F32 && round_up(n, 256) > SVR_MAXNR * (PASS_THREADS / 16)))) {
        const int n_rows = (int)round_up(n, pack ? 256 : 8);
        const int nchunks = sv_rows_chunks(n_rows / (kq >= 8 ? SvbRows<8>::R : SvbRows<1>::R), m, plan.sv_grid);
        if (parts) *parts = nchunks;
#define DFS_SVB(KQ)                                                                                          \
    case KQ:                                                                                                 \
        return s_dtype == DFS_F32                                                                            \
                   ? launch_sv_rows_kq<float, KQ>(pack, nchunks, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, st, \
                                                  stream, rinv)                                              \
                   : launch_sv_rows_kq<__nv_bfloat16, KQ>(pack, nchunks, S, n, n_rows, m, lds, V, ldv, k, Rpart, \
                                                          Sp, st, stream, rinv);
        switch (kq) {
            DFS_SVB(1)
            DFS_SVB(2)
            DFS_SVB(4)
            DFS_SVB(8)
            default:
                return cudaErrorInvalidValue;
        }
#undef DFS_SVB
    }
    if (pack == 3 && s_dtype != DFS_F32) return cudaErrorInvalidValue;
    if (pack == 4 && (rinv == nullptr || s_dtype == DFS_F64)) return cudaErrorInvalidValue;
    // packed rows: an even number of 128-row blocks (the Gram's units pair blocks), zero past n
    const int n_rows = pack ? (int)round_up(n, 256) : n;
    const int64_t nkb = pack ? pack_kblocks(s_dtype, pack, m) : 0;
    const int grid = plan.sv_grid;
    // the streaming form: FP32 S, no packing or BF16 (H / L) tiles, up to 1024 rows and 2 RHS
    if (s_dtype == DFS_F32 && pack != 2 && n_rows <= SVR_MAXNR * (PASS_THREADS / 16) && kq <= 2) {
#define DFS_SVR(KQ)                                                                                      \
    switch (pack) {                                                                                        \
        case 4: return launch_sv_ring_t<KQ, 4>(grid, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st,   \
                                               stream, rinv);                                              \
        case 3: return launch_sv_ring_t<KQ, 3>(grid, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st,   \
                                               stream, rinv);                                              \
        case 1: return launch_sv_ring_t<KQ, 1>(grid, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st,   \
                                               stream, rinv);                                              \
        default: return launch_sv_ring_t<KQ, 0>(grid, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st,  \
                                                stream, rinv);                                             \
    }
        if (kq == 1) DFS_SVR(1)
        DFS_SVR(2)
#undef DFS_SVR
    }
switch (kq) {
        case 1: return launch_sv_kq<1>(grid, s_dtype, pack, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st, stream, rinv);
        case 2: return launch_sv_kq<2>(grid, s_dtype, pack, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st, stream, rinv);
        case 4: return launch_sv_kq<4>(grid, s_dtype, pack, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st, stream, rinv);
        case 8: return launch_sv_kq<8>(grid, s_dtype, pack, S, n, n_rows, m, lds, V, ldv, k, Rpart, Sp, nkb, st, stream, rinv);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass_reduce(int f64, const double* Rpart, int nparts, int n, int n_out, int KQ, int k,
                               const double* Y, int64_t ldy, double lambda, double* R, int64_t ldr, void* Rt,
                               const double* U2part, double* U2, const DevStatus* st, int honor_stop,
                               cudaStream_t stream) {
    const int blocks = (int)ceil_div((int64_t)n_out * KQ, 32);
    if (f64) {
        pass_reduce_kernel<double><<<blocks, RED_GROUPS * 32, 0, stream>>>(Rpart, nparts, n, n_out, KQ, k, Y, ldy, lambda, R, ldr,
                                                               static_cast<double*>(Rt), U2part, U2, st, honor_stop);
    } else {
        pass_reduce_kernel<float><<<blocks, RED_GROUPS * 32, 0, stream>>>(Rpart, nparts, n, n_out, KQ, k, Y, ldy, lambda, R, ldr,
                                                              static_cast<float*>(Rt), U2part, U2, st, honor_stop);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace dfs
