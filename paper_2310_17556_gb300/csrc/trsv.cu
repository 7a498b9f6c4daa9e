// The two triangular solves of Section 2 (Q inlined): A = L^{-1} B, then Y = L^{-T} A.
//
// Both run in ONE CTA over the padded factor held in W (L in the lower triangle and, written by
// the Cholesky, U = L^T in the upper triangle) and the inverses Linv_i of its 32 x 32 diagonal
// blocks.  Row block i of the solve is
//   forward   t = B_i - L[i, <i] A_<i ,  A_i = Linv_i t
//   backward  t = A_i - U[i, >i] Y_>i ,  Y_i = Linv_i^T t
// so both stream row segments of W (contiguous in memory) in the order the solve consumes them.
// None of these loads depends on the solution, so a producer thread streams them ahead through an
// up-to-8-stage shared-memory ring, one TMA tile load (32 rows x 512 bytes of W, through a 2-D
// tensor map) per stage with completion on an mbarrier, keeping ~128 KB in flight from L2; eight
// consumer warps do the GEMV on each stage as it lands (thread: one row, 16-byte column groups),
// reduce per row block with shuffles, and apply Linv_i, which arrives as the block's last stage.
// The right-hand sides (n_pad x KQ, interleaved) stay in shared memory for the whole solve.
// Products and sums are in the storage type of L (FP32 on the FP32/mixed paths, FP64 on the FP64
// path).  With `stop` set in the device status (refinement already converged) the kernel returns
// at once; every wait is bounded (DFS_ERR_TIMEOUT).
#include <cudaTypedefs.h>

#include <cstring>

#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dfs {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();  // gram_tc.cu

constexpr int TB = 32;                  // rows per block (the Cholesky's NB)
constexpr int TS_CONS_WARPS = 8;        // consumer warps
constexpr int TS_THREADS = (TS_CONS_WARPS + 1) * 32;
constexpr int TS_STAGES = 8;
constexpr int TS_STAGE_BYTES = 16384;   // 32 rows x 512 bytes

// Items of the stream: for row block i (in solve order), chunks of up to CW columns of the row
// segment, then Linv_i.  Returned through (ncols of this chunk, c0), or ncols == 0 for Linv.
template <typename T>
struct TrsvSeq {
    static constexpr int CW = TS_STAGE_BYTES / (TB * (int)sizeof(T));  // columns per chunk
    int n_pad, dir;
    __device__ int block_of(int step) const { return dir == 0 ? step : n_pad / TB - 1 - step; }
    // columns [lo, hi) of row block ib that enter the GEMV
    __device__ void span(int ib, int& lo, int& hi) const {
        if (dir == 0) {
            lo = 0;
            hi = ib * TB;
        } else {
            lo = (ib + 1) * TB;
            hi = n_pad;
        }
    }
    __device__ int chunks(int ib) const {
        int lo, hi;
        span(ib, lo, hi);
        return (hi - lo + CW - 1) / CW;
    }
};

template <typename T, int KQ>
__global__ void __launch_bounds__(TS_THREADS, 1)
trsv_stream_kernel(const __grid_constant__ CUtensorMap tmap, int n_pad, const T* __restrict__ Linv,
                   T* __restrict__ B, int64_t ldb, int k, int dir, int nst, DevStatus* st, int honor_stop) {
    using Seq = TrsvSeq<T>;
    constexpr int CW = Seq::CW;
    constexpr int VEC = 16 / (int)sizeof(T);  // elements per 16-byte column group
    constexpr int GPR = 8;                    // threads per row
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage = smem;                                              // nst x 16 KB
    T* x = reinterpret_cast<T*>(smem + (size_t)nst * TS_STAGE_BYTES);         // n_pad x KQ
    T* tb = x + (size_t)n_pad * KQ;                                           // TB x KQ
    __shared__ __align__(8) uint64_t full[TS_STAGES], empty[TS_STAGES];
    __shared__ int s_abort;
    if (block_should_exit(st, honor_stop)) return;
    const uint64_t wait_ns = wait_limit(st);  // the call's wait limit, read once
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Seq seq{n_pad, dir};
    const int nblk = n_pad / TB;
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], TS_CONS_WARPS);
        }
        tc::fence_mbar_init();
        s_abort = 0;
    }
    for (int e = tid; e < n_pad * KQ; e += blockDim.x) {
        const int i = e / KQ, q = e % KQ;
        x[e] = (q < k) ? B[(int64_t)i * ldb + q] : (T)0;
    }
    __syncthreads();

    if (warp == TS_CONS_WARPS) {
        // ---------------- producer (one thread) ----------------
        if (lane != 0) return;
        tc::prefetch_tmap(&tmap);
        uint32_t it = 0;
        for (int step = 0; step < nblk; ++step) {
            const int ib = seq.block_of(step);
            int lo, hi;
            seq.span(ib, lo, hi);
            const int nch = seq.chunks(ib);
            for (int c = 0; c <= nch; ++c, ++it) {
                const int s = (int)(it % nst);
                const uint32_t ph = (it / nst) & 1u;
                if (it >= (uint32_t)nst && !tc::mbar_wait_bounded(&empty[s], ph ^ 1u, &s_abort, wait_ns)) {
                    s_abort = 1;
                    set_status(st, DFS_ERR_TIMEOUT);
                    return;
                }
                unsigned char* dst = stage + (size_t)s * TS_STAGE_BYTES;
                if (c < nch) {
                    // the whole 32 x CW box lands (columns past the span are read but unused;
                    // past n_pad they are zero-filled)
                    tc::mbar_arrive_expect_tx(&full[s], TS_STAGE_BYTES);
                    tc::tma_load_2d(dst, &tmap, lo + c * CW, ib * TB, &full[s]);
                } else {
                    tc::mbar_arrive_expect_tx(&full[s], TB * TB * sizeof(T));
                    tc::bulk_load(dst, Linv + (int64_t)ib * TB * TB, TB * TB * sizeof(T), &full[s]);
                }
            }
        }
        return;
    }

    // ---------------- consumer warps: thread = (row r, column group g) ----------------
    const int ctid = tid;  // 0 .. 255
    const int r = ctid / GPR, g = ctid % GPR;
    uint32_t it = 0;
    for (int step = 0; step < nblk; ++step) {
        const int ib = seq.block_of(step);
        int lo, hi;
        seq.span(ib, lo, hi);
        const int nch = seq.chunks(ib);
        T acc[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q] = 0;
        for (int c = 0; c <= nch; ++c, ++it) {
            const int s = (int)(it % nst);
            const uint32_t ph = (it / nst) & 1u;
            if (!tc::mbar_wait_bounded(&full[s], ph, &s_abort, wait_ns)) {
                if (lane == 0) {
                    s_abort = 1;
                    set_status(st, DFS_ERR_TIMEOUT);
                }
                return;
            }
            const T* sl = reinterpret_cast<const T*>(stage + (size_t)s * TS_STAGE_BYTES);
            if (c < nch) {
                const int c0 = lo + c * CW;
                const int w = (hi - c0) < CW ? (hi - c0) : CW;
                for (int u = g * VEC; u < w; u += GPR * VEC) {
                    T lv[VEC];
                    load16_smem<T, T>(sl + r * CW + u, lv);
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
#pragma unroll
                        for (int q = 0; q < KQ; ++q) acc[q] = fma(lv[e], x[(c0 + u + e) * KQ + q], acc[q]);
                }
            } else {
                // t = rhs_i - (row sums), then X_i = Linv_i t (forward) or Linv_i^T t (backward)
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
#pragma unroll
                    for (int o = 1; o < GPR; o <<= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
                    if (g == 0) tb[r * KQ + q] = x[(ib * TB + r) * KQ + q] - acc[q];
                }
                asm volatile("bar.sync 1, %0;" ::"n"(TS_CONS_WARPS * 32) : "memory");
                T y[KQ];
#pragma unroll
                for (int q = 0; q < KQ; ++q) y[q] = 0;
#pragma unroll
                for (int e = 0; e < TB / GPR; ++e) {
                    const int p = g * (TB / GPR) + e;
                    const T li = dir == 0 ? sl[r * TB + p] : sl[p * TB + r];
#pragma unroll
                    for (int q = 0; q < KQ; ++q) y[q] = fma(li, tb[p * KQ + q], y[q]);
                }
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
#pragma unroll
                    for (int o = 1; o < GPR; o <<= 1) y[q] += __shfl_xor_sync(0xffffffffu, y[q], o);
                    if (g == 0) x[(ib * TB + r) * KQ + q] = y[q];
                }
                asm volatile("bar.sync 1, %0;" ::"n"(TS_CONS_WARPS * 32) : "memory");
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
        }
    }
    for (int e = ctid; e < n_pad * KQ; e += TS_CONS_WARPS * 32) {
        const int i = e / KQ, q = e % KQ;
        if (q < k) B[(int64_t)i * ldb + q] = x[e];
    }
}

// Ring stages that fit next to the right-hand sides (at most TS_STAGES, at least 2; 0: none).
static int trsv_stages(int n_pad, int KQ, int elem, size_t smem_limit) {
    const size_t rhs = ((size_t)n_pad * KQ + TB * KQ) * elem + 1024;  // + static shared memory
    if (rhs + 2 * (size_t)TS_STAGE_BYTES > smem_limit) return 0;
    const size_t n = (smem_limit - rhs) / TS_STAGE_BYTES;
    return n > (size_t)TS_STAGES ? TS_STAGES : (int)n;
}

size_t trsv_smem_bytes(int n_pad, int KQ, int elem, int nst) {
    return (size_t)nst * TS_STAGE_BYTES + ((size_t)n_pad * KQ + TB * KQ) * elem;
}

static size_t device_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

template <typename T, int KQ>
static cudaError_t launch_trsv_t(int trans, const void* L, int64_t ld, int n_pad, const void* Linv, void* B,
                                 int64_t ldb, int k, const DevStatus* st, int honor_stop, cudaStream_t stream) {
    const int nst = trsv_stages(n_pad, KQ, sizeof(T), device_smem_optin());
    if (nst < 2) return cudaErrorInvalidValue;
    const size_t smem = trsv_smem_bytes(n_pad, KQ, sizeof(T), nst);
    auto encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)n_pad};
    cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)TrsvSeq<T>::CW, (cuuint32_t)TB};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&map, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void*>(L), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    auto kern = trsv_stream_kernel<T, KQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, TS_THREADS, smem, stream>>>(map, n_pad, static_cast<const T*>(Linv),
                                          static_cast<T*>(B), ldb, k, trans, nst, const_cast<DevStatus*>(st),
                                          honor_stop);
    count_launch();
    return cudaGetLastError();
}

// Largest RHS group (1, 2, 4 or 8) for which the solve fits in shared memory.
int trsv_max_group(int n_pad, int elem, size_t smem_limit) {
    for (int kq = 8; kq >= 1; kq >>= 1)
        if (trsv_stages(n_pad, kq, elem, smem_limit) >= 2) return kq;
    return 0;
}

// U = L^T into the upper triangle of the padded factor (for triangular solves with a factor
// the caller supplies; the Cholesky writes U itself).  One 32 x 32 tile per CTA.
template <typename T>
__global__ void __launch_bounds__(256) mirror_lower_kernel(T* L, int64_t ld) {
    __shared__ T t[TB][TB + 1];
    const int bi = blockIdx.y, bp = blockIdx.x;
    if (bp >= bi) return;
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int r = e / TB, c = e % TB;
        t[r][c] = L[((int64_t)bi * TB + r) * ld + (int64_t)bp * TB + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int c = e / TB, r = e % TB;
        L[((int64_t)bp * TB + c) * ld + (int64_t)bi * TB + r] = t[r][c];
    }
}

cudaError_t launch_mirror_lower(int f64, void* L, int64_t ld, int n_pad, cudaStream_t stream) {
    const dim3 grid(n_pad / TB, n_pad / TB);
    if (f64)
        mirror_lower_kernel<double><<<grid, 256, 0, stream>>>(static_cast<double*>(L), ld);
    else
        mirror_lower_kernel<float><<<grid, 256, 0, stream>>>(static_cast<float*>(L), ld);
    count_launch();
    return cudaGetLastError();
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
