// Algorithm 1's Gram W = S S^T on the 5th-generation tensor cores: W = S S^T (lower triangle), the O(n^2 m)
// contraction that Section 2 of arXiv 2310.17556 names as the dominant cost.
//
// Work decomposition.  S (n x m, row-major, K = m contiguous) is cut into T = ceil(n/128) row
// blocks.  The lower triangle of W (T(T+1)/2 tiles of 128 x 128) is covered exactly once by
//   pairs   (I; J0, J0+1): one tcgen05.mma with M = 128, N = 256, A = block I, B = blocks J0, J0+1
//   singles (I; I):        M = 128, N = 128, for the diagonal tiles no pair covers.
// For even I the "diagonal pair" (I; I, I+1) computes tile (I, I) and tile (I, I+1), which is
// the transpose of the lower tile (I+1, I) (W is symmetric), so no tile is computed twice:
//   even row I: pairs J0 = 0, 2, ..., I (the last one diagonal; a single if I is the last row)
//   odd row I:  pairs J0 = 0, 2, ..., I-3, then the single (I; I)   [(I, I-1) came transposed].
// Each unit is split into `c` (singles) or `2c` (pairs) tasks of equal cost; task `slot` of a
// unit with `g` tasks takes the k-blocks slot, slot+g, slot+2g, ...  Tasks are dealt round-robin
// to a persistent grid of one CTA per SM.  Because every task advances through m at the same
// cost per k-block position, all CTAs of a round read the same few k-blocks at any moment: S
// is fetched from DRAM about once per round and the other reads hit L2.  Each task writes one
// FP32 partial block; gram_tc_finalize sums the tasks of each tile in a fixed order (FP64),
// transposes where needed and adds lambda.
//
// Per CTA (192 threads, warp-specialised):
//   warp 0     TMA producer: per 128-byte k-block, one 128-row box of A and one (single) or two
//              (pair) of B land in a 4-stage ring of 48 KB stages (128-byte swizzle).
//   warp 1     MMA issuer: 4 MMAs (K = 32 bytes each) per stage into a 128 x 256 (or 128) FP32
//              accumulator in TMEM (two accumulators, 512 columns, so the epilogue of one task
//              overlaps the MMAs of the next); tcgen05.commit releases stages and accumulators.
//   warps 2-5  epilogue: tcgen05.ld 32 columns at a time (each warp its 32-lane quarter),
//              16-byte stores of the partial block.
// Every mbarrier wait is bounded (2 s of wall time); a timeout sets DFS_ERR_TIMEOUT, makes the
// other roles stop, waits for TMA copies and MMAs in flight and frees TMEM before returning.
//
// Kinds: TF32 MMA directly on FP32 S (the tensor core takes the top 19 bits of each value),
// and BF16 MMA on BF16-stored S.
#include <cudaTypedefs.h>

#include <cstring>

#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dfs {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_ROW_BYTES = 128;
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_ROW_BYTES;
constexpr int TC_B_BYTES = TC_BN * TC_ROW_BYTES;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

struct TcSmem {
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t accf[2];
    uint64_t acce[2];
    uint64_t done;
    uint32_t tmem_base;
    int abort;
    int never;  // stays 0: the abort flag for waits that must not be cut short
};

constexpr size_t TC_SMEM_BYTES = 1024 + (size_t)TC_STAGES * TC_STAGE_BYTES + sizeof(TcSmem);

// Warp roles: warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 epilogue.
constexpr int TC_THREADS = 192;
constexpr int kMmaWarp = 1;


}  // namespace

// Units per row I of the unit enumeration (see the header comment).
__host__ __device__ __forceinline__ int tc_row_pairs(int I, int T) {
    return (I & 1) ? (I - 1) / 2 : I / 2 + ((I + 1 < T) ? 1 : 0);
}
__host__ __device__ __forceinline__ int tc_row_single(int I, int T) { return ((I & 1) || I + 1 >= T) ? 1 : 0; }

// Pairs come first (row by row, J0 ascending), then singles (row by row).
__host__ __device__ inline void tc_unit_ij(int u, int T, int& I, int& J0, int& wide) {
    int before = 0;
    for (int i = 0; i < T; ++i) {
        const int c = tc_row_pairs(i, T);
        if (u < before + c) {
            I = i;
            J0 = 2 * (u - before);
            wide = 1;
            return;
        }
        before += c;
    }
    for (int i = 0; i < T; ++i) {
        const int c = tc_row_single(i, T);
        if (u < before + c) {
            I = i;
            J0 = i;
            wide = 0;
            return;
        }
        before += c;
    }
    I = J0 = wide = 0;
}

__host__ __device__ inline void tc_counts(int T, int& P, int& Sg) {
    P = 0;
    Sg = 0;
    for (int i = 0; i < T; ++i) {
        P += tc_row_pairs(i, T);
        Sg += tc_row_single(i, T);
    }
}

// Task t -> unit, slot and stride (pairs have 2c tasks each, singles c).
struct TcTask {
    int I, J0, wide, slot, stride;
};
__host__ __device__ inline TcTask tc_task(int t, int T, int c, int P) {
    TcTask k;
    int u;
    if (t < 2 * c * P) {
        u = t / (2 * c);
        k.slot = t % (2 * c);
        k.stride = 2 * c;
    } else {
        const int t2 = t - 2 * c * P;
        u = P + t2 / c;
        k.slot = t2 % c;
        k.stride = c;
    }
    tc_unit_ij(u, T, k.I, k.J0, k.wide);
    return k;
}

__host__ __device__ __forceinline__ int tc_task_nk(const TcTask& k, int64_t nkb) {
    return k.slot < nkb ? (int)((nkb - 1 - k.slot) / k.stride + 1) : 0;
}

// KIND: 1 = TF32 MMA, 0 = BF16 MMA.  PACKED: 1 = operands from the packed 16 KB tiles written by
// the S v pass (one contiguous bulk copy per tile), 0 = TMA boxes straight from S (row-major,
// used when S has short rows and no tile copy was made).
template <int KIND, int PACKED>
__global__ void __launch_bounds__(TC_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const unsigned char* __restrict__ Sp, int T, int c, int P,
               int ntasks, int64_t nkb, int row_elems, float* __restrict__ part, DevStatus* st) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* stage_mem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcSmem* sm = reinterpret_cast<TcSmem*>(stage_mem + TC_STAGES * TC_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            tc::mbar_init(&sm->full[s], 1);
            tc::mbar_init(&sm->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&sm->accf[a], 1);
            tc::mbar_init(&sm->acce[a], 128);
        }
        tc::mbar_init(&sm->done, 1);
        sm->abort = 0;
        sm->never = 0;
        tc::fence_mbar_init();
        if (!PACKED) tc::prefetch_tmap(&tmap);
    }
    if (warp == kMmaWarp) tc::tmem_alloc(&sm->tmem_base, TC_TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm->tmem_base;
    volatile int* abort = &sm->abort;
    volatile int* never = &sm->never;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t last_parity[TC_STAGES];
            bool issued[TC_STAGES];
            for (int s = 0; s < TC_STAGES; ++s) issued[s] = false;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntasks; t += gridDim.x) {
                const TcTask tk = tc_task(t, T, c, P);
                const int nk = tc_task_nk(tk, nkb);
                for (int kt = 0; kt < nk; ++kt) {
                    if (!tc::mbar_wait_bounded(&sm->empty[stage], phase ^ 1u, abort, TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    unsigned char* a = stage_mem + stage * TC_STAGE_BYTES;
                    unsigned char* b = a + TC_A_BYTES;
                    tc::mbar_arrive_expect_tx(&sm->full[stage], tk.wide ? TC_STAGE_BYTES : 2 * TC_A_BYTES);
                    const int64_t kb = tk.slot + (int64_t)kt * tk.stride;
                    if (PACKED) {
                        tc::bulk_load(a, Sp + (((int64_t)tk.I * nkb + kb) << 14), TC_A_BYTES, &sm->full[stage]);
                        tc::bulk_load(b, Sp + (((int64_t)tk.J0 * nkb + kb) << 14), TC_A_BYTES, &sm->full[stage]);
                        if (tk.wide)
                            tc::bulk_load(b + TC_A_BYTES, Sp + (((int64_t)(tk.J0 + 1) * nkb + kb) << 14), TC_A_BYTES,
                                          &sm->full[stage]);
                    } else {
                        const int32_t x = (int32_t)(kb * row_elems);
                        tc::tma_load_2d(a, &tmap, x, tk.I * TC_BM, &sm->full[stage]);
                        tc::tma_load_2d(b, &tmap, x, tk.J0 * TC_BM, &sm->full[stage]);
                        if (tk.wide) tc::tma_load_2d(b + TC_A_BYTES, &tmap, x, tk.J0 * TC_BM + TC_BM, &sm->full[stage]);
                    }
                    issued[stage] = true;
                    last_parity[stage] = phase;
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                *abort = 1;
                set_status(st, DFS_ERR_TIMEOUT);
            }
            // Every issued copy must have landed before the CTA may exit.
            for (int s = 0; s < TC_STAGES; ++s)
                if (issued[s] && !tc::mbar_wait_bounded(&sm->full[s], last_parity[s], never, TC_WAIT_NS))
                    set_status(st, DFS_ERR_TIMEOUT);
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc_wide =
                tc::instr_desc_f32acc(KIND == 1 ? tc::kFmtTF32 : tc::kFmtBF16, TC_BM, TC_BN);
            constexpr uint32_t idesc_single =
                tc::instr_desc_f32acc(KIND == 1 ? tc::kFmtTF32 : tc::kFmtBF16, TC_BM, TC_BM);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntasks; t += gridDim.x) {
                const TcTask tk = tc_task(t, T, c, P);
                const int nk = tc_task_nk(tk, nkb);
                if (nk == 0) continue;  // the epilogue writes zeros for an empty task
                const uint32_t idesc = tk.wide ? idesc_wide : idesc_single;
                if (!tc::mbar_wait_bounded(&sm->acce[acc], acc_phase ^ 1u, abort, TC_WAIT_NS)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(acc * TC_BN);
                for (int kt = 0; kt < nk; ++kt) {
                    if (!tc::mbar_wait_bounded(&sm->full[stage], phase, abort, TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_addr = tc::smem_u32(stage_mem + stage * TC_STAGE_BYTES);
                    const uint32_t b_addr = a_addr + TC_A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_ROW_BYTES / 32; ++kk)
                        tc::mma_ss<KIND>(d, tc::sw128_kmajor_desc(a_addr + kk * 32),
                                         tc::sw128_kmajor_desc(b_addr + kk * 32), idesc, (kt | kk) != 0);
                    tc::mma_commit(&sm->empty[stage]);
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                tc::mma_commit(&sm->accf[acc]);
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (!ok) {
                *abort = 1;
                set_status(st, DFS_ERR_TIMEOUT);
            }
            // All MMAs issued by this thread must complete before TMEM is freed.
            tc::mma_commit(&sm->done);
            if (!tc::mbar_wait_bounded(&sm->done, 0, never, TC_WAIT_NS)) set_status(st, DFS_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue (the four warps after the MMA warp) ----------------
        const int q = warp & 3;  // TMEM lane quarter accessible to this warp
        const int row = q * 32 + lane;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
            const TcTask tk = tc_task(t, T, c, P);
            const int ncols = tk.wide ? TC_BN : TC_BM;
            float* dst = part + (size_t)t * (TC_BM * TC_BN) + (size_t)row * TC_BN;
            if (tc_task_nk(tk, nkb) == 0) {
                for (int j = 0; j < ncols; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            bool ok = tc::mbar_wait_bounded(&sm->accf[acc], acc_phase, abort, TC_WAIT_NS);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    *abort = 1;
                    set_status(st, DFS_ERR_TIMEOUT);
                }
                break;
            }
            tc::fence_after_sync();
            const uint32_t tbase = tmem + (uint32_t)(acc * TC_BN) + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int cc = 0; cc < ncols / 32; ++cc) {
                uint32_t v[32];
                tc::tmem_ld_32x32b_x32(tbase + (uint32_t)(cc * 32), v);
                tc::tmem_ld_wait();
                float4* d4 = reinterpret_cast<float4*>(dst + cc * 32);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    d4[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                        __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&sm->acce[acc]);
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// W[gi][gj] (lower, rows < n_out) = sum over the tasks of the unit holding tile (I, J) (FP64, in
// task order), plus lambda on the diagonal; rows/cols in [n, n_out) get the identity.  Tile
// (I, I-1) for odd I is read transposed from the diagonal pair of row I-1.  One CTA per 8 rows
// of a 128 x 128 tile; thread = (row, 4 consecutive columns).
__global__ void __launch_bounds__(256)
gram_tc_finalize_kernel(const float* __restrict__ part, int T, int c, int P, int64_t n, int64_t n_out, double lambda,
                        float* __restrict__ W, int64_t ldw) {
    int I, J;
    {
        const int t = blockIdx.x;
        int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        while (i * (i + 1) / 2 > t) --i;
        I = i;
        J = t - i * (i + 1) / 2;
    }
    const int r = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int c4 = (threadIdx.x & 31) * 4;
    const int64_t gi = (int64_t)I * TC_BM + r;
    if (gi >= n_out) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (gi < n && I < T) {
        // locate the unit, its first task and task count, the column offset, transposition
        int unit, coff = 0;
        bool transposed = false;
        int pairs_before = 0;
        for (int i = 0; i < I; ++i) pairs_before += tc_row_pairs(i, T);
        if (J == I && !tc_row_single(I, T)) {
            unit = pairs_before + I / 2;  // diagonal pair of an even row
        } else if (J == I) {
            int singles_before = 0;
            for (int i = 0; i < I; ++i) singles_before += tc_row_single(i, T);
            unit = P + singles_before;
        } else if ((I & 1) && J == I - 1) {
            int pb = 0;
            for (int i = 0; i < I - 1; ++i) pb += tc_row_pairs(i, T);
            unit = pb + (I - 1) / 2;  // diagonal pair of row I-1, second tile, transposed
            coff = TC_BM;
            transposed = true;
        } else {
            unit = pairs_before + J / 2;
            coff = (J & 1) * TC_BM;
        }
        const int g = unit < P ? 2 * c : c;
        const int t0 = unit < P ? unit * 2 * c : 2 * c * P + (unit - P) * c;
        for (int q = 0; q < g; ++q) {
            const float* blk = part + (size_t)(t0 + q) * TC_BM * TC_BN;
            if (!transposed) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(blk + (size_t)r * TC_BN + coff + c4));
                v[0] += x.x;
                v[1] += x.y;
                v[2] += x.z;
                v[3] += x.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] += __ldg(blk + (size_t)(c4 + e) * TC_BN + coff + r);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t gj = (int64_t)J * TC_BM + c4 + e;
        if (gj > gi) continue;
        double w;
        if (gi >= n || gj >= n) w = (gi == gj) ? 1.0 : 0.0;
        else w = v[e] + ((gi == gj) ? lambda : 0.0);
        W[gi * ldw + gj] = (float)w;
    }
}

// ---- host side ------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// kind 0 = BF16 MMA (FP32 S is packed to BF16 tiles, BF16 S used directly or re-laid out),
// kind 1 = TF32 MMA (FP32 S, packed to TF32 tiles or read directly).
int gram_tc_supported(int s_dtype, int kind) {
    if (kind == 1) return s_dtype == DFS_F32;
    if (kind == 0) return s_dtype == DFS_F32 || s_dtype == DFS_BF16;
    return 0;
}

// elements per 128-byte k-block row: BF16 MMA -> 64, TF32 MMA -> 32
static int tc_row_elems_kind(int kind) { return kind == 0 ? 64 : 32; }

GramTcPlan gram_tc_plan(int s_dtype, int kind, int64_t n, int64_t m, int num_sms) {
    GramTcPlan p{};
    p.kind = kind;
    // FP32 S always goes through packed tiles (BF16 needs the conversion; TF32 avoids the
    // address-translation cost of boxes spanning rows that are megabytes apart); BF16 S with
    // rows >= 1 MiB too.
    p.packed = (s_dtype == DFS_F32) || ((int64_t)m * 2 >= (1 << 20));
    p.n_tiles = (int)ceil_div(n, TC_BM);
    int P, Sg;
    tc_counts(p.n_tiles, P, Sg);
    p.npairs = P;
    const int C = 2 * P + Sg;  // cost units (a pair costs two singles)
    const int64_t nkb = ceil_div(m, tc_row_elems_kind(kind));
    // Tasks per cost unit: the smallest c that fills the grid evenly (at most 16 partial blocks
    // per tile and at least 32 k-blocks per task).
    int best_c = 1;
    double best = -1.0;
    for (int c = 1; c <= 16; ++c) {
        if (c > 1 && nkb / (2 * c) < 32) break;
        const double tasks = (double)c * C;
        const double eff = tasks / (std::ceil(tasks / num_sms) * num_sms);
        if (eff > best + 0.02) {
            best = eff;
            best_c = c;
        }
    }
    p.c = best_c;
    p.ntasks = best_c * C;
    p.nkb = nkb;
    p.partial_bytes = (size_t)p.ntasks * TC_BM * TC_BN * sizeof(float);
    return p;
}

cudaError_t launch_gram_tc(const GramTcPlan& plan, int s_dtype, const void* S, int64_t n, int64_t m, int64_t lds,
                           const void* Sp, void* P, DevStatus* st, cudaStream_t stream) {
    if (!gram_tc_supported(s_dtype, plan.kind)) return cudaErrorNotSupported;
    const int re = tc_row_elems_kind(plan.kind);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (!plan.packed) {
        auto encode = tensor_map_encoder();
        if (!encode || s_dtype != (plan.kind == 0 ? DFS_BF16 : DFS_F32)) return cudaErrorNotSupported;
        const int esz = s_dtype == DFS_BF16 ? 2 : 4;
        cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
        cuuint64_t strides[1] = {(cuuint64_t)lds * esz};
        cuuint32_t box[2] = {(cuuint32_t)re, (cuuint32_t)TC_BM};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&map, s_dtype == DFS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                            2, const_cast<void*>(S), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    } else if (Sp == nullptr) {
        return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = plan.ntasks < sms ? plan.ntasks : sms;
    const unsigned char* sp = static_cast<const unsigned char*>(Sp);
    float* part = static_cast<float*>(P);
#define DFS_TC_LAUNCH(K, PK)                                                                                        \
    {                                                                                                               \
        auto kern = gram_tc_kernel<K, PK>;                                                                          \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BYTES); \
        if (e != cudaSuccess) return e;                                                                             \
        kern<<<grid, TC_THREADS, TC_SMEM_BYTES, stream>>>(map, sp, plan.n_tiles, plan.c, plan.npairs, plan.ntasks,  \
                                                          plan.nkb, re, part, st);                                 \
        count_launch();                                                                                             \
    }
    if (plan.kind == 1) {
        if (plan.packed) DFS_TC_LAUNCH(1, 1) else DFS_TC_LAUNCH(1, 0)
    } else {
        if (plan.packed) DFS_TC_LAUNCH(0, 1) else DFS_TC_LAUNCH(0, 0)
    }
#undef DFS_TC_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_gram_tc_finalize(const GramTcPlan& plan, const void* P, int64_t n, int64_t n_out, double lambda,
                                    void* W, int64_t ldw, cudaStream_t stream) {
    const int T = (int)ceil_div(n_out, TC_BM);
    {
        gram_tc_finalize_kernel<<<dim3(T * (T + 1) / 2, TC_BM / 8), 256, 0, stream>>>(
            static_cast<const float*>(P), plan.n_tiles, plan.c, plan.npairs, n, n_out, lambda,
            static_cast<float*>(W), ldw);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace dfs
