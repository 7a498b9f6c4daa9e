// Algorithm 1's Gram W = S S^T on the 5th-generation tensor cores (lower triangle), the O(n^2 m)
// contraction that Section 2 of arXiv 2310.17556 names as the dominant cost.
//
// Work decomposition.  S (n x m, row-major, K = m contiguous) is cut into T 128-row blocks (T
// rounded up to even with zero rows), paired into T / 2 super-rows.  The lower triangle of W is
// covered by "quad units" (I2; J2), J2 <= I2, each two tcgen05.mma chains that share their B
// operand:  A0 = block 2 I2, A1 = block 2 I2 + 1, B = blocks 2 J2, 2 J2 + 1 (on the diagonal B is
// [A0 | A1] itself, read from the A tiles), D0 = A0 B^T and D1 = A1 B^T (M = 128, N = 256 each).
// On the diagonal the tile (2 I2, 2 I2 + 1) of D0 lies above the diagonal and is not stored: every
// unit then costs the same per k-step (4 tile products), so all tasks run at one rate.
// One k-step stages A0, A1, B0, B1 (64 KB; 32 KB on the diagonal) for 8.4 MFLOP.
// Every unit has the same c tasks; task (unit, slot) takes the k-blocks slot, slot + c, slot + 2c,
// ...  A CTA runs a group of G consecutive slots of one unit and adds them into one FP32 partial
// block (256 x 256: rows 0..127 from A0, 128..255 from A1).  Groups are numbered slot-group
// major, gi = (slot / G) U + unit, and dealt round-robin to a persistent grid of at most one CTA
// per SM: the CTAs of one wave hold every unit of a few slot groups, advance through m together,
// and so touch a window of at most c k-blocks at a time; each operand tile is fetched from DRAM
// about once and re-read from L2 by the other units that need it.  (A unit-major order would
// sweep m once per unit in a wave and re-read every tile from DRAM several times.)
// gram_tc_finalize sums the c / G partial blocks of each tile in group order and adds lambda.
// Per CTA (192 threads, warp-specialised):
//   warp 0     producer: per 128-byte k-block, the unit's 128-row tiles land in a 3-stage ring of
//              64 KB stages (bulk copies of the packed tiles, or TMA boxes of S, 128-byte swizzle).
//   warp 1     MMA issuer: per stage 4 + 4 MMAs (K = 32 bytes each) into two 128 x 256 FP32
//              accumulators in TMEM (all 512 columns); tcgen05.commit releases stages and, at the
//              end of a task, the accumulators.
//   warps 2-5  epilogue: tcgen05.ld 32 columns at a time (each warp its 32-lane quarter),
//              16-byte stores of the partial block.
// Every mbarrier wait is bounded (2 s of wall time); a timeout sets DFS_ERR_TIMEOUT, makes the
// other roles stop, waits for TMA copies and MMAs in flight and frees TMEM before returning.
//
// Kinds: BF16 MMA (kind::f16) on BF16 tiles, TF32 MMA (kind::tf32) on FP32 / TF32 tiles, and
// FP8: S scaled per row by a power of two r_i (so that max_j |s_ij| / r_i <= 448, exact) and
// rounded to e4m3 (round to nearest even) by the S v pass; kind::f8f6f4 MMAs on 128-column
// k-blocks; the finalize multiplies by r_i r_k (exact) before adding lambda.
// BF16x3: FP32 S split as S = H + L (H = bf16(S), L = bf16(S - H), both round to nearest even), so
// S S^T = H H^T + L H^T + (L H^T)^T + L L^T; the last term (relative size 2^-16) is dropped.  The
// packed operand is the stacked 2 T_h-block matrix Z = [H; L] (T_h = T rounded up to even, so no
// super-row mixes H and L blocks) and the kernel runs the units of Gram(Z) with J2 < H2 = T_h / 2:
// the H H^T triangle and the full L H^T rectangle (3 of the 4 quarters of Z Z^T, the work of three
// BF16 Grams); gram_tc_finalize_x3 forms W = H H^T + L H^T + (L H^T)^T.
#define DFS_SRC_ID 3
#include <cudaTypedefs.h>

#include <cstring>

#include <algorithm>
#include <cmath>

#include "gram_tc.cuh"

namespace dfs {

// KIND: 1 = TF32 MMA, 0 = BF16 MMA, 2 = FP8 (e4m3) MMA.  PACKED: 1 = operands from the packed 16 KB tiles written by
// the S v pass (one contiguous bulk copy per tile), 0 = TMA boxes straight from S (row-major,
// used when S has short rows and no tile copy was made).
template <int KIND, int PACKED>
__global__ void __launch_bounds__(TC_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const unsigned char* __restrict__ Sp, int T, int H2, int U,
               int c, int G, int64_t nkb, int row_elems, float* __restrict__ part, DevStatus* st) {
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
        tc::mbar_init(&sm->accf, 1);
        tc::mbar_init(&sm->acce, 128);
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
    const uint64_t wait_ns = wait_limit(st);

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t last_parity[TC_STAGES];
            bool issued[TC_STAGES];
            for (int s = 0; s < TC_STAGES; ++s) issued[s] = false;
            bool ok = true;
            const int ngroups = U * (c / G);
            for (int t = 0, gi = blockIdx.x; ok && gi < ngroups; t = (t + 1 == G ? 0 : t + 1), gi += (t == 0 ? gridDim.x : 0)) {
                const TcTask tk = tc_task(gi, t, U, c, G, H2);
                const int nk = tc_task_nk(tk, nkb);
                const int i0 = 2 * tk.I2, j0 = 2 * tk.J2;
                const bool diag = tk.J2 == tk.I2;
                // tiles: A0, A1, and for off-diagonal units B0, B1
                const uint32_t bytes = (uint32_t)TC_TILE_BYTES * (diag ? 2u : 4u);
                for (int kt = 0; kt < nk; ++kt) {
                    if (!tc::mbar_wait_bounded(&sm->empty[stage], phase ^ 1u, abort, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const int64_t kb = tk.slot + (int64_t)kt * tk.stride;
                    if (!DFS_IN_BOUNDS(st, kb < nkb && i0 + 1 < T && (diag || j0 + 1 < T))) {
                        *abort = 1;
                        ok = false;
                        break;
                    }
                    unsigned char* a = stage_mem + stage * TC_STAGE_BYTES;
                    unsigned char* b = a + 2 * TC_TILE_BYTES;
                    tc::mbar_arrive_expect_tx(&sm->full[stage], bytes);
                    if (PACKED) {
                        tc::bulk_load(a, Sp + ((kb * T + i0) << 14), TC_TILE_BYTES, &sm->full[stage]);
                        tc::bulk_load(a + TC_TILE_BYTES, Sp + ((kb * T + i0 + 1) << 14), TC_TILE_BYTES,
                                      &sm->full[stage]);
                        if (!diag) {
                            tc::bulk_load(b, Sp + ((kb * T + j0) << 14), TC_TILE_BYTES, &sm->full[stage]);
                            tc::bulk_load(b + TC_TILE_BYTES, Sp + ((kb * T + j0 + 1) << 14), TC_TILE_BYTES,
                                          &sm->full[stage]);
                        }
                    } else {
                        const int32_t x = (int32_t)(kb * row_elems);
                        tc::tma_load_2d(a, &tmap, x, i0 * TC_BM, &sm->full[stage]);
                        tc::tma_load_2d(a + TC_TILE_BYTES, &tmap, x, (i0 + 1) * TC_BM, &sm->full[stage]);
                        if (!diag) {
                            tc::tma_load_2d(b, &tmap, x, j0 * TC_BM, &sm->full[stage]);
                            tc::tma_load_2d(b + TC_TILE_BYTES, &tmap, x, (j0 + 1) * TC_BM, &sm->full[stage]);
                        }
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
                if (issued[s] && !tc::mbar_wait_bounded(&sm->full[s], last_parity[s], never, kDefaultWaitNs))
                    set_status(st, DFS_ERR_TIMEOUT);
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t fmt = KIND == 1 ? tc::kFmtTF32 : (KIND == 2 ? tc::kFmtE4M3 : tc::kFmtBF16);
            constexpr uint32_t idesc_wide = tc::instr_desc_f32acc(fmt, TC_BM, TC_BN);
            int stage = 0;
            uint32_t phase = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            const int ngroups = U * (c / G);
            for (int t = 0, gi = blockIdx.x; ok && gi < ngroups; t = (t + 1 == G ? 0 : t + 1), gi += (t == 0 ? gridDim.x : 0)) {
                const TcTask tk = tc_task(gi, t, U, c, G, H2);
                const int nk = tc_task_nk(tk, nkb);
                if (nk == 0) continue;  // the epilogue writes zeros for an empty task
                const bool diag = tk.J2 == tk.I2;
                // the accumulators are free once the epilogue has read the previous task's
                if (!tc::mbar_wait_bounded(&sm->acce, acc_phase ^ 1u, abort, wait_ns)) {
                    ok = false;
                    break;
                }
                acc_phase ^= 1u;
                tc::fence_after_sync();
                for (int kt = 0; kt < nk; ++kt) {
                    if (!tc::mbar_wait_bounded(&sm->full[stage], phase, abort, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(stage_mem + stage * TC_STAGE_BYTES);
                    const uint32_t a1a = a0 + TC_TILE_BYTES;
                    const uint32_t bb = diag ? a0 : a0 + 2 * TC_TILE_BYTES;  // diagonal: B = [A0 | A1]
#pragma unroll
                    for (int kk = 0; kk < TC_ROW_BYTES / 32; ++kk)
                        tc::mma_ss<KIND>(tmem, tc::sw128_kmajor_desc(a0 + kk * 32), tc::sw128_kmajor_desc(bb + kk * 32),
                                         idesc_wide, (kt | kk) != 0);
#pragma unroll
                    for (int kk = 0; kk < TC_ROW_BYTES / 32; ++kk)
                        tc::mma_ss<KIND>(tmem + (uint32_t)TC_BN, tc::sw128_kmajor_desc(a1a + kk * 32),
                                         tc::sw128_kmajor_desc(bb + kk * 32), idesc_wide, (kt | kk) != 0);
                    tc::mma_commit(&sm->empty[stage]);
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                tc::mma_commit(&sm->accf);
            }
            if (!ok) {
                *abort = 1;
                set_status(st, DFS_ERR_TIMEOUT);
            }
            // All MMAs issued by this thread must complete before TMEM is freed.
            tc::mma_commit(&sm->done);
            if (!tc::mbar_wait_bounded(&sm->done, 0, never, kDefaultWaitNs)) set_status(st, DFS_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue (the four warps after the MMA warp) ----------------
        const int q = warp & 3;  // TMEM lane quarter accessible to this warp
        const int row = q * 32 + lane;
        uint32_t acc_phase = 0;
        const int ngroups = U * (c / G);
        for (int t = 0, gi = blockIdx.x; gi < ngroups; t = (t + 1 == G ? 0 : t + 1), gi += (t == 0 ? gridDim.x : 0)) {
            const TcTask tk = tc_task(gi, t, U, c, G, H2);
            const bool diag = tk.J2 == tk.I2;
            // the group's tasks (separate FP32 accumulation chains) are added into one partial
            // block in task order: the first stores, the others add (read-modify-write)
            const bool first = (t == 0);
            float* blk = part + (size_t)gi * TC_PART;
            if (tc_task_nk(tk, nkb) == 0) {
                if (first)
                    for (int h = 0; h < 2; ++h)
                        for (int j = 0; j < TC_BN; j += 4)
                            *reinterpret_cast<float4*>(blk + (size_t)(h * TC_BM + row) * TC_BN + j) =
                                make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            bool ok = tc::mbar_wait_bounded(&sm->accf, acc_phase, abort, wait_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    *abort = 1;
                    set_status(st, DFS_ERR_TIMEOUT);
                }
                break;
            }
            acc_phase ^= 1u;
            tc::fence_after_sync();
            for (int h = 0; h < 2; ++h) {
                const int ncols = (h == 0 && diag) ? TC_BM : TC_BN;  // D0's right half lies above the diagonal
                const uint32_t tbase = tmem + (uint32_t)(h * TC_BN) + ((uint32_t)(q * 32) << 16);
                float* dst = blk + (size_t)(h * TC_BM + row) * TC_BN;
#pragma unroll 1
                for (int cc = 0; cc < ncols / 32; ++cc) {
                    uint32_t v[32];
                    tc::tmem_ld_32x32b_x32(tbase + (uint32_t)(cc * 32), v);
                    tc::tmem_ld_wait();
                    float4* d4 = reinterpret_cast<float4*>(dst + cc * 32);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float4 o = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                               __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
                        if (!first) {
                            const float4 p = d4[j];
                            o.x += p.x;
                            o.y += p.y;
                            o.z += p.z;
                            o.w += p.w;
                        }
                        d4[j] = o;
                    }
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&sm->acce);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// W[gi][gj] (lower, rows < n_out) = sum over the task groups of the unit holding tile (I, J) (FP32,
// in group order), plus lambda on the diagonal; rows/cols in [n, n_out) get the identity.  Tile (I, J)
// is block (I mod 2, J mod 2) of unit (I / 2, J / 2).  One CTA per 8 rows of a 128 x 128 tile;
// thread = (row, 4 consecutive columns).
__global__ void __launch_bounds__(256)
gram_tc_finalize_kernel(const float* __restrict__ part, int U, int c, int G, int64_t n, int64_t n_out, double lambda,
                        float* __restrict__ W, int64_t ldw, const float* __restrict__ rscale) {
    constexpr int H2 = 0;
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
    // FP32 sum of the FP32 partial blocks in block order: each block already carries FP32
    // accumulation error of a few 1e-6 to 1e-5, adding a handful of them in FP32 changes nothing
    // measurable, and FP64 adds are too slow on GB300 to be worth it here
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (gi < n) {
        const int I2 = I / 2, J2 = J / 2;
        const int u = tc_unit_index(I2, J2, H2);
        const int g = c / G;  // partial blocks (task groups) of the unit: u, u + U, u + 2U, ...
        const size_t off = (size_t)((I & 1) * TC_BM + r) * TC_BN + (J & 1) * TC_BM + c4;
        const float* p0 = part + (size_t)u * TC_PART + off;
        const size_t gstride = (size_t)U * TC_PART;
        int q = 0;
        for (; q + 4 <= g; q += 4) {  // four loads in flight, added in block order
            float4 x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = __ldg(reinterpret_cast<const float4*>(p0 + (size_t)(q + e) * gstride));
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                v[0] += x[e].x;
                v[1] += x[e].y;
                v[2] += x[e].z;
                v[3] += x[e].w;
            }
        }
        for (; q < g; ++q) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(p0 + (size_t)q * gstride));
            v[0] += x.x;
            v[1] += x.y;
            v[2] += x.z;
            v[3] += x.w;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t gj = (int64_t)J * TC_BM + c4 + e;
        if (gj > gi) continue;
        float w;
        if (gi >= n || gj >= n) w = (gi == gj) ? 1.f : 0.f;
        else w = (rscale ? v[e] * (rscale[gi] * rscale[gj]) : v[e]) + ((gi == gj) ? (float)lambda : 0.f);
        W[gi * ldw + gj] = w;
    }
}

// FP32 sum, in group order, of the partial blocks of unit (I2, J2) at offset `off` of each block.
__device__ __forceinline__ float4 tc_sum_groups(const float* __restrict__ part, int I2, int J2, int U, int H2, int c,
                                                int G, size_t off) {
    const int g = c / G;
    const float* p0 = part + (size_t)tc_unit_index(I2, J2, H2) * TC_PART + off;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < g; ++q) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p0 + (size_t)q * U * TC_PART));
        v.x += x.x;
        v.y += x.y;
        v.z += x.z;
        v.w += x.w;
    }
    return v;
}

// BF16x3 finalize: W[gi][gj] (lower, rows < n_out) = (H H^T)[gi][gj] + (L H^T)[gi][gj] + (L H^T)[gj][gi]
// plus lambda on the diagonal, from the partial blocks of the stacked Gram (Z block b = H block b,
// Z block T_h + b = L block b); rows/cols in [n, n_out) get the identity.  One CTA per 32 rows of a
// 128 x 128 tile (I, J): the transposed term (128 x 32 of Z tile (T_h + J, I)) is summed into
// shared memory first, then thread (row, 4 x 4 columns) adds the two direct terms.
__global__ void __launch_bounds__(256)
gram_tc_finalize_x3_kernel(const float* __restrict__ part, int U, int H2, int c, int G, int64_t n, int64_t n_out,
                           double lambda, float* __restrict__ W, int64_t ldw) {
    __shared__ float sT[TC_BM][33];
    int I, J;
    {
        const int t = blockIdx.x;
        int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        while (i * (i + 1) / 2 > t) --i;
        I = i;
        J = t - i * (i + 1) / 2;
    }
    const int Th = 2 * H2;
    const int r0 = blockIdx.y * 32;
    const int tid = threadIdx.x;
    const bool live = (int64_t)I * TC_BM < n;  // tiles entirely in the padding only get the identity
    // (L H^T)[k][i] for k in tile J (128 rows), i in rows r0..r0+31 of tile I
    for (int e = tid; e < TC_BM * 8; e += 256) {
        const int kk = e >> 3, i4 = (e & 7) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live) {
            const int I2 = (Th + J) / 2, J2 = I / 2;
            const size_t off = (size_t)((J & 1) * TC_BM + kk) * TC_BN + (I & 1) * TC_BM + r0 + i4;
            v = tc_sum_groups(part, I2, J2, U, H2, c, G, off);
        }
        sT[kk][i4] = v.x;
        sT[kk][i4 + 1] = v.y;
        sT[kk][i4 + 2] = v.z;
        sT[kk][i4 + 3] = v.w;
    }
    __syncthreads();
    const int rr = tid >> 3;
    const int64_t gi = (int64_t)I * TC_BM + r0 + rr;
    if (gi >= n_out) return;
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
        const int cc = (tid & 7) * 4 + 32 * u;
        float4 hh = make_float4(0.f, 0.f, 0.f, 0.f), lh = hh;
        if (live && gi < n) {
            const size_t off = (size_t)((I & 1) * TC_BM + r0 + rr) * TC_BN + (J & 1) * TC_BM + cc;
            hh = tc_sum_groups(part, I / 2, J / 2, U, H2, c, G, off);
            lh = tc_sum_groups(part, (Th + I) / 2, J / 2, U, H2, c, G, off);
        }
        const float a[4] = {hh.x + lh.x, hh.y + lh.y, hh.z + lh.z, hh.w + lh.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t gj = (int64_t)J * TC_BM + cc + e;
            if (gj > gi) continue;
            float w;
            if (gi >= n || gj >= n) w = (gi == gj) ? 1.f : 0.f;
            else w = (a[e] + sT[cc + e][rr]) + ((gi == gj) ? (float)lambda : 0.f);
            W[gi * ldw + gj] = w;
        }
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
// kind 1 = TF32 MMA (FP32 S, packed to TF32 tiles or read directly),
// kind 2 = BF16x3 (FP32 S packed to stacked H / L BF16 tiles),
// kind 3 = FP8 (FP32 or BF16 S packed to row-scaled e4m3 tiles).
int gram_tc_supported(int s_dtype, int kind) {
    if (kind == 1 || kind == 2) return s_dtype == DFS_F32;
    if (kind == 3) return s_dtype == DFS_F32 || s_dtype == DFS_BF16;
    if (kind == 0) return s_dtype == DFS_F32 || s_dtype == DFS_BF16;
    return 0;
}

// elements per 128-byte k-block row: BF16 MMA -> 64, TF32 MMA -> 32
static int tc_row_elems_kind(int kind) { return kind == 1 ? 32 : (kind == 3 ? 128 : 64); }

GramTcPlan gram_tc_plan(int s_dtype, int kind, int64_t n, int64_t m, int num_sms) {
    GramTcPlan p{};
    p.kind = kind;
    // FP32 S always goes through packed tiles (BF16 needs the conversion; TF32 avoids the
    // address-translation cost of boxes spanning rows that are megabytes apart); BF16 S with
    // rows >= 1 MiB too.
    p.packed = (s_dtype == DFS_F32) || ((int64_t)m * 2 >= (1 << 20)) || kind == 3;
    p.n_tiles = (int)round_up(ceil_div(n, TC_BM), 2);  // even: every super-row has A0 and A1
    p.h2 = 0;
    if (kind == 2) {  // stacked [H; L]: T_h = T rounded up to even blocks of each
        p.h2 = p.n_tiles / 2;
        p.n_tiles = 4 * p.h2;
    }
    const int U = tc_num_units(p.n_tiles, p.h2);
    p.npairs = U;
    const int64_t nkb = ceil_div(m, tc_row_elems_kind(kind));
    // Slot groups per unit w = c / G: the smallest w whose U w groups fill waves of num_sms CTAs to
    // >= 95 % (else the best w up to 64).  Then G, the tasks per group, is the smallest that keeps
    // each task's FP32 accumulation chain (nkb / c k-blocks) at most 1024 k-blocks long.
    int best_w = 1;
    double best = -1.0;
    for (int w = 1; w <= 64; ++w) {
        if ((int64_t)w > nkb) break;
        const double groups = (double)U * w;
        const double eff = groups / (std::ceil(groups / num_sms) * num_sms);
        if (eff > best + 1e-9) {
            best = eff;
            best_w = w;
        }
        if (eff >= 0.95) break;
    }
    int G = 1;
    while ((int64_t)best_w * G * 1024 < nkb) ++G;
    p.c = best_w * G;
    p.group = G;
    p.ntasks = U * p.c;
    p.nkb = nkb;
    p.partial_bytes = (size_t)(U * best_w) * TC_PART * sizeof(float);
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
    const int ngroups = plan.npairs * (plan.c / plan.group);
    const int grid = ngroups < sms ? ngroups : sms;
    const unsigned char* sp = static_cast<const unsigned char*>(Sp);
    float* part = static_cast<float*>(P);
#define DFS_TC_LAUNCH(K, PK)                                                                                        \
    {                                                                                                               \
        auto kern = gram_tc_kernel<K, PK>;                                                                          \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BYTES); \
        if (e != cudaSuccess) return e;                                                                             \
        kern<<<grid, TC_THREADS, TC_SMEM_BYTES, stream>>>(map, sp, plan.n_tiles, plan.h2, plan.npairs, plan.c,       \
                                                          plan.group, plan.nkb, re, part, st);                     \
        count_launch();                                                                                             \
    }
    if (plan.kind == 3) {
        if (!plan.packed) return cudaErrorNotSupported;
        DFS_TC_LAUNCH(2, 1)
    } else if (plan.kind == 1) {
        if (plan.packed) DFS_TC_LAUNCH(1, 1) else DFS_TC_LAUNCH(1, 0)
    } else {
        if (plan.packed) DFS_TC_LAUNCH(0, 1) else DFS_TC_LAUNCH(0, 0)
    }
#undef DFS_TC_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_gram_tc_finalize(const GramTcPlan& plan, const void* P, int64_t n, int64_t n_out, double lambda,
                                    void* W, int64_t ldw, cudaStream_t stream, const float* rscale) {
    const int T = (int)ceil_div(n_out, TC_BM);
    if (plan.kind == 2) {
        gram_tc_finalize_x3_kernel<<<dim3(T * (T + 1) / 2, TC_BM / 32), 256, 0, stream>>>(
            static_cast<const float*>(P), plan.npairs, plan.h2, plan.c, plan.group, n, n_out, lambda,
            static_cast<float*>(W), ldw);
        count_launch();
    } else {
        gram_tc_finalize_kernel<<<dim3(T * (T + 1) / 2, TC_BM / 8), 256, 0, stream>>>(
            static_cast<const float*>(P), plan.npairs, plan.c, plan.group, n, n_out, lambda,
            static_cast<float*>(W), ldw, rscale);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace dfs
