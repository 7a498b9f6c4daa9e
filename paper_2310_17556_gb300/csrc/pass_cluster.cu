// The fused refinement pass of pass.cu (U = V - S^T Y, X = U / lambda, R = S U - lambda Y in one
// read of S) for FP32 S with n <= 4096, as thread-block clusters.
//
// Reading S in strips of all n rows x 128 bytes (one CTA per strip) tops out near 4.8 TB/s on
// GB300: every 128 KB strip touches n rows megabytes apart.  Row segments of >= 256 bytes with
// <= 512 rows per CTA reach the copy rate, so here a cluster of cs = ceil(n / RC) CTAs shares
// one strip of 64 columns (256 bytes per row): CTA `rank` owns rows [rank RC, rank RC + RC)
// (RC = 32 RPT), keeps its RC x 64 slice in registers (16 lanes x 16 bytes per row, RPT rows per
// thread) and stages the next strips' slices (about 128 KB) in shared memory with cp.async
// meanwhile.
// Per strip:
//   phase 1  column sums of S^T Y over the CTA's rows (shuffle + shared memory), written to every
//            CTA of the cluster with asynchronous 16-byte remote stores that complete the
//            transaction count of the receiver's mbarrier (no fence, so the next strip's loads stay
//            in flight), then each CTA forms U = V - sum over ranks in rank order (so all ranks
//            hold identical U);
//            rank r writes X (and the stopping-rule sums) for columns c with floor(c cs / 64) = r;
//   phase 2  per-row dot products with U into FP32 row sums, folded into FP64 every 32 strips.
// The multiply-adds of both phases run as pairs (__ffma2_rn: two IEEE fmaf results per
// instruction, the same values as scalar code).
// Partials are per cluster: Rpart[c] holds all n rows (each rank its own rows), U2part[c] the
// per-RHS sums (combined over ranks through rank 0).  The exchange buffers and their mbarriers are
// double-buffered by strip parity: a rank sends strip s + 2's partials (same parity as s) only
// after it has received strip s + 1's from every rank, which each rank sends only after its own
// reads of strip s's buffer, so no buffer is overwritten while it is read.
#define DFS_SRC_ID 1
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dfs {

constexpr int CL_THREADS = 512;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int CL_LPR = 16;               // lanes per row
constexpr int CL_W = CL_LPR * 4;         // strip width (FP32 columns)
constexpr int CL_SWEEP = CL_THREADS / CL_LPR;  // 32 rows per sweep
constexpr int CL_MAX_CS = 8;
constexpr int CL_FOLD = 32;
constexpr bool kPreferLaneAcc = true;  // see cluster_rpt

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store a float / double into the shared memory of CTA `rank` of the cluster at the address
// that `local` has in this CTA
__device__ __forceinline__ void st_cluster_f32(const void* local, uint32_t rank, float v) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(r), "f"(v) : "memory");
}
// Asynchronous remote store of 16 bytes (4 floats at a 16-byte aligned `local`) into CTA `rank`'s
// copy of `local`, completing 16 bytes of the transaction count of that CTA's copy of mbarrier
// `bar`.
__device__ __forceinline__ void st_async_v4(const void* local, const uint64_t* bar, uint32_t rank, float4 v) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), b = static_cast<uint32_t>(
                 __cvta_generic_to_shared(bar)), ra, rb;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(b), "r"(rank));
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(ra),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w)), "r"(rb)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_f64(const void* local, uint32_t rank, double v) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(r), "d"(v) : "memory");
}

// Paired FP32 fused multiply-add: two IEEE fmaf results (round to nearest) in one instruction.
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2dup(float a) { return make_float2(a, a); }

// Shared-memory layouts, chosen so that every access below is contiguous across the lanes that
// make it (no bank conflicts) and 16 bytes wide where a lane moves several values:
//   Ys    [row][q][2]        each y twice, the pair operand of phase 1's paired multiply-adds
//   ured  [warp][q][col]     phase 1's per-warp column sums (float4 stores of 4 columns)
//   pbuf  [par][rank][q][col] the ranks' column sums
//   us    u_{col,q} for phase 2: KQ >= 2 as [q / 2][col % 4 / 2][col / 4][col % 2][q % 2], so a lane
//         reads the (q, q + 1) pairs of its 4 columns as two float4 loads; KQ = 1 as [col]
template <int KQ>
__device__ __forceinline__ int us_index(int c, int q) {
    if constexpr (KQ >= 2)
        return ((((q >> 1) * 2 + ((c & 3) >> 1)) * (CL_W / 4) + (c >> 2)) * 2 + (c & 1)) * 2 + (q & 1);
    else
        return c;
}

// Shared memory of a CTA beyond its stage ring (row sums, y, the exchange buffers, u).
constexpr size_t cl_rest_bytes(int rpt, int kq) {
    return (size_t)rpt * CL_SWEEP * kq * (8 + 4 + 8) + (size_t)CL_WARPS * CL_W * kq * 4 +
           (size_t)2 * CL_MAX_CS * CL_W * kq * 4 + (size_t)CL_W * kq * 4;
}
// Strips in flight in the stage ring: about 128 KB of S per CTA (HBM latency x the SM's share of
// the bandwidth is ~66 KB), as far as shared memory allows.
constexpr int cl_depth(int rpt, int kq) {
    const size_t strip = (size_t)rpt * CL_THREADS * 16;
    int d = (int)(131072 / strip);
    d = d > 4 ? 4 : (d < 1 ? 1 : d);
    while (d > 1 && d * strip + cl_rest_bytes(rpt, kq) > 220 * 1024) d >>= 1;
    return d;
}

template <int KQ, int RPT>
__global__ void __launch_bounds__(CL_THREADS, 1)
fisher_pass_cluster_kernel(const float* __restrict__ S, int n, int64_t m, int64_t lds, const float* __restrict__ V,
                           int64_t ldv, int k, const double* __restrict__ Y, int64_t ldy, double lambda,
                           float* __restrict__ X, int64_t ldx, double* __restrict__ Rpart,
                           double* __restrict__ U2part, int dmode, const DevStatus* st, int honor_stop) {
    constexpr int RC = RPT * CL_SWEEP;  // rows per CTA
    constexpr int KP = KQ >= 2 ? KQ / 2 : 1;  // right-hand-side pairs of phase 2
    constexpr int DEPTH = cl_depth(RPT, KQ);  // strips of the stage ring
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* stage = reinterpret_cast<uint4*>(smem);  // DEPTH x RPT x 512 x 16 B
    double* Rs64 = reinterpret_cast<double*>(smem + (size_t)DEPTH * RPT * CL_THREADS * 16);  // RC x KQ
    float* Rs32 = reinterpret_cast<float*>(Rs64 + RC * KQ);                         // RC x KQ
    float* Ys = Rs32 + RC * KQ;                                                      // RC x KQ x 2
    float* ured = Ys + RC * KQ * 2;                                                  // warps x KQ x W
    float* pbuf = ured + CL_WARPS * KQ * CL_W;                                       // 2 x MAX_CS x KQ x W
    float* us = pbuf + 2 * CL_MAX_CS * KQ * CL_W;                                    // W x KQ
    __shared__ double u2s[CL_WARPS][2];
    __shared__ double u2c[CL_MAX_CS][16];
    __shared__ __align__(8) uint64_t xbar[2];  // partials from the other ranks landed (by parity)
    __shared__ int s_abort;

    // every CTA of the launch reads the same status (only earlier launches on this stream
    // write it), so the early exit is cluster-uniform
    if (block_should_exit(st, honor_stop)) return;
    // the call's wait limit and test hook, read once (not in the strip loop)
    const uint64_t wait_ns = wait_limit(st);
    const int fault = test_fault(st);
    const uint32_t cs = cl_size(), rank = cl_rank();
    const int64_t cid = blockIdx.x / cs, ncl = gridDim.x / cs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rr = lane / CL_LPR, cq = lane % CL_LPR;
    const int r0 = (int)rank * RC;
    const bool haveY = (Y != nullptr);
    const bool wantR = (Rpart != nullptr);
    const float inv_lambda = (float)(1.0 / lambda);
    for (int e = tid; e < RC * KQ; e += CL_THREADS) {
        const int i = r0 + e / KQ, q = e % KQ;
        Rs64[e] = 0.0;
        Rs32[e] = 0.f;
        const float y = (haveY && i < n && q < k && DFS_IN_BOUNDS(st, q < ldy)) ? (float)Y[(int64_t)i * ldy + q] : 0.f;
        Ys[2 * e] = y;
        Ys[2 * e + 1] = y;
    }
    const int64_t nstrips = ceil_div(m, CL_W);
    const int lrow0 = warp * 2 + rr;  // local row of t = 0
    // A strip's rows arrive in NSUB sub-stages (rows t in [j RPT/NSUB, (j+1) RPT/NSUB) of every
    // thread) in ring slot g mod DEPTH (g: the CTA's strip count); sub-stage j of a slot is
    // refilled with strip g + DEPTH's as soon as this thread has moved it into registers (each
    // thread copies and reads only its own 16-byte pieces, so no barrier), so about DEPTH strips
    // stay in flight at all times.
    constexpr int NSUB = RPT >= 4 ? 4 : RPT;
    constexpr int TPS = RPT / NSUB;  // rows per thread per sub-stage
    auto issue_sub = [&](int64_t sidx, int64_t g, int j) {
        if (sidx < nstrips) {
            const int64_t jn = sidx * CL_W + cq * 4;
            const int64_t rem = m - jn;
            const int bytes_col = rem >= 4 ? 16 : (rem > 0 ? (int)rem * 4 : 0);
            uint4* slot = stage + (size_t)(g % DEPTH) * RPT * CL_THREADS;
#pragma unroll
            for (int tt = 0; tt < TPS; ++tt) {
                const int t = j * TPS + tt;
                const int i = r0 + lrow0 + t * CL_SWEEP;
                int bytes = i < n ? bytes_col : 0;
                if (bytes && !DFS_IN_BOUNDS(st, jn + bytes / 4 <= m && jn + bytes / 4 <= lds)) bytes = 0;
                const float* src = bytes ? S + (int64_t)i * lds + jn : S;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                 static_cast<uint32_t>(__cvta_generic_to_shared(&slot[t * CL_THREADS + tid]))),
                             "l"(src), "r"(bytes)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");  // (empty past the last strip)
    };
#pragma unroll
    for (int d = 0; d < DEPTH; ++d)
#pragma unroll
        for (int j = 0; j < NSUB; ++j) issue_sub(cid + d * ncl, d, j);
    // A thread of the first KQ x 64 forms u for column uc and right-hand side uq of every strip
    // (a warp: 32 consecutive columns of one right-hand side), and keeps that RHS's stopping-rule
    // sums.
    const bool u_thread = tid < CL_W * KQ;
    const int uc = tid % CL_W, uq = tid / CL_W;
    const bool writer = u_thread && (uc * (int)cs) / CL_W == (int)rank;  // ranks split the columns
    const int us_at = us_index<KQ>(uc, uq);
    float u2f = 0.f, d2f = 0.f;
    double u2 = 0.0, d2 = 0.0;
    if (tid == 0) {
        tc::mbar_init(&xbar[0], 1);
        tc::mbar_init(&xbar[1], 1);
        tc::fence_mbar_init();
        s_abort = 0;
    }
    const uint32_t xbytes = (cs - 1) * CL_W * KQ * 4;  // partial bytes received per strip
    uint32_t xphase = 0;                              // bit p: phase parity of xbar[p]
    __syncthreads();
    cl_sync();  // every CTA of the cluster is running (and its barriers initialised) before any remote store

    // Phase 2's row sums: with few rows and right-hand sides a lane keeps its own partial sums
    // (its 4 columns of every strip) in registers, as (q, q + 1) pairs, and the 16 lanes of a row
    // are added only at each fold, in place of 4 shuffles per row and right-hand side on every
    // strip.
    constexpr bool kLaneAcc = RPT * KQ <= 32;
    constexpr int LR = kLaneAcc ? RPT : 1, LP = kLaneAcc ? KP : 1;
    float2 racc[LR][LP];
#pragma unroll
    for (int t = 0; t < LR; ++t)
#pragma unroll
        for (int p = 0; p < LP; ++p) racc[t][p] = make_float2(0.f, 0.f);
    auto fold_lanes = [&]() {
#pragma unroll
        for (int t = 0; t < LR; ++t) {
            const int li = lrow0 + t * CL_SWEEP;
#pragma unroll
            for (int p = 0; p < LP; ++p) {
                float a = racc[t][p].x, b = racc[t][p].y;
#pragma unroll
                for (int o = 1; o < CL_LPR; o <<= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    if constexpr (KQ >= 2) b += __shfl_xor_sync(0xffffffffu, b, o);
                }
                if (cq == 0) {
                    Rs64[li * KQ + (KQ >= 2 ? 2 * p : 0)] += (double)a;
                    if constexpr (KQ >= 2) Rs64[li * KQ + 2 * p + 1] += (double)b;
                }
                racc[t][p] = make_float2(0.f, 0.f);
            }
        }
    };
    int since_fold = 0, par = 0;
    int64_t g = 0;  // strips of this CTA so far
    for (int64_t s = cid; s < nstrips; s += ncl, par ^= 1, ++g) {
        const int64_t j0 = s * CL_W;
        float sv[RPT][4];
        float v_pre = 0.f, x_pre = 0.f;
        const bool u_valid = u_thread && (j0 + uc < m) && (uq < k) &&
                             DFS_IN_BOUNDS(st, j0 + uc < ldv && (X == nullptr || j0 + uc < ldx));
        if (u_valid) {
            v_pre = V[(int64_t)uq * ldv + j0 + uc];
            if (writer && X != nullptr && dmode == 1) x_pre = X[(int64_t)uq * ldx + j0 + uc];
        }
        // ---- phase 1: this CTA's column sums of S^T Y -> every rank's pbuf[par][rank] ----
        const bool exch = haveY && cs > 1;
        if (exch && tid == 0 && !s_abort) tc::mbar_arrive_expect_tx(&xbar[par], xbytes);
        float2 acc[KQ][2];  // columns (0, 1) and (2, 3) of this lane
#pragma unroll
        for (int q = 0; q < KQ; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NSUB; ++j) {
            // sub-stage j of strip s is the oldest pending group but DEPTH NSUB - 1
            asm volatile("cp.async.wait_group %0;" ::"n"(DEPTH * NSUB - 1) : "memory");
            const uint4* slot = stage + (size_t)(g % DEPTH) * RPT * CL_THREADS;
#pragma unroll
            for (int tt = 0; tt < TPS; ++tt) {
                const int t = j * TPS + tt;
                load16_smem<float, float>(reinterpret_cast<const float*>(&slot[t * CL_THREADS + tid]), sv[t]);
            }
            issue_sub(s + DEPTH * ncl, g + DEPTH, j);
            if (haveY) {
#pragma unroll
                for (int tt = 0; tt < TPS; ++tt) {
                    const int t = j * TPS + tt;
                    const int li = lrow0 + t * CL_SWEEP;
                    const float2 s01 = make_float2(sv[t][0], sv[t][1]), s23 = make_float2(sv[t][2], sv[t][3]);
                    if constexpr (KQ >= 2) {
#pragma unroll
                        for (int q = 0; q < KQ; q += 2) {
                            const float4 y4 = *reinterpret_cast<const float4*>(&Ys[(li * KQ + q) * 2]);
                            const float2 ya = make_float2(y4.x, y4.y), yb = make_float2(y4.z, y4.w);
                            acc[q][0] = f2fma(s01, ya, acc[q][0]);
                            acc[q][1] = f2fma(s23, ya, acc[q][1]);
                            acc[q + 1][0] = f2fma(s01, yb, acc[q + 1][0]);
                            acc[q + 1][1] = f2fma(s23, yb, acc[q + 1][1]);
                        }
                    } else {
                        const float2 ya = *reinterpret_cast<const float2*>(&Ys[li * 2]);
                        acc[0][0] = f2fma(s01, ya, acc[0][0]);
                        acc[0][1] = f2fma(s23, ya, acc[0][1]);
                    }
                }
            }
        }
        if (haveY) {
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    acc[q][h].x += __shfl_xor_sync(0xffffffffu, acc[q][h].x, 16);
                    acc[q][h].y += __shfl_xor_sync(0xffffffffu, acc[q][h].y, 16);
                }
            if (rr == 0) {
#pragma unroll
                for (int q = 0; q < KQ; ++q)
                    *reinterpret_cast<float4*>(&ured[(warp * KQ + q) * CL_W + cq * 4]) =
                        make_float4(acc[q][0].x, acc[q][0].y, acc[q][1].x, acc[q][1].y);
            }
            __syncthreads();
            float* qslot = pbuf + ((size_t)(par * CL_MAX_CS + rank) * KQ + uq) * CL_W + (uc & ~3);
            if (u_thread) {
                float p = 0.f;
#pragma unroll 4
                for (int w = 0; w < CL_WARPS; ++w) p += ured[(w * KQ + uq) * CL_W + uc];
                qslot[uc & 3] = p;
            }
            __syncwarp();
            if (u_thread) {
                // the 4 lanes of a column quad send its 16 bytes to the other ranks, lane j to the
                // peers j, j + 4 after this rank, one asynchronous remote store each
                // (test hook: rank 1 of the first cluster withholds its first strip's partials, so
                // the other ranks' bounded waits for them run out)
                const bool withhold = fault == DFS_TEST_FAULT_CLUSTER_PASS && cid == 0 && rank == 1 && s == cid;
                const float4 v4 = *reinterpret_cast<const float4*>(qslot);
                for (int pi = uc & 3; pi < (int)cs - 1; pi += 4)
                    if (!withhold) st_async_v4(qslot, &xbar[par], (rank + 1 + (uint32_t)pi) % cs, v4);
            }
            // (ured is rewritten only after the barrier below that ends this strip's u step)
        }
        // ---- U = V - S^T Y (ranks summed in order), X = U / lambda ----
        if (exch && u_thread) {
            if (!tc::mbar_wait_bounded(&xbar[par], (xphase >> par) & 1u, &s_abort, wait_ns)) {
                s_abort = 1;
                set_status(const_cast<DevStatus*>(st), DFS_ERR_TIMEOUT);
            }
        }
        if (exch) xphase ^= 1u << par;
        if (u_thread) {
            float sum = 0.f;
            if (haveY)
                for (uint32_t r = 0; r < cs; ++r) sum += pbuf[((size_t)(par * CL_MAX_CS + r) * KQ + uq) * CL_W + uc];
            const float u = u_valid ? v_pre - sum : 0.f;
            us[us_at] = u;
            if (u_valid && writer) {
                if (X != nullptr) {
                    const float xn = u * inv_lambda;
                    float dx = 0.f;
                    if (dmode == 1) dx = xn - x_pre;
                    else if (dmode == 2) dx = (u - v_pre) * inv_lambda;
                    d2f += dx * dx;
                    X[(int64_t)uq * ldx + j0 + uc] = xn;
                }
                u2f += u * u;
            }
        }
        __syncthreads();
        // ---- phase 2: R_rows += S_strip U_strip ----
        if (wantR) {
            if constexpr (KQ >= 2) {
#pragma unroll
                for (int p = 0; p < KP; ++p) {
                    const float4 ua = *reinterpret_cast<const float4*>(&us[((p * 2 + 0) * (CL_W / 4) + cq) * 4]);
                    const float4 ub = *reinterpret_cast<const float4*>(&us[((p * 2 + 1) * (CL_W / 4) + cq) * 4]);
                    // (u_{c,2p}, u_{c,2p+1}) for the lane's columns c = 4 cq + e
                    const float2 up[4] = {make_float2(ua.x, ua.y), make_float2(ua.z, ua.w), make_float2(ub.x, ub.y),
                                          make_float2(ub.z, ub.w)};
#pragma unroll
                    for (int t = 0; t < RPT; ++t) {
                        if constexpr (kLaneAcc) {
                            // this lane's 4 columns only; the 16 lanes of the row are added at the fold
#pragma unroll
                            for (int e = 0; e < 4; ++e) racc[t][p] = f2fma(f2dup(sv[t][e]), up[e], racc[t][p]);
                        } else {
                            float2 a = make_float2(0.f, 0.f);
#pragma unroll
                            for (int e = 0; e < 4; ++e) a = f2fma(f2dup(sv[t][e]), up[e], a);
#pragma unroll
                            for (int o = 1; o < CL_LPR; o <<= 1) {
                                a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
                                a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
                            }
                            if (cq == 0) {
                                const int li = lrow0 + t * CL_SWEEP;
                                Rs32[li * KQ + 2 * p] += a.x;
                                Rs32[li * KQ + 2 * p + 1] += a.y;
                            }
                        }
                    }
                }
            } else {
                const float4 u4 = *reinterpret_cast<const float4*>(&us[cq * 4]);
#pragma unroll
                for (int t = 0; t < RPT; ++t) {
                    if constexpr (kLaneAcc) {
                        float a = racc[t][0].x;
                        a = fmaf(sv[t][0], u4.x, a);
                        a = fmaf(sv[t][1], u4.y, a);
                        a = fmaf(sv[t][2], u4.z, a);
                        a = fmaf(sv[t][3], u4.w, a);
                        racc[t][0].x = a;
                    } else {
                        float a = sv[t][0] * u4.x;
                        a = fmaf(sv[t][1], u4.y, a);
                        a = fmaf(sv[t][2], u4.z, a);
                        a = fmaf(sv[t][3], u4.w, a);
#pragma unroll
                        for (int o = 1; o < CL_LPR; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                        if (cq == 0) Rs32[(lrow0 + t * CL_SWEEP) * KQ] += a;
                    }
                }
            }
        }
        if (++since_fold == CL_FOLD) {
            since_fold = 0;
            if constexpr (kLaneAcc) {
                if (wantR) fold_lanes();
            } else if (wantR && cq == 0) {
                for (int li = lrow0; li < RC; li += CL_SWEEP)
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        Rs64[li * KQ + q] += (double)Rs32[li * KQ + q];
                        Rs32[li * KQ + q] = 0.f;
                    }
            }
            u2 += (double)u2f;
            d2 += (double)d2f;
            u2f = d2f = 0.f;
        }
        // us is rewritten by the next strip only after that strip's first barrier, which every
        // thread of this CTA reaches after finishing phase 2 here
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if constexpr (kLaneAcc) {
        if (wantR) fold_lanes();
    } else if (wantR && cq == 0) {
        for (int li = lrow0; li < RC; li += CL_SWEEP)
#pragma unroll
            for (int q = 0; q < KQ; ++q) Rs64[li * KQ + q] += (double)Rs32[li * KQ + q];
    }
    u2 += (double)u2f;
    d2 += (double)d2f;
    __syncthreads();
    if (wantR) {
        double* dst = Rpart + cid * (int64_t)n * KQ;
        for (int e = tid; e < RC * KQ; e += CL_THREADS) {
            const int i = r0 + e / KQ;
            if (i < n && DFS_IN_BOUNDS(st, cid < ncl)) dst[(int64_t)i * KQ + e % KQ] = Rs64[e];
        }
    }
    // per-RHS sums of U^2 and dX^2: lanes -> warp; the two warps of a right-hand side -> CTA;
    // ranks in order -> rank 0 -> U2part[cid] (u2 for q = 0..KQ-1, then dX^2)
    {
        double v = u2, w = d2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (lane == 0) {
            u2s[warp][0] = v;
            u2s[warp][1] = w;
        }
    }
    __syncthreads();
    if (tid < 2 * KQ) {
        const int q = tid % KQ, which = tid / KQ;
        const double v = u2s[2 * q][which] + u2s[2 * q + 1][which];
        st_cluster_f64(&u2c[rank][tid], 0, v);
    }
    cl_sync();
    if (rank == 0 && tid < 2 * KQ) {
        double v = 0.0;
        for (uint32_t r = 0; r < cs; ++r) v += u2c[r][tid];
        if (DFS_IN_BOUNDS(st, cid < ncl)) U2part[cid * 2 * KQ + tid] = v;
    }
}

// ---- host side ------------------------------------------------------------------------------

// Rows per thread for n rows split over cs CTAs of at most 512 rows; 0 if the cluster form does
// not apply (needs FP32 S, KQ <= 8, n <= 4096; n <= 2048 for KQ = 8).  Where n fits in 8 CTAs
// whose lanes can keep their row sums in registers (RPT KQ <= 32), those are used.
static int cluster_rpt(int n, int KQ, int* cs_out) {
    if (KQ > 8) return 0;
    const int lane_rpt = KQ >= 2 ? 32 / KQ < 16 ? 32 / KQ : 16 : 16;
    // eight right-hand sides fill all 512 threads with column sums and hold twice the
    // accumulators: at most 8 rows a thread (256 a CTA), so n <= 2048
    int max_rpt = KQ == 8 ? 8 : 16;
    if (kPreferLaneAcc && n <= CL_MAX_CS * lane_rpt * CL_SWEEP) max_rpt = lane_rpt;
    if (n > CL_MAX_CS * max_rpt * CL_SWEEP) return 0;
    const int cs = (n + max_rpt * CL_SWEEP - 1) / (max_rpt * CL_SWEEP);
    const int per = (n + cs - 1) / cs;
    int rpt = 4;
    while (rpt * CL_SWEEP < per) rpt *= 2;
    *cs_out = cs;
    return rpt;
}

static size_t cluster_smem_bytes(int rpt, int KQ) {
    return (size_t)cl_depth(rpt, KQ) * rpt * CL_THREADS * 16 + cl_rest_bytes(rpt, KQ);
}

template <int KQ, int RPT>
static int max_active_clusters_t(int cs) {
    const size_t smem = cluster_smem_bytes(RPT, KQ);
    auto kern = fisher_pass_cluster_kernel<KQ, RPT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Clusters of cs CTAs that can be resident at once (the GPCs bound this below num_sms / cs).
static int max_active_clusters(int kq, int rpt, int cs) {
#define DFS_CLMAX(KQ, R) \
    if (kq == KQ && rpt == R) return max_active_clusters_t<KQ, R>(cs);
    DFS_CLMAX(1, 4) DFS_CLMAX(1, 8) DFS_CLMAX(1, 16)
    DFS_CLMAX(2, 4) DFS_CLMAX(2, 8) DFS_CLMAX(2, 16)
    DFS_CLMAX(4, 4) DFS_CLMAX(4, 8) DFS_CLMAX(4, 16)
    DFS_CLMAX(8, 4) DFS_CLMAX(8, 8)
#undef DFS_CLMAX
    return 0;
}

int pass_cluster_plan(int s_dtype, int n, int KQ, int num_sms, int64_t m, size_t smem_limit, int* cs_out,
                      int* rpt_out) {
    *cs_out = 0;
    *rpt_out = 0;
    if (s_dtype != DFS_F32) return 0;
    int cs = 0;
    const int rpt = cluster_rpt(n, KQ, &cs);
    if (rpt == 0 || cluster_smem_bytes(rpt, KQ) + 4096 > smem_limit) return 0;
    // every cluster resident at once (static strip assignment: a second wave would double the time)
    int64_t ncl = max_active_clusters(KQ, rpt, cs);
    if (ncl > num_sms / cs) ncl = num_sms / cs;
    const int64_t nstrips = ceil_div(m, CL_W);
    if (ncl > nstrips) ncl = nstrips;
    if (ncl < 1) return 0;
    *cs_out = cs;
    *rpt_out = rpt;
    return (int)ncl;
}

template <int KQ, int RPT>
static cudaError_t launch_cl_t(int ncl, int cs, const float* S, int n, int64_t m, int64_t lds, const float* V,
                               int64_t ldv, int k, const double* Y, int64_t ldy, double lambda, float* X, int64_t ldx,
                               double* Rpart, double* U2part, int dmode, const DevStatus* st, int honor_stop,
                               cudaStream_t stream) {
    const size_t smem = cluster_smem_bytes(RPT, KQ);
    auto kern = fisher_pass_cluster_kernel<KQ, RPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ncl * cs));
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, S, n, m, lds, V, ldv, k, Y, ldy, lambda, X, ldx, Rpart, U2part, dmode, st,
                           honor_stop);
    count_launch();
    return e;
}

cudaError_t launch_pass_cluster(int ncl, int cs, int rpt, int kq, const void* S, int n, int64_t m, int64_t lds,
                                const void* V, int64_t ldv, int k, const double* Y, int64_t ldy, double lambda,
                                void* X, int64_t ldx, double* Rpart, double* U2part, int dmode, const DevStatus* st,
                                int honor_stop, cudaStream_t stream) {
    const float* s = static_cast<const float*>(S);
    const float* v = static_cast<const float*>(V);
    float* x = static_cast<float*>(X);
#define DFS_CL(KQ, R)                                                                                             \
    if (kq == KQ && rpt == R)                                                                                     \
        return launch_cl_t<KQ, R>(ncl, cs, s, n, m, lds, v, ldv, k, Y, ldy, lambda, x, ldx, Rpart, U2part, dmode, \
                                  st, honor_stop, stream);
    DFS_CL(1, 4) DFS_CL(1, 8) DFS_CL(1, 16)
    DFS_CL(2, 4) DFS_CL(2, 8) DFS_CL(2, 16)
    DFS_CL(4, 4) DFS_CL(4, 8) DFS_CL(4, 16)
    DFS_CL(8, 4) DFS_CL(8, 8)
#undef DFS_CL
    return cudaErrorInvalidValue;
}

}  // namespace dfs
