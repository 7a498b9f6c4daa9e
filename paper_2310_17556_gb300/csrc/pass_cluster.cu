// The fused refinement pass of pass.cu (U = V - S^T Y, X = U / lambda, R = S U - lambda Y in one
// read of S) for FP32 S with n <= 4096, as thread-block clusters.
//
// Reading S in strips of all n rows x 128 bytes (one CTA per strip) tops out near 4.8 TB/s on
// GB300: every 128 KB strip touches n rows megabytes apart.  Row segments of >= 256 bytes with
// <= 512 rows per CTA reach the copy rate, so here a cluster of cs = ceil(n / RC) CTAs shares
// one strip of 64 columns (256 bytes per row): CTA `rank` owns rows [rank RC, rank RC + RC)
// (RC = 32 RPT), keeps its RC x 64 slice in registers (16 lanes x 16 bytes per row, RPT rows per
// thread) and stages the next strip's slice in shared memory with cp.async meanwhile.
// Per strip:
//   phase 1  column sums of S^T Y over the CTA's rows (shuffle + shared memory), written to every
//            CTA of the cluster with asynchronous remote stores that complete the transaction count
//            of the receiver's mbarrier (no fence, so the next strip's loads stay in flight), then
//            each CTA forms U = V - sum over ranks in rank order (so all ranks hold identical U);
//            rank r writes X (and the stopping-rule sums) for columns c with floor(c cs / 64) = r;
//   phase 2  per-row dot products with U into FP32 row sums, folded into FP64 every 32 strips.
// Partials are per cluster: Rpart[c] holds all n rows (each rank its own rows), U2part[c] the
// per-RHS sums (combined over ranks through rank 0).  The exchange buffers and their mbarriers are
// double-buffered by strip parity: a rank sends strip s + 2's partials (same parity as s) only
// after it has received strip s + 1's from every rank, which each rank sends only after its own
// reads of strip s's buffer, so no buffer is overwritten while it is read.
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
// Asynchronous remote store of a float into CTA `rank`'s copy of `local`, completing 4 bytes of
// the transaction count of that CTA's copy of mbarrier `bar`.
__device__ __forceinline__ void st_async_f32(const void* local, const uint64_t* bar, uint32_t rank, float v) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), b = static_cast<uint32_t>(
                 __cvta_generic_to_shared(bar)), ra, rb;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(b), "r"(rank));
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(ra),
                 "r"(__float_as_uint(v)), "r"(rb)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_f64(const void* local, uint32_t rank, double v) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(r), "d"(v) : "memory");
}

template <int KQ, int RPT>
__global__ void __launch_bounds__(CL_THREADS, 1)
fisher_pass_cluster_kernel(const float* __restrict__ S, int n, int64_t m, int64_t lds, const float* __restrict__ V,
                           int64_t ldv, int k, const double* __restrict__ Y, int64_t ldy, double lambda,
                           float* __restrict__ X, int64_t ldx, double* __restrict__ Rpart,
                           double* __restrict__ U2part, int dmode, const DevStatus* st, int honor_stop) {
    constexpr int RC = RPT * CL_SWEEP;  // rows per CTA
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* stage = reinterpret_cast<uint4*>(smem);                                  // RPT x 512 x 16 B
    double* Rs64 = reinterpret_cast<double*>(smem + (size_t)RPT * CL_THREADS * 16);  // RC x KQ
    float* Rs32 = reinterpret_cast<float*>(Rs64 + RC * KQ);                         // RC x KQ
    float* Ys = Rs32 + RC * KQ;                                                      // RC x KQ
    float* ured = Ys + RC * KQ;                                                      // warps x W x KQ
    float* pbuf = ured + CL_WARPS * CL_W * KQ;                                       // 2 x MAX_CS x W x KQ
    float* us = pbuf + 2 * CL_MAX_CS * CL_W * KQ;                                    // W x KQ
    __shared__ double u2s[CL_WARPS][16];
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
        Ys[e] = (haveY && i < n && q < k) ? (float)Y[(int64_t)i * ldy + q] : 0.f;
    }
    const int64_t nstrips = ceil_div(m, CL_W);
    const int lrow0 = warp * 2 + rr;  // local row of t = 0
    // The strip's rows arrive in NSUB sub-stages (rows t in [j RPT/NSUB, (j+1) RPT/NSUB) of every
    // thread); slot j of the ring is refilled with the next strip's sub-stage j as soon as this
    // thread has moved it into registers, so about one strip stays in flight at all times.
    constexpr int NSUB = RPT >= 4 ? 4 : RPT;
    constexpr int TPS = RPT / NSUB;  // rows per thread per sub-stage
    auto issue_sub = [&](int64_t sidx, int j) {
        if (sidx < nstrips) {
            const int64_t jn = sidx * CL_W + cq * 4;
            const int64_t rem = m - jn;
            const int bytes_col = rem >= 4 ? 16 : (rem > 0 ? (int)rem * 4 : 0);
#pragma unroll
            for (int tt = 0; tt < TPS; ++tt) {
                const int t = j * TPS + tt;
                const int i = r0 + lrow0 + t * CL_SWEEP;
                const int bytes = i < n ? bytes_col : 0;
                const float* src = bytes ? S + (int64_t)i * lds + jn : S;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                 static_cast<uint32_t>(__cvta_generic_to_shared(&stage[t * CL_THREADS + tid]))),
                             "l"(src), "r"(bytes)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");  // (empty past the last strip)
    };
#pragma unroll
    for (int j = 0; j < NSUB; ++j) issue_sub(cid, j);
    float u2f[KQ], d2f[KQ];
    double u2[KQ], d2[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) u2f[q] = d2f[q] = 0.f, u2[q] = d2[q] = 0.0;
    const bool u_thread = tid < CL_W * KQ;
    const int uc = tid / KQ, uq = tid % KQ;
    const bool writer = u_thread && (uc * (int)cs) / CL_W == (int)rank;  // ranks split the columns
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
    // (its 4 columns of every strip) in registers and the 16 lanes of a row are added only at
    // each fold, in place of 4 shuffles per row and right-hand side on every strip.
    constexpr bool kLaneAcc = RPT * KQ <= 32;
    float racc[kLaneAcc ? RPT : 1][kLaneAcc ? KQ : 1];
#pragma unroll
    for (int t = 0; t < (kLaneAcc ? RPT : 1); ++t)
#pragma unroll
        for (int q = 0; q < (kLaneAcc ? KQ : 1); ++q) racc[t][q] = 0.f;
    auto fold_lanes = [&]() {
#pragma unroll
        for (int t = 0; t < (kLaneAcc ? RPT : 1); ++t) {
            const int li = lrow0 + t * CL_SWEEP;
#pragma unroll
            for (int q = 0; q < (kLaneAcc ? KQ : 1); ++q) {
                float a = racc[t][q];
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                a += __shfl_xor_sync(0xffffffffu, a, 4);
                a += __shfl_xor_sync(0xffffffffu, a, 8);
                if (cq == 0) Rs64[li * KQ + q] += (double)a;
                racc[t][q] = 0.f;
            }
        }
    };
    int since_fold = 0, par = 0;
    for (int64_t s = cid; s < nstrips; s += ncl, par ^= 1) {
        const int64_t j0 = s * CL_W;
        float sv[RPT][4];
        float v_pre = 0.f, x_pre = 0.f;
        const bool u_valid = u_thread && (j0 + uc < m) && (uq < k);
        if (u_valid) {
            v_pre = V[(int64_t)uq * ldv + j0 + uc];
            if (writer && X != nullptr && dmode == 1) x_pre = X[(int64_t)uq * ldx + j0 + uc];
        }
        // ---- phase 1: this CTA's column sums of S^T Y -> every rank's pbuf[par][rank] ----
        const bool exch = haveY && cs > 1;
        if (exch && tid == 0 && !s_abort) tc::mbar_arrive_expect_tx(&xbar[par], xbytes);
        float acc[KQ][4];
#pragma unroll
        for (int q = 0; q < KQ; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
#pragma unroll
        for (int j = 0; j < NSUB; ++j) {
            // sub-stage j of strip s is the oldest pending group but NSUB - 1
            asm volatile("cp.async.wait_group %0;" ::"n"(NSUB - 1) : "memory");
#pragma unroll
            for (int tt = 0; tt < TPS; ++tt) {
                const int t = j * TPS + tt;
                load16_smem<float, float>(reinterpret_cast<const float*>(&stage[t * CL_THREADS + tid]), sv[t]);
            }
            issue_sub(s + ncl, j);
            if (haveY) {
#pragma unroll
                for (int tt = 0; tt < TPS; ++tt) {
                    const int t = j * TPS + tt;
                    const int li = lrow0 + t * CL_SWEEP;
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        const float yv = Ys[li * KQ + q];
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[q][e] = fmaf(sv[t][e], yv, acc[q][e]);
                    }
                }
            }
        }
        if (haveY) {
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[q][e] += __shfl_xor_sync(0xffffffffu, acc[q][e], 16);
            if (rr == 0) {
#pragma unroll
                for (int q = 0; q < KQ; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) ured[(warp * CL_W + cq * 4 + e) * KQ + q] = acc[q][e];
            }
            __syncthreads();
            if (u_thread) {
                float p = 0.f;
#pragma unroll 4
                for (int w = 0; w < CL_WARPS; ++w) p += ured[(w * CL_W + uc) * KQ + uq];
                float* slot = pbuf + ((size_t)(par * CL_MAX_CS + rank) * CL_W + uc) * KQ + uq;
                *slot = p;
                // (test hook: rank 1 of the first cluster withholds its first strip's partials, so
                // the other ranks' bounded waits for them run out)
                const bool withhold = fault == DFS_TEST_FAULT_CLUSTER_PASS && cid == 0 && rank == 1 && s == cid;
                for (uint32_t r = 0; r < cs; ++r)
                    if (r != rank && !withhold) st_async_f32(slot, &xbar[par], r, p);
            }
            __syncthreads();
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
                for (uint32_t r = 0; r < cs; ++r) sum += pbuf[((size_t)(par * CL_MAX_CS + r) * CL_W + uc) * KQ + uq];
            const float u = u_valid ? v_pre - sum : 0.f;
            us[uc * KQ + uq] = u;
            if (u_valid && writer) {
                if (X != nullptr) {
                    const float xn = u * inv_lambda;
                    float dx = 0.f;
                    if (dmode == 1) dx = xn - x_pre;
                    else if (dmode == 2) dx = (u - v_pre) * inv_lambda;
                    d2f[uq] += dx * dx;
                    X[(int64_t)uq * ldx + j0 + uc] = xn;
                }
                u2f[uq] += u * u;
            }
        }
        __syncthreads();
        // ---- phase 2: R_rows += S_strip U_strip ----
        if (wantR) {
            float uu[KQ][4];
#pragma unroll
            for (int q = 0; q < KQ; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) uu[q][e] = us[(cq * 4 + e) * KQ + q];
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int li = lrow0 + t * CL_SWEEP;
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    if constexpr (kLaneAcc) {
                        // this lane's 4 columns only; the 16 lanes of the row are added at the fold
#pragma unroll
                        for (int e = 0; e < 4; ++e) racc[t][q] = fmaf(sv[t][e], uu[q][e], racc[t][q]);
                    } else {
                        float a = 0.f;
#pragma unroll
                        for (int e = 0; e < 4; ++e) a = fmaf(sv[t][e], uu[q][e], a);
                        a += __shfl_xor_sync(0xffffffffu, a, 1);
                        a += __shfl_xor_sync(0xffffffffu, a, 2);
                        a += __shfl_xor_sync(0xffffffffu, a, 4);
                        a += __shfl_xor_sync(0xffffffffu, a, 8);
                        if (cq == 0) Rs32[li * KQ + q] += a;
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
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                u2[q] += (double)u2f[q];
                d2[q] += (double)d2f[q];
                u2f[q] = d2f[q] = 0.f;
            }
        }
        // us is rewritten by the next strip only after its cluster barrier, which every thread
        // of this CTA reaches after finishing phase 2 here
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if constexpr (kLaneAcc) {
        if (wantR) fold_lanes();
    } else if (wantR && cq == 0) {
        for (int li = lrow0; li < RC; li += CL_SWEEP)
#pragma unroll
            for (int q = 0; q < KQ; ++q) Rs64[li * KQ + q] += (double)Rs32[li * KQ + q];
    }
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        u2[q] += (double)u2f[q];
        d2[q] += (double)d2f[q];
    }
    __syncthreads();
    if (wantR) {
        double* dst = Rpart + cid * (int64_t)n * KQ;
        for (int e = tid; e < RC * KQ; e += CL_THREADS) {
            const int i = r0 + e / KQ;
            if (i < n) dst[(int64_t)i * KQ + e % KQ] = Rs64[e];
        }
    }
    // per-RHS sums of U^2 and dX^2: warps -> CTA -> rank 0 (ranks in order) -> U2part[cid]
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
    if (tid < 2 * KQ) {
        const int slot = tid < KQ ? tid : 8 + (tid - KQ);
        double v = 0.0;
        for (int wp = 0; wp < CL_WARPS; ++wp) v += u2s[wp][slot];
        st_cluster_f64(&u2c[rank][tid], 0, v);
    }
    cl_sync();
    if (rank == 0 && tid < 2 * KQ) {
        double v = 0.0;
        for (uint32_t r = 0; r < cs; ++r) v += u2c[r][tid];
        U2part[cid * 2 * KQ + tid] = v;
    }
}

// ---- host side ------------------------------------------------------------------------------

// Rows per thread for n rows split over cs CTAs of at most 512 rows; 0 if the cluster form does
// not apply (needs FP32 S, KQ <= 4, n <= 4096).
static int cluster_rpt(int n, int KQ, int* cs_out) {
    // eight right-hand sides fill all 512 threads with column sums and hold twice the
    // accumulators: at most 8 rows a thread (256 a CTA), so n <= 2048
    const int max_rpt = KQ == 8 ? 8 : 16;
    if (KQ > 8 || n > CL_MAX_CS * max_rpt * CL_SWEEP) return 0;
    const int cs = (n + max_rpt * CL_SWEEP - 1) / (max_rpt * CL_SWEEP);
    const int per = (n + cs - 1) / cs;
    int rpt = 4;
    while (rpt * CL_SWEEP < per) rpt *= 2;
    *cs_out = cs;
    return rpt;
}

static size_t cluster_smem_bytes(int rpt, int KQ) {
    const size_t rc = (size_t)rpt * CL_SWEEP;
    return (size_t)rpt * CL_THREADS * 16 + rc * KQ * (8 + 4 + 4) + (size_t)CL_WARPS * CL_W * KQ * 4 +
           (size_t)2 * CL_MAX_CS * CL_W * KQ * 4 + (size_t)CL_W * KQ * 4;
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
