// The n-space part of Algorithm 1 between two passes over S, as one cluster kernel:
//   (optional) r = sum of the pass partials (fixed order) [- lambda y]   (the right-hand side b = S v,
//              or the refinement residual r = S u - lambda y of Appendix A's identity)
//   a = L^{-1} r   (forward block substitution)
//   z = L^{-T} a   (backward block substitution, on U = L^T held in W's upper triangle)
// replacing a reduction kernel and two single-CTA triangular solves.
//
// A cluster of cs CTAs shares the work by 64-row super-blocks: super-block sb (rows 64 sb ..
// 64 sb + 63) is owned by rank sb mod cs, which reduces its right-hand side, applies every update
// to it and solves its diagonal 64 x 64 block with that block's inverse (formed at the start from the
// Cholesky's 32 x 32 inverses: [[A, 0], [B, C]]^-1 has off-diagonal block -C^-1 B A^-1).  The solved
// values are broadcast to every other rank with asynchronous 16-byte remote stores (st.async) that
// complete the transaction count of the receiver's per-super-block mbarrier, one warp per
// receiver; a rank that owns a later super-block I then applies
// t_I -= L[I, sb] y_sb.  Each rank streams the 64 x 64 tiles of L (forward) and U (backward) it
// needs, in the order it consumes them, through a cp.async ring in shared memory (the loads do not
// depend on the solution, so the ring runs ahead); the diagonal pieces and inverses of its own
// super-blocks are formed once at the start.  The critical path per super-block is one 64 x 64
// tile update, one 64 x 64 product with the inverse and one broadcast.
//
// Products and sums in T (FP32 on the FP32 / mixed paths, FP64 on the FP64 path); the reduction in
// FP64.  Every wait is bounded (DFS_ERR_TIMEOUT); with `stop` set (refinement converged) the kernel
// returns at once.
#define DFS_SRC_ID 6
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dfs {

namespace {

constexpr int NS_THREADS = 512;
constexpr int NS_SB = 64;          // super-block rows
constexpr int NS_B = 32;           // Cholesky block (Linv granularity)
constexpr int NS_MAX_CS = 8;
constexpr int NS_MAX_SLOTS = 8;

__device__ __forceinline__ uint32_t ns_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t ns_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void ns_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t ns_mapa(const void* p, uint32_t rank) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// Bounded wait for phase `parity` of a local mbarrier: spins on try_wait, and only every 1024
// polls looks at the abort flag and the clock (the call's wait limit).
__device__ __forceinline__ bool ns_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint64_t limit_ns) {
    uint64_t t0 = 0;
    for (uint32_t spins = 1;; ++spins) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((spins & 1023u) == 0) {
            if (*abort) return false;
            const uint64_t t = tc::globaltimer_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}

template <typename T>
struct NsLayout {
    static constexpr int RS = NS_SB + 16 / (int)sizeof(T);  // padded tile row (elements)
    static constexpr int TILE = NS_SB * RS;                  // elements per ring slot
    static constexpr int P65 = NS_SB + 1;                    // padded row of a diagonal inverse
    static constexpr int DIAG = NS_SB * P65;                 // inverse of one 64 x 64 diagonal block
};
__device__ __forceinline__ void ns_st_async_v4(uint32_t raddr, uint32_t rbar, uint4 v) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     raddr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar)
                 : "memory");
}

}  // namespace

// Counts of a rank's off-diagonal tiles.  In consumption order the tiles are: forward, for
// sb = 0 .. nsb-2, owned I > sb ascending, tile (I, sb) of L; backward, for sb = nsb-1 .. 1, owned
// I < sb descending, tile (I, sb) of U (W's upper triangle).  The kernel lists them once in
// shared memory.
struct NsSeq {
    int nsb, cs, rank, fwd, bwd;
    // number of owned super-blocks strictly after / before sb
    __device__ int owned_after(int sb) const {
        // owned I in (sb, nsb): I = rank + j cs
        const int first = sb + 1 + ((rank - (sb + 1)) % cs + cs) % cs;
        return first < nsb ? (nsb - 1 - first) / cs + 1 : 0;
    }
    __device__ int owned_before(int sb) const {
        // owned I in [0, sb)
        return sb > rank ? (sb - 1 - rank) / cs + 1 : 0;
    }
    __device__ int total() const {
        int t = 0;
        if (fwd)
            for (int sb = 0; sb < nsb; ++sb) t += owned_after(sb);
        if (bwd)
            for (int sb = nsb - 1; sb >= 0; --sb) t += owned_before(sb);
        return t;
    }
};

constexpr int NS_REDUCE = NS_MODE_REDUCE;
constexpr int NS_LAMBDA_Y = NS_MODE_LAMBDA_Y;
constexpr int NS_FWD = NS_MODE_FWD;
constexpr int NS_BWD = NS_MODE_BWD;

template <typename T, int KQ>
__global__ void __launch_bounds__(NS_THREADS, 1)
nspace_kernel(const T* __restrict__ W, int64_t ld, int n_pad, const T* __restrict__ Linv, int mode,
              const double* __restrict__ Rpart, int nparts, int n, int k, const double* __restrict__ Y,
              double lambda, const T* __restrict__ B, int64_t ldb, double* __restrict__ R, T* __restrict__ Z,
              int64_t ldz, const double* __restrict__ U2part, double* __restrict__ U2, int nslots, DevStatus* st,
              int honor_stop) {
    using L = NsLayout<T>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nsb = n_pad / NS_SB;
    // layout: ring | x (n_pad x KQ) | own diag data | reduction scratch | mbarriers
    T* ring = reinterpret_cast<T*>(smem);
    T* x = ring + (size_t)nslots * L::TILE;
    T* diag = x + (size_t)n_pad * KQ;
    __shared__ int s_abort;
    __shared__ double red[NS_THREADS / NS_SB][NS_SB];  // the reduction's group sums

    if (block_should_exit(st, honor_stop)) return;  // cluster-uniform: earlier launches write it
    const uint64_t wait_ns = wait_limit(st);  // the call's wait limit, read once
    const uint32_t cs = ns_size(), rank = ns_rank();
    const int nown = (nsb - (int)rank + (int)cs - 1) / (int)cs;  // owned super-blocks
    const int nown_max = (nsb + (int)cs - 1) / (int)cs;          // same offset in every rank
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(diag + (size_t)nown_max * L::DIAG) + 7) & ~uintptr_t(7));  // 2 x nsb
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool fwd = (mode & NS_FWD) != 0, bwd = (mode & NS_BWD) != 0;
    const NsSeq seq{nsb, (int)cs, (int)rank, fwd ? 1 : 0, bwd ? 1 : 0};
    const uint32_t ybytes = NS_SB * KQ * sizeof(T);

    // the tile sequence of this rank, (I << 16 | sb) per entry, in consumption order
    int* tseq = reinterpret_cast<int*>(bars + 2 * nsb);
    if (tid == 0) {
        int t = 0;
        if (fwd)
            for (int sb = 0, first = (int)rank; sb < nsb; ++sb) {  // first owned I > sb
                if (first <= sb) first += (int)cs;
                for (int I = first; I < nsb; I += (int)cs) tseq[t++] = (I << 16) | sb;
            }
        if (bwd)
            for (int sb = nsb - 1; sb >= 0; --sb) {
                const int c = seq.owned_before(sb);
                for (int j = 0, I = (int)rank + (c - 1) * (int)cs; j < c; ++j, I -= (int)cs) tseq[t++] = (I << 16) | sb;
            }
    }
    if (tid == 0) s_abort = 0;
    if (tid < 2 * nsb) {  // one mbarrier per thread; armed for the super-blocks other ranks solve
        const int sb = tid % nsb;
        const bool dir_on = tid < nsb ? fwd : bwd;
        tc::mbar_init(&bars[tid], 1);
        tc::fence_mbar_init();
        if (dir_on && sb % (int)cs != (int)rank) tc::mbar_arrive_expect_tx(&bars[tid], ybytes);
    }

    // ---- ring prologue: the first nslots - 1 tiles ----
    const int ntiles = seq.total();
    __syncthreads();  // tseq
    // Threads 0..255 work the tiles: thread (r = tid / 4, part = tid % 4) copies and later reads
    // 16 elements of row r (columns 16 part ..), so a tile needs no barrier between its copy and
    // its use, and a slot is refilled by the threads that just read it.
    constexpr int NS_GT = 4 * NS_SB;             // GEMV threads
    constexpr int CPT = 16 * (int)sizeof(T) / 16;  // 16-byte chunks per thread and tile
    const bool gthread = tid < NS_GT;
    const int gr = tid >> 2, gpart = tid & 3;
    auto issue_tile = [&](int idx) {
        if (!gthread) return;
        if (idx < ntiles) {
            const int I = tseq[idx] >> 16, sb = tseq[idx] & 0xffff;
            if (!DFS_IN_BOUNDS(st, I < nsb && sb < nsb && (I + 1) * NS_SB <= n_pad)) {
                asm volatile("cp.async.commit_group;" ::: "memory");
                return;
            }
            T* dst = ring + (size_t)(idx % nslots) * L::TILE + gr * L::RS + gpart * 16;
            const T* src = W + ((int64_t)I * NS_SB + gr) * ld + (int64_t)sb * NS_SB + gpart * 16;
#pragma unroll
            for (int c = 0; c < CPT; ++c) cp_async16(dst + c * (16 / (int)sizeof(T)), src + c * (16 / (int)sizeof(T)));
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int i = 0; i < nslots - 1; ++i) issue_tile(i);

    // ---- inverse of each owned 64 x 64 diagonal block: [[A, 0], [B, C]]^-1 = [[A^-1, 0], [X, C^-1]]
    // with X = -C^-1 (B A^-1); A^-1, C^-1 are the Cholesky's 32 x 32 inverses, B = L[64 sb + 32.., 64 sb..]
    for (int j = 0; j < nown; ++j) {
        const int sb = (int)rank + j * (int)cs;
        T* dd = diag + (size_t)j * L::DIAG;
        const int64_t o = (int64_t)sb * NS_SB;
        const T* A = Linv + (int64_t)(2 * sb) * NS_B * NS_B;
        const T* C = Linv + (int64_t)(2 * sb + 1) * NS_B * NS_B;
        // pass 1: A^-1 and C^-1 into place, B into the (unused until pass 3) upper-right block
        for (int e = tid; e < NS_B * NS_B; e += NS_THREADS) {
            const int r = e / NS_B, c = e % NS_B;
            const T a = A[e], cc = C[e], b = W[(o + NS_B + r) * ld + o + c];
            dd[r * L::P65 + c] = a;
            dd[(NS_B + r) * L::P65 + NS_B + c] = cc;
            dd[r * L::P65 + NS_B + c] = b;  // B parked in the zero block
        }
        __syncthreads();
        // pass 2: T = B A^-1 into the lower-left block
        for (int e = tid; e < NS_B * NS_B; e += NS_THREADS) {
            const int r = e / NS_B, c = e % NS_B;
            T t = 0;
#pragma unroll 8
            for (int p = c; p < NS_B; ++p) t = fma(dd[r * L::P65 + NS_B + p], dd[p * L::P65 + c], t);
            dd[(NS_B + r) * L::P65 + c] = t;
        }
        __syncthreads();
        // pass 3: X = -C^-1 T (C^-1 lower triangular), and the upper-right block back to zero
        T xv[NS_B * NS_B / NS_THREADS];
#pragma unroll
        for (int u = 0; u < NS_B * NS_B / NS_THREADS; ++u) {
            const int e = tid + u * NS_THREADS, r = e / NS_B, c = e % NS_B;
            T t = 0;
#pragma unroll 8
            for (int p = 0; p <= r; ++p) t = fma(dd[(NS_B + r) * L::P65 + NS_B + p], dd[(NS_B + p) * L::P65 + c], t);
            xv[u] = -t;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NS_B * NS_B / NS_THREADS; ++u) {
            const int e = tid + u * NS_THREADS, r = e / NS_B, c = e % NS_B;
            dd[(NS_B + r) * L::P65 + c] = xv[u];
            dd[r * L::P65 + NS_B + c] = (T)0;
        }
        __syncthreads();
    }

    // ---- right-hand side of the owned rows (and the FP64 residual R) ----
    // Thread (g, r, q) adds the parts b = g, g + NG, ... of entry (row r, RHS q) of each owned
    // super-block (8 interleaved sums, then their fixed tree); the NG groups are then added in order.
    constexpr int NE = NS_SB * KQ;          // entries of a super-block
    constexpr int NG = NS_THREADS / NE;     // part groups (1 with 8 right-hand sides)
    double* redf = &red[0][0];              // NG x NE
    for (int j = 0; j < nown; ++j) {
        const int sb = (int)rank + j * (int)cs;
        const int e = tid % NE, g = tid / NE;
        const int r = e / KQ, q = e % KQ;
        const int i = sb * NS_SB + r;
        if (g < NG) {
            double v = 0.0;
            if ((mode & NS_REDUCE) && i < n && q < k) {
                const double* p = Rpart + (int64_t)i * KQ + q;
                const int64_t stride = (int64_t)n * KQ;
                double a8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                int b = g;
                for (; b + 7 * NG < nparts; b += 8 * NG) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) a8[u] += p[(int64_t)(b + u * NG) * stride];
                }
                for (; b < nparts; b += NG) a8[0] += p[(int64_t)b * stride];
                v = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
            }
            redf[g * NE + e] = v;
        }
        __syncthreads();
        if (tid < NE) {  // g = 0, e = tid: row sb * 64 + r, RHS q
            if (mode & NS_REDUCE) {
                double t = 0.0;
#pragma unroll
                for (int gg = 0; gg < NG; ++gg) t += redf[gg * NE + tid];
                if (!(i < n && q < k)) t = 0.0;
                if ((mode & NS_LAMBDA_Y) && i < n && q < k) t -= lambda * Y[(int64_t)i * KQ + q];
                if (R != nullptr) R[(int64_t)i * KQ + q] = t;
                x[i * KQ + q] = (T)t;
            } else {
                x[i * KQ + q] = (q < k) ? B[(int64_t)i * ldb + q] : (T)0;
            }
        }
        __syncthreads();
    }
    // the refinement's stopping sums: one warp per entry
    if (U2 != nullptr && U2part != nullptr && rank == 0 && warp < 2 * KQ) {
        const int q = warp;
        double v = 0.0;
        for (int b = lane; b < nparts; b += 32) v += U2part[(int64_t)b * 2 * KQ + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) U2[q] = v;
    }
    __syncthreads();
    ns_cluster_sync();  // barriers initialised everywhere before any remote store

    bool ok = true;
    int it = 0;  // ring position
    // y_sb has landed (the GEMV threads, which read it, wait on the mbarrier themselves)
    auto wait_y = [&](uint64_t* bar) {
        if (gthread && !s_abort) {
            if (!ns_wait(bar, 0, &s_abort, wait_ns)) {
                s_abort = 1;
                set_status(st, DFS_ERR_TIMEOUT);
            }
        }
    };
    // t_I -= tile * y_sb for the next ring tile (rows of super-block I, columns of super-block sb)
    auto consume = [&](int I, int sb) {
        if (gthread) {
            // this thread's part of the tile (nslots - 2 younger groups may stay in flight)
            if (nslots >= 8) asm volatile("cp.async.wait_group 6;" ::: "memory");
            else if (nslots == 7) asm volatile("cp.async.wait_group 5;" ::: "memory");
            else if (nslots == 6) asm volatile("cp.async.wait_group 4;" ::: "memory");
            else if (nslots == 5) asm volatile("cp.async.wait_group 3;" ::: "memory");
            else if (nslots == 4) asm volatile("cp.async.wait_group 2;" ::: "memory");
            else if (nslots == 3) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            const T* row = ring + (size_t)(it % nslots) * L::TILE + gr * L::RS + gpart * 16;
            const T* ys = x + ((size_t)sb * NS_SB + gpart * 16) * KQ;
            T acc[2][KQ];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int q = 0; q < KQ; ++q) acc[h][q] = 0;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const T lv = row[c];
#pragma unroll
                for (int q = 0; q < KQ; ++q) acc[c & 1][q] = fma(lv, ys[c * KQ + q], acc[c & 1][q]);
            }
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                T a = acc[0][q] + acc[1][q];
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                if (gpart == 0) x[((size_t)I * NS_SB + gr) * KQ + q] -= a;
            }
            issue_tile(it + nslots - 1);
        }
        ++it;
    };
    // named barrier of the GEMV threads (warps 0-7)
    auto gsync = [&]() {
        if (gthread) asm volatile("bar.sync 1, %0;" ::"n"(NS_GT) : "memory");
    };
    // solve the owned diagonal super-block sb in place in x (all GEMV threads: y = D t forward,
    // y = D^T t backward, D the block's inverse), then broadcast it to the other ranks
    auto solve_diag = [&](int sb, int dir) {
        gsync();  // the block's rows, updated by all GEMV threads, are final
        const T* dd = diag + (size_t)((sb - (int)rank) / (int)cs) * L::DIAG;
        T* xs = x + (size_t)sb * NS_SB * KQ;
        T acc[KQ];
        if (gthread) {
#pragma unroll
            for (int q = 0; q < KQ; ++q) acc[q] = 0;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int cc = gpart * 16 + c;
                const T d = dir == 0 ? dd[gr * L::P65 + cc] : dd[cc * L::P65 + gr];
#pragma unroll
                for (int q = 0; q < KQ; ++q) acc[q] = fma(d, xs[cc * KQ + q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 1);
                acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 2);
            }
        }
        gsync();  // every read of the old values is done
        if (gthread && gpart == 0)
#pragma unroll
            for (int q = 0; q < KQ; ++q) xs[gr * KQ + q] = acc[q];
        gsync();  // solved values visible to the GEMV threads, which also broadcast them
        // GEMV warp w sends the block to ranks (rank + 1 + w + 8 j) mod cs, 16 bytes per lane and
        // store (only the GEMV warps have passed the barrier above: with a 16-CTA cluster the
        // other warps must not send)
        if (gthread) {
            const uint4* src = reinterpret_cast<const uint4*>(xs);
            for (int pw = warp; pw < (int)cs - 1; pw += NS_GT / 32) {
                const uint32_t peer = (rank + 1 + (uint32_t)pw) % cs;
                const uint32_t rb = ns_mapa(&bars[dir * nsb + sb], peer);
                const uint32_t rx = ns_mapa(xs, peer);
                for (int ch = lane; ch < (int)(NS_SB * KQ * sizeof(T) / 16); ch += 32)
                    ns_st_async_v4(rx + (uint32_t)ch * 16u, rb, src[ch]);
            }
        }
    };
    const auto owner = [&](int sb) { return sb % (int)cs == (int)rank; };
    // ---- forward: a = L^{-1} r.  The owner of sb + 1 solves it right after the tile (sb + 1, sb)
    // that completes it (look-ahead), before the rest of column sb. ----
    if (fwd) {
        if (owner(0)) solve_diag(0, 0);
        for (int sb = 0; sb + 1 < nsb; ++sb) {
            if (!owner(sb)) wait_y(&bars[sb]);
            const int c = seq.owned_after(sb);
            for (int j = 0; j < c; ++j) {
                const int I = tseq[it] >> 16;
                consume(I, sb);
                if (I == sb + 1) solve_diag(I, 0);
            }
        }
    }
    // ---- backward: z = U^{-1} a, the same from the last super-block down ----
    if (bwd) {
        if (owner(nsb - 1)) solve_diag(nsb - 1, 1);
        for (int sb = nsb - 1; sb > 0; --sb) {
            if (!owner(sb)) wait_y(&bars[nsb + sb]);
            const int c = seq.owned_before(sb);
            for (int j = 0; j < c; ++j) {
                const int I = tseq[it] >> 16;
                consume(I, sb);
                if (I == sb - 1) solve_diag(I, 1);
            }
        }
    }
    __syncthreads();
    (void)ok;
    asm volatile("cp.async.wait_all;" ::: "memory");
    // every broadcast addressed to this rank has landed before it may exit
    if (tid == 0)
        for (int sb = 0; sb < nsb; ++sb)
            if (sb % (int)cs != (int)rank)
                for (int d = 0; d < 2; ++d)
                    if ((d == 0 ? fwd : bwd) && !tc::mbar_wait_bounded(&bars[d * nsb + sb], 0, &s_abort, kDefaultWaitNs))
                        set_status(st, DFS_ERR_TIMEOUT);
    __syncthreads();
    // outputs of the owned rows
    for (int j = 0; j < nown; ++j) {
        const int sb = (int)rank + j * (int)cs;
        for (int e = tid; e < NS_SB * KQ; e += NS_THREADS) {
            const int i = sb * NS_SB + e / KQ, q = e % KQ;
            Z[(int64_t)i * ldz + q] = x[(size_t)i * KQ + q];
        }
    }
    ns_cluster_sync();
}

// ---- host side ------------------------------------------------------------------------------

static size_t ns_fixed_bytes(int n_pad, int KQ, int elem, int cs) {
    const int nsb = n_pad / NS_SB;
    const int nown = (nsb + cs - 1) / cs;
    const size_t diag_elems = (size_t)nown * NS_SB * (NS_SB + 1);
    // x, own diagonal data, alignment, mbarriers (2 nsb), tile sequence (<= 2 nsb nown entries)
    return (size_t)n_pad * KQ * elem + diag_elems * elem + 16 + (size_t)2 * nsb * 8 + (size_t)2 * nsb * nown * 4;
}
static size_t ns_slot_bytes(int elem) { return (size_t)NS_SB * (NS_SB + 16 / elem) * elem; }

static bool ns_fits(int n_pad, int KQ, int elem, int cs, size_t smem_limit) {
    return ns_fixed_bytes(n_pad, KQ, elem, cs) + 8192 + 2 * ns_slot_bytes(elem) <= smem_limit;
}

// Cluster size: up to 8 CTAs (portable); 16 (a non-portable cluster, 7 of which fit on a GB300)
// when the owned diagonal inverses of 8 ranks do not fit in shared memory (n_pad > 4608 in FP32).
int nspace_cluster_size(int n_pad, int KQ, int elem, size_t smem_limit) {
    const int nsb = n_pad / NS_SB;
    const int cs = nsb < NS_MAX_CS ? nsb : NS_MAX_CS;
    if (ns_fits(n_pad, KQ, elem, cs, smem_limit) || nsb < 2 * NS_MAX_CS) return cs;
    return ns_fits(n_pad, KQ, elem, 2 * NS_MAX_CS, smem_limit) ? 2 * NS_MAX_CS : cs;
}

// Ring slots that fit (0: the cluster form does not apply).
int nspace_slots(int n_pad, int KQ, int elem, size_t smem_limit) {
    if (n_pad % NS_SB != 0 || n_pad < NS_SB) return 0;
    const int cs = nspace_cluster_size(n_pad, KQ, elem, smem_limit);
    const size_t fixed = ns_fixed_bytes(n_pad, KQ, elem, cs) + 8192;  // + static shared memory
    if (fixed + 2 * ns_slot_bytes(elem) > smem_limit) return 0;
    size_t s = (smem_limit - fixed) / ns_slot_bytes(elem);
    return s > (size_t)NS_MAX_SLOTS ? NS_MAX_SLOTS : (int)s;
}

template <typename T, int KQ>
static cudaError_t launch_ns_t(const void* W, int64_t ld, int n_pad, const void* Linv, int mode, const double* Rpart,
                               int nparts, int n, int k, const double* Y, double lambda, const void* B, int64_t ldb,
                               double* R, void* Z, int64_t ldz, const double* U2part, double* U2, int nslots,
                               int cs, DevStatus* st, int honor_stop, cudaStream_t stream) {
    const size_t smem = (size_t)nslots * ns_slot_bytes(sizeof(T)) + ns_fixed_bytes(n_pad, KQ, sizeof(T), cs);
    auto kern = nspace_kernel<T, KQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > NS_MAX_CS && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                              cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(NS_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, static_cast<const T*>(W), ld, n_pad, static_cast<const T*>(Linv), mode, Rpart,
                           nparts, n, k, Y, lambda, static_cast<const T*>(B), ldb, R, static_cast<T*>(Z), ldz, U2part,
                           U2, nslots, st, honor_stop);
    count_launch();
    return e;
}

cudaError_t launch_nspace(int f64, int kq, const void* W, int64_t ld, int n_pad, const void* Linv, int mode,
                          const double* Rpart, int nparts, int n, int k, const double* Y, double lambda, const void* B,
                          int64_t ldb, double* R, void* Z, int64_t ldz, const double* U2part, double* U2,
                          size_t smem_limit, DevStatus* st, int honor_stop, cudaStream_t stream) {
    const int nslots = nspace_slots(n_pad, kq, f64 ? 8 : 4, smem_limit);
    if (nslots < 2) return cudaErrorInvalidValue;
    const int cs = nspace_cluster_size(n_pad, kq, f64 ? 8 : 4, smem_limit);
#define DFS_NS(KQ)                                                                                                 \
    case KQ:                                                                                                       \
        return f64 ? launch_ns_t<double, KQ>(W, ld, n_pad, Linv, mode, Rpart, nparts, n, k, Y, lambda, B, ldb, R, \
                                             Z, ldz, U2part, U2, nslots, cs, st, honor_stop, stream)                  \
                   : launch_ns_t<float, KQ>(W, ld, n_pad, Linv, mode, Rpart, nparts, n, k, Y, lambda, B, ldb, R,  \
                                            Z, ldz, U2part, U2, nslots, cs, st, honor_stop, stream);
    switch (kq) {
        DFS_NS(1)
        DFS_NS(2)
        DFS_NS(4)
        DFS_NS(8)
        default:
            return cudaErrorInvalidValue;
    }
#undef DFS_NS
}

}  // namespace dfs
