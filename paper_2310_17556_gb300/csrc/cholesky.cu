// Algorithm 1, Cholesky: L = Chol(W), W = L L^T, L lower triangular with a positive diagonal.
//
// Blocked right-looking factorisation of the padded n_pad x n_pad matrix W (row-major, lower
// triangle) in NB x NB tiles, as ONE persistent cooperative kernel (one CTA per SM, every CTA
// resident; two per SM when they fit, so that one CTA's L2 round trips overlap the other's work).
// Tile t = (i, p), i >= p, t = i (i + 1) / 2 + p, is owned by CTA t mod G for the whole
// factorisation.  Step j applies column block j to the trailing matrix:
//   A[i, p] -= P_i P_p^T,   P_i = A[i, j] Linv_j^T   (panel TRSM, recomputed where needed)
// for all i >= p > j.  The panels A[i, j] stay unscaled while the steps run (so no tile is read
// after its owner overwrote it) and are scaled in place once every CTA has finished; that last
// pass also writes U = L^T into the (otherwise unused) upper triangle for the backward solve.
// Dependencies are tracked per tile instead of with grid-wide barriers:
//   done[t]   tile t = (i, p) has received its last update (after step p - 1);
//   diag[j]   diagonal block j is factored: L_jj written and Linv_j = L_jj^{-1} published.
// Within a step a CTA first updates its tiles of column j + 1 (the next panel); the owner of
// diagonal tile j + 1 fetches that tile and panel tile (j + 1, j) before diagonal block j is
// published, then applies the last update and factors block j + 1 at once, so the factor of the
// next block overlaps the rest of step j's trailing update (look-ahead).
// Each diagonal block is factored by one warp with the block's rows in registers, in the
// compute type CT (double: the FP64 diagonal panel; float: the fast variant).  Its inverse (all
// 8 warps, 4 columns each) feeds the panel TRSM and the triangular solves.
// Every wait is bounded (DFS_ERR_TIMEOUT after 2 s) and also ends when another CTA has set an
// error status: a pivot <= 0 (DFS_ERR_NOT_SPD) or NaN/Inf (DFS_ERR_NONFINITE) with its index.
#define DFS_SRC_ID 5
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dfs {

constexpr int NB = 32;
constexpr int CC_THREADS = 256;

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits (acquire) until *f >= target.  Block-uniform result: false when the device
// status is or becomes non-zero, or after the call's wait limit (then DFS_ERR_TIMEOUT is recorded).
// Contains a __syncthreads().
__device__ bool block_wait(const int* f, int target, DevStatus* st, int* s_ok, int sleep_ns) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_gpu(f) < target) {
            const volatile int* vs = &st->status;
            const uint64_t limit_ns = wait_limit(st);
            const uint64_t t0 = tc::globaltimer_ns();
            for (;;) {
                if (ld_acquire_gpu(f) >= target) break;
                if (*vs != 0) {
                    ok = 0;
                    break;
                }
                if (tc::globaltimer_ns() - t0 > limit_ns) {
                    set_status(st, DFS_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (sleep_ns) __nanosleep(sleep_ns);
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Publish this CTA's global writes: after the barrier, thread 0 fences (cumulative over the
// writes the barrier ordered before it) and sets *f = 1 with a release store.
__device__ __forceinline__ void block_publish(int* f) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_gpu(f, 1);
    }
}

__device__ __forceinline__ void tile_ij(int t, int& i, int& p) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    i = r;
    p = t - r * (r + 1) / 2;
}
__device__ __forceinline__ int tile_id(int i, int p) { return i * (i + 1) / 2 + p; }


// 1/sqrt(d): FP32 hardware estimate, then (FP64) two Newton steps r <- r (3 - d r^2) / 2, each
// doubling the correct bits (~2^-22 -> 2^-44 -> below FP64 rounding): a short dependent chain.
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

// dst(r, c, v) receives L^{-1} (zeros above the diagonal) for the lower-triangular L in sF,
// with s_rinv[i] = 1 / L[i][i].  Needs 256 threads: warp w forms columns c = w + 8 u (u < 4) of
// X = L^{-1} by forward substitution on L x = e_c, lane i holding x_i; the four chains are
// interleaved.  Arithmetic in T.
template <typename T, typename CT, typename D>
__device__ __forceinline__ void invert_lower_32(const CT (*sF)[NB + 1], const T* s_rinv, D&& dst) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = (lane == warp + 8 * u) ? (T)1 : (T)0;
#pragma unroll
    for (int p = 0; p < NB; ++p) {
        const T rp = s_rinv[p];
        const T lip = (T)sF[lane][p];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (lane == p) x[u] *= rp;
            const T xp = __shfl_sync(0xffffffffu, x[u], p);
            if (lane > p) x[u] = fma(-lip, xp, x[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = warp + 8 * u;
        dst(lane, c, (lane >= c) ? x[u] : (T)0);
    }
}

// Factor diagonal block kb, whose updated entries (lower triangle) are in sF; all threads of the
// CTA call it.  Warp 0: lane i holds row i in registers; for each column j every lane scales its
// entry by the broadcast 1/sqrt(pivot), the scaled column goes through a shared-memory vector
// (double-buffered by column parity, read by all lanes at one address: no bank conflicts, no
// shuffle latency per entry), and every lane applies the rank-1 update to its entries right of
// column j.  Lane j + 1 forms the next pivot from its own scaled entry and it is broadcast before
// the update runs, so the dependent chain per column is one shuffle, one rsqrt and two
// multiply-adds.  L_kb goes back to sF; then all threads store it to W (coalesced) and form
// Linv_kb (4 columns per warp, forward substitution on L x = e_c with the 4 chains interleaved)
// into sX, stored to Linv (coalesced).  Returns false (uniformly) on a bad pivot, after recording it.
template <typename T, typename CT>
__device__ __noinline__ bool factor_diag(T* W, int64_t ld, int kb, T* Linv, DevStatus* st, CT (*sF)[NB + 1],
                                         T (*sX)[NB + 1], T* s_rinv, int* s_fail, CT (*sCol)[NB]) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t o = (int64_t)kb * NB;
    if (warp == 0) {
        CT a[NB];
#pragma unroll
        for (int p = 0; p < NB; ++p) a[p] = (p <= lane) ? sF[lane][p] : (CT)0;
        int fail = -1;
        CT d = __shfl_sync(0xffffffffu, a[0], 0);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (fail == -1 && (!(d > (CT)0) || !isfinite(d))) fail = isfinite(d) ? j : -2 - j;  // the first bad pivot
            const CT r = rsqrt_ct(d);
            const CT l = a[j] * r;
            a[j] = (lane >= j) ? l : (CT)0;
            sCol[j & 1][lane] = l;
            // lane j + 1's pivot after this column (the same multiply-add its own update does),
            // broadcast before the update
            if (j + 1 < NB) d = __shfl_sync(0xffffffffu, fma(-l, l, a[j + 1]), j + 1);
            __syncwarp();
            // constant trip count (fully unrolled, a[] stays in registers); p <= j is skipped.  The
            // entries above the diagonal (lane < p) take the update too: they are never read back
            // (the factor reads p <= lane, W and the inverse only the lower triangle, and a column
            // broadcast through sCol is read at p > j only), so no mask is needed
#pragma unroll
            for (int p = 0; p < NB; ++p) {
                if (p > j) a[p] = fma(-l, sCol[j & 1][p], a[p]);
            }
        }
        if (lane == 0) *s_fail = fail;
        if (fail == -1) {
            // a[lane] by an unrolled select: a dynamic index would move all of a[] to local memory
            CT dl = (CT)0;
#pragma unroll
            for (int p = 0; p < NB; ++p) {
                sF[lane][p] = a[p];
                if (p == lane) dl = a[p];
            }
            s_rinv[lane] = (T)1 / (T)dl;
        }
    }
    __syncthreads();
    const int fail = *s_fail;
    if (fail != -1) {
        if (tid == 0) {
            const int j = fail >= 0 ? fail : -2 - fail;
            set_status(st, fail >= 0 ? DFS_ERR_NOT_SPD : DFS_ERR_NONFINITE);
            atomicCAS(&st->failed_pivot, -1, (int)(o + j));
        }
        return false;
    }
#pragma unroll
    for (int u = 0; u < NB * NB / CC_THREADS; ++u) {
        const int e = tid + u * CC_THREADS, r = e / NB, c = e % NB;
        if (c <= r) W[(o + r) * ld + o + c] = (T)sF[r][c];
    }
    invert_lower_32<T, CT>(sF, s_rinv, [&](int r, int c, T v) { sX[r][c] = v; });
    __syncthreads();
    T* dst = Linv + (int64_t)kb * NB * NB;
#pragma unroll
    for (int u = 0; u < NB * NB / CC_THREADS; ++u) {
        const int e = tid + u * CC_THREADS;
        dst[e] = sX[e / NB][e % NB];
    }
    return true;
}

// s = the NB x NB tile of W at (r0, c0) (L2 loads: other CTAs wrote it)
template <typename T>
__device__ __forceinline__ void load_tile(const T* W, int64_t ld, int64_t r0, int64_t c0, T (*s)[NB + 1]) {
#pragma unroll
    for (int u = 0; u < NB * NB / CC_THREADS; ++u) {
        const int e = threadIdx.x + u * CC_THREADS;
        s[e / NB][e % NB] = __ldcg(W + (r0 + e / NB) * ld + c0 + e % NB);
    }
}

// sA <- sA Linv^T in place: sA[r][c] = sum_q A[r][q] Li[c][q] (Li lower triangular, zeros above
// the diagonal).  Thread: row tid / 8, columns tid % 8 + 8 u.  Starts and ends with a barrier.
template <typename T>
__device__ __forceinline__ void times_linv_t(T (*sA)[NB + 1], const T (*sLi)[NB + 1]) {
    const int tid = threadIdx.x;
    __syncthreads();
    const int r = tid >> 3, c = tid & 7;
    T acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const T a = sA[r][q];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(a, sLi[c + 8 * u][q], acc[u]);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) sA[r][c + 8 * u] = acc[u];
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void load_linv(const T* Linv, int kb, T (*sLi)[NB + 1]) {
#pragma unroll
    for (int u = 0; u < NB * NB / CC_THREADS; ++u) {
        const int e = threadIdx.x + u * CC_THREADS;
        sLi[e / NB][e % NB] = __ldcg(Linv + (int64_t)kb * NB * NB + e);
    }
    __syncthreads();
}

// Lane 0 waits (acquire) until *f >= target, as block_wait but for one warp; warp-uniform result.
__device__ bool warp_wait(const int* f, int target, DevStatus* st) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0 && ld_acquire_gpu(f) < target) {
        const volatile int* vs = &st->status;
        const uint64_t limit_ns = wait_limit(st);
        const uint64_t t0 = tc::globaltimer_ns();
        for (;;) {
            if (ld_acquire_gpu(f) >= target) break;
            if (*vs != 0) {
                ok = 0;
                break;
            }
            if (tc::globaltimer_ns() - t0 > limit_ns) {
                set_status(st, DFS_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();  // the other lanes' reads come after lane 0's acquire
    return ok != 0;
}

// Warp-private tiles of the trailing update, rows padded to a multiple of 4 (16-byte row loads).
constexpr int WT_LD = NB + 4;
constexpr int CC_WARPS = CC_THREADS / 32;
constexpr size_t CC_WARP_SMEM = (size_t)CC_WARPS * 2 * NB * WT_LD * sizeof(float);

// sum_q a[q] b[q] over 32 terms, in order: a is a shared-memory row read as 16-byte broadcasts,
// b is in registers.
__device__ __forceinline__ float warp_dot32(const float* a, const float (&b)[NB]) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < NB; q += 4) {
        const float4 x = *reinterpret_cast<const float4*>(a + q);
        s = fmaf(x.x, b[q], s);
        s = fmaf(x.y, b[q + 1], s);
        s = fmaf(x.z, b[q + 2], s);
        s = fmaf(x.w, b[q + 3], s);
    }
    return s;
}

// sOut <- sA Li^T for one warp (FP32; sOut may be sA): lane c forms column c,
// acc[r] = sum_q A[r][q] Li[c][q], with Li's row c in registers and A's rows read as 16-byte
// broadcasts (warp_dot32).
__device__ __forceinline__ void warp_times_linv_t(const float (*sA)[WT_LD], const float (*sLi)[NB + 1],
                                                  float (*sOut)[WT_LD]) {
    const int lane = threadIdx.x & 31;
    float li[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) li[q] = sLi[lane][q];
    float acc[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) acc[r] = warp_dot32(&sA[r][0], li);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < NB; ++r) sOut[r][lane] = acc[r];
    __syncwarp();
}

// One tile of the trailing update by one warp (FP32 W): A[i, p] -= P_i P_p^T with P = A[., j]
// Linv_j^T, evaluated as (A[i, j] M_j) A[p, j]^T with M_j = Linv_j^T Linv_j (the inverse of the
// factored diagonal block, formed once per step by the CTA), so a tile costs two 32^3 products
// instead of three.  Waits for tiles (i, j) and (p, j) first.  Used for the tiles of columns
// beyond j + 1 (no flag to publish: their last update comes in a later step).  The two panel
// tiles come in with 16-byte asynchronous copies (all in flight at once), and the target tile's
// 32 rows are loaded together before it is written back.  Lane c owns column c of the tile: its
// loads and stores of W are whole 128-byte rows.  Returns false when a wait gave up (the device
// status says why).
__device__ bool warp_tile_update(float* W, int64_t ld, int j, int i, int p, const float (*sM)[NB + 1],
                                 float (*sPw)[WT_LD], float (*sQw)[WT_LD], const int* done, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    if (j > 0) {
        if (!warp_wait(&done[tile_id(i, j)], 1, st)) return false;
        if (p != i && !warp_wait(&done[tile_id(p, j)], 1, st)) return false;
    }
    const int64_t c0 = (int64_t)j * NB;
    // 32 rows x 8 chunks of 16 bytes per tile: lane takes chunk lane % 8 of rows lane / 8 + 4 u
#pragma unroll
    for (int u = 0; u < NB / 4; ++u) {
        const int r = (lane >> 3) + 4 * u, ch = lane & 7;
        const float* gp = W + ((int64_t)i * NB + r) * ld + c0 + 4 * ch;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&sPw[r][4 * ch]))), "l"(gp) : "memory");
        if (p != i) {
            const float* gq = W + ((int64_t)p * NB + r) * ld + c0 + 4 * ch;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             static_cast<uint32_t>(__cvta_generic_to_shared(&sQw[r][4 * ch]))), "l"(gq) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    // T = A[i, j] M_j (M_j symmetric: its row c is its column c), in place, or into the unused
    // second buffer on a diagonal tile, whose unscaled rows are the other operand
    float(*sT)[WT_LD] = (p != i) ? sPw : sQw;
    float(*sB)[WT_LD] = (p != i) ? sQw : sPw;  // A[p, j], unscaled: M_j carries both solves
    warp_times_linv_t(sPw, sM, sT);
    float qrow[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) qrow[q] = sB[lane][q];
    __syncwarp();  // every lane holds its row of A[p, j]: sB takes the product
    // D[r][lane] = sum_q T[r][q] A_p[lane][q]
#pragma unroll 4
    for (int r = 0; r < NB; ++r) sB[r][lane] = warp_dot32(&sT[r][0], qrow);
    // A[i, p] -= D: the target tile's column `lane`, all rows in flight at once
    float wv[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) wv[r] = __ldcg(W + ((int64_t)i * NB + r) * ld + (int64_t)p * NB + lane);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (i == p && lane > r) continue;
        if (!DFS_IN_BOUNDS(st, p <= i)) continue;
        W[((int64_t)i * NB + r) * ld + (int64_t)p * NB + lane] = wv[r] - sB[r][lane];
    }
    __syncwarp();  // sPw / sQw are reused by the warp's next tile
    return true;
}

// flags (int32, zeroed before the launch): diag[nb] | done[nb (nb + 1) / 2] | finished-CTA count
template <typename T, typename CT, bool WARP_TILES>
__global__ void __launch_bounds__(CC_THREADS)
chol_coop_kernel(T* W, int64_t ld, int nb, T* Linv, int* flags, DevStatus* st) {
    __shared__ __align__(16) T sLi[NB][NB + 1];
    __shared__ __align__(16) T sM[WARP_TILES ? NB : 1][NB + 1];  // Linv_j^T Linv_j (warp-tile steps)
    __shared__ __align__(16) T sP[NB][NB + 1];
    __shared__ __align__(16) T sQ[NB][NB + 1];
    __shared__ __align__(16) T sD[NB][NB + 1];  // the next diagonal tile (owner only), before its update
    __shared__ __align__(16) CT sF[NB][NB + 1];
    __shared__ __align__(16) CT sCol[2][NB];
    __shared__ T s_rinv[NB];
    __shared__ int s_ok, s_fail;
    // WARP_TILES (FP32 W and FP32 diagonal blocks, n >= 2048): the bulk of each step's trailing
    // update (tiles of columns beyond j + 1) runs one tile per warp, 8 tiles at once per CTA, in
    // warp-private tiles (dynamic shared memory); column j + 1, on the critical path, keeps the
    // whole CTA per tile.  Below 2048 rows a CTA rarely has three such tiles in a step, and the
    // kernel without them (fewer registers, no dynamic shared memory) is the faster one.
    constexpr bool kWarpTiles = WARP_TILES && sizeof(T) == 4 && sizeof(CT) == 4;
    extern __shared__ __align__(16) float wtiles[];  // [warp][P | Q][NB][WT_LD] (FP32 W only)
    if (block_should_exit(st, 0)) return;
    // every tile of the nb x nb block grid lies inside W's rows of ld elements (uniform over the
    // grid: all CTAs return alike)
    if (!DFS_IN_BOUNDS(st, ld >= (int64_t)nb * NB)) return;
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const int fault = test_fault(st);  // the test hook, read once
    const int ntiles = nb * (nb + 1) / 2;
    int* diag = flags;
    int* done = flags + nb;
    int* fin = flags + nb + ntiles;

    if (tile_id(0, 0) % G == cta) {
        load_tile<T>(W, ld, 0, 0, sD);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NB * NB / CC_THREADS; ++u) {
            const int e = tid + u * CC_THREADS;
            sF[e / NB][e % NB] = (CT)sD[e / NB][e % NB];
        }
        __syncthreads();
        if (!factor_diag<T, CT>(W, ld, 0, Linv, st, sF, sQ, s_rinv, &s_fail, sCol)) return;
        block_publish(&diag[0]);
    }
    int last_p = -1;  // the largest column index among this CTA's tiles: no work after step last_p - 1
    for (int t = cta; t < ntiles; t += G) {
        int i, p;
        tile_ij(t, i, p);
        last_p = p > last_p ? p : last_p;
    }
    for (int j = 0; j + 1 < nb && j < last_p; ++j) {
        // The owner of the next diagonal tile (j + 1, j + 1) is on the critical path: it fetches
        // that tile and the panel tile (j + 1, j) before it waits for diagonal block j.
        const bool diag_owner = tile_id(j + 1, j + 1) % G == cta;
        if (diag_owner) {
            if (j > 0 && !block_wait(&done[tile_id(j + 1, j)], 1, st, &s_ok, 0)) return;
            load_tile<T>(W, ld, (int64_t)(j + 1) * NB, (int64_t)j * NB, sP);
            load_tile<T>(W, ld, (int64_t)(j + 1) * NB, (int64_t)(j + 1) * NB, sD);
        }
        if (!block_wait(&diag[j], 1, st, &s_ok, 0)) return;
        load_linv<T>(Linv, j, sLi);
        if constexpr (kWarpTiles) {
            // M_j = Linv_j^T Linv_j = (L_jj L_jj^T)^{-1} for this step's per-warp tiles:
            // M[r][c] = sum_q Li[q][r] Li[q][c] (Li lower triangular: q >= max(r, c))
            const int r = tid >> 3, cb = tid & 7;
            T acc[4] = {0, 0, 0, 0};
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const T a = sLi[q][r];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(a, sLi[q][cb + 8 * u], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) sM[r][cb + 8 * u] = acc[u];
            __syncthreads();
        }
        // pass 0: tiles of column j + 1 (diagonal first: it has the smallest id); pass 1: the rest
        for (int pass = 0; pass < 2; ++pass) {
            // With three or more tiles in the pass (large n), they are dealt to the CTA's warps (a
            // warp takes about twice as long over a tile as the whole CTA, but eight run at once);
            // with fewer (small n, where the step's latency matters more than its throughput) the
            // whole CTA takes one tile at a time, as for column j + 1.
            int npass1 = 0;
            if (kWarpTiles && pass == 1) {
                for (int t = cta; t < ntiles; t += G) {
                    int i, p;
                    tile_ij(t, i, p);
                    npass1 += p > j + 1;
                }
            }
            if (kWarpTiles && pass == 1 && npass1 >= 3) {
                // the CTA's tiles of the pass dealt to its warps in order, one tile per warp at a time
                const int warp = tid >> 5;
                float (*sPw)[WT_LD] = reinterpret_cast<float (*)[WT_LD]>(wtiles + (size_t)warp * 2 * NB * WT_LD);
                float (*sQw)[WT_LD] = sPw + NB;
                const float(*sMf)[NB + 1] = reinterpret_cast<const float(*)[NB + 1]>(sM);
                int kk = 0;
                for (int t = cta; t < ntiles; t += G) {
                    int i, p;
                    tile_ij(t, i, p);
                    if (p <= j + 1) continue;
                    if ((kk++ % CC_WARPS) != warp) continue;
                    // a wait that gave up leaves the rest to the next block_wait, which sees the status
                    if (!warp_tile_update(reinterpret_cast<float*>(W), ld, j, i, p, sMf, sPw, sQw, done, st)) break;
                }
                continue;
            }
            for (int t = cta; t < ntiles; t += G) {
                int i, p;
                tile_ij(t, i, p);
                if (pass == 0 ? (p != j + 1) : (p <= j + 1)) continue;
                const bool is_next_diag = (i == p) && (p == j + 1);
                if (j > 0 && !is_next_diag) {
                    if (!block_wait(&done[tile_id(i, j)], 1, st, &s_ok, 0)) return;
                    if (p != i && !block_wait(&done[tile_id(p, j)], 1, st, &s_ok, 0)) return;
                }
                const int64_t c0 = (int64_t)j * NB;
                if (!is_next_diag) {
                    load_tile<T>(W, ld, (int64_t)i * NB, c0, sP);
                    if (p != i) load_tile<T>(W, ld, (int64_t)p * NB, c0, sQ);
                }
                times_linv_t<T>(sP, sLi);
                if (p != i) times_linv_t<T>(sQ, sLi);
                const T(*pq)[NB + 1] = (p != i) ? sQ : sP;
                // A[i, p] -= P_i P_p^T; thread: rows ty + 16 a, columns tx + 16 b
                const int tx = tid & 15, ty = tid >> 4;
                T acc[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    const T a0 = sP[ty][q], a1 = sP[ty + 16][q];
                    const T b0 = pq[tx][q], b1 = pq[tx + 16][q];
                    acc[0][0] = fma(a0, b0, acc[0][0]);
                    acc[0][1] = fma(a0, b1, acc[0][1]);
                    acc[1][0] = fma(a1, b0, acc[1][0]);
                    acc[1][1] = fma(a1, b1, acc[1][1]);
                }
                if (is_next_diag) {
                    // the updated tile goes straight to the factorisation (W gets L from it)
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 2; ++b) {
                            const int r = ty + 16 * a, c = tx + 16 * b;
                            sF[r][c] = (CT)(sD[r][c] - acc[a][b]);
                        }
                    __syncthreads();
                    if (!factor_diag<T, CT>(W, ld, p, Linv, st, sF, sQ, s_rinv, &s_fail, sCol)) return;
                    block_publish(&diag[p]);
                    continue;
                }
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int r = ty + 16 * a, c = tx + 16 * b;
                        if (i == p && c > r) continue;
                        if (!DFS_IN_BOUNDS(st, i < nb && p <= i)) continue;
                        T* w = W + ((int64_t)i * NB + r) * ld + (int64_t)p * NB + c;
                        *w = __ldcg(w) - acc[a][b];
                    }
                if (p == j + 1) {  // the tile's last update
                    if (fault == DFS_TEST_FAULT_CHOLESKY && t == tile_id(2, 1))
                        __syncthreads();  // test hook: this tile's flag is never set, its waiter times out
                    else
                        block_publish(&done[t]);
                } else {
                    __syncthreads();  // sP / sQ are reused by the next tile
                }
            }
        }
    }
    // every CTA has applied all its steps: scale the panels in place, L[i, p] = A[i, p] Linv_p^T
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        atomicAdd(fin, 1);
    }
    if (!block_wait(fin, G, st, &s_ok, 64)) return;
    for (int t = cta; t < ntiles; t += G) {
        int i, p;
        tile_ij(t, i, p);
        if (i == p) continue;
        if (!DFS_IN_BOUNDS(st, i < nb && p < i)) continue;  // (uniform over the CTA)
        load_linv<T>(Linv, p, sLi);
        load_tile<T>(W, ld, (int64_t)i * NB, (int64_t)p * NB, sP);
        times_linv_t<T>(sP, sLi);
#pragma unroll
        for (int u = 0; u < NB * NB / CC_THREADS; ++u) {
            const int e = tid + u * CC_THREADS;
            W[((int64_t)i * NB + e / NB) * ld + (int64_t)p * NB + e % NB] = sP[e / NB][e % NB];
            // U = L^T in the upper triangle: the backward triangular solve streams its rows
            W[((int64_t)p * NB + e / NB) * ld + (int64_t)i * NB + e % NB] = sP[e % NB][e / NB];
        }
        __syncthreads();
    }
}

size_t cholesky_flag_bytes(int64_t n_pad) {
    const int64_t nb = n_pad / NB;
    return (size_t)(nb + nb * (nb + 1) / 2 + 1) * sizeof(int);
}

// Inverses of all diagonal blocks of an existing factor L (for triangular solves with a
// caller-supplied L).  A zero or non-finite diagonal entry sets DFS_ERR_INVALID_ARG.
template <typename T>
__global__ void __launch_bounds__(256) diag_inverse_kernel(const T* L, int64_t ld, T* Linv, DevStatus* st) {
    __shared__ T a[NB][NB + 1];
    __shared__ T rinv[NB];
    __shared__ int bad;
    const int kb = blockIdx.x;
    const int64_t o = (int64_t)kb * NB;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        const T v = (j <= i) ? L[(o + i) * ld + o + j] : (T)0;
        a[i][j] = v;
        if (i == j) {
            if (!(v != (T)0) || !isfinite(v)) atomicExch(&bad, 1);
            rinv[i] = (T)1 / v;
        }
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) set_status(st, DFS_ERR_INVALID_ARG);
        return;
    }
    T* dst = Linv + (int64_t)kb * NB * NB;
    invert_lower_32<T, T>(a, rinv, [&](int r, int c, T v) { dst[r * NB + c] = v; });
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
static cudaError_t launch_cholesky_t(void* W_, int64_t ld, int64_t n_pad, void* Linv_, int* flags, DevStatus* st,
                                     cudaStream_t stream, int share) {
    T* W = static_cast<T*>(W_);
    T* Linv = static_cast<T*>(Linv_);
    int nb = (int)(n_pad / NB);
    const int ntiles = nb * (nb + 1) / 2;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const bool warp_tiles = sizeof(T) == 4 && sizeof(CT) == 4 && nb >= 64;
    auto kern = warp_tiles ? chol_coop_kernel<T, CT, true> : chol_coop_kernel<T, CT, false>;
    const size_t dsmem = warp_tiles ? CC_WARP_SMEM : 0;  // warp tiles of the FP32 trailing update
    if (dsmem && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CC_THREADS, dsmem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // two CTAs per SM where they fit (all resident): a CTA waiting on an L2 round trip leaves the
    // SM to the other
    int G = sms * (per_sm >= 2 ? 2 : 1);
    // concurrent factorisations (share > 1) each take 1 / share of that capacity, so all of their
    // CTAs can be resident together and none waits for another's to leave
    if (share > 1) G = G / share > 0 ? G / share : 1;
    if (G > ntiles) G = ntiles;
    if ((e = cudaMemsetAsync(flags, 0, cholesky_flag_bytes(n_pad), stream)) != cudaSuccess) return e;
    void* args[] = {&W, &ld, &nb, &Linv, &flags, &st};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(CC_THREADS), args, dsmem, stream);
    count_launch();
    return e;
}

cudaError_t launch_cholesky(int w_f64, void* W, int64_t ld, int64_t n_pad, void* Linv, int* flags, DevStatus* st,
                            cudaStream_t stream, int fp64_panel, int share) {
    if (n_pad % NB != 0) return cudaErrorInvalidValue;
    if (w_f64) return launch_cholesky_t<double, double>(W, ld, n_pad, Linv, flags, st, stream, share);
    return fp64_panel ? launch_cholesky_t<float, double>(W, ld, n_pad, Linv, flags, st, stream, share)
                      : launch_cholesky_t<float, float>(W, ld, n_pad, Linv, flags, st, stream, share);
}

}  // namespace dfs
