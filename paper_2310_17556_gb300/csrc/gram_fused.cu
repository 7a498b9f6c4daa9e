// The first pass over FP32 S of Algorithm 1 as one kernel: b = S V (the rightmost product of
// S^T L^{-T} L^{-1} S v, Section 2), the BF16 tensor-core tiles of S, and the Gram partial blocks
// of W = S S^T (lower triangle, the O(n^2 m) contraction Section 2 names as the dominant cost) on
// tcgen05, overlapped on every SM so that the HBM stream of S and the tensor cores run at once.
//
// One cooperative, persistent launch with one CTA per SM.  Per CTA (512 threads, four warpgroups):
//   warp 0      tile producer: per k-step of its Gram task, checks (a window of relaxed loads and
//               one acquire fence) that every tile of the k-block has been written (a per-k-block
//               ready count in global memory), then bulk-copies the unit's 2-4 BF16 tiles (16 KB
//               each, still in L2) into a 3-stage ring of 64 KB stages;
//   warp 1      MMA issuer: tcgen05.mma kind::f16, two M = 128 x N = 256 chains sharing B, FP32
//               accumulators in all 512 TMEM columns (as gram_tc_kernel);
//   warp 2      signaler: publishes each converted tile to the other CTAs (a gpu-scope fence and
//               an add to the k-block's ready count), so that the converter threads, which keep
//               the loads of their next items in flight, never execute a fence (a fence would
//               wait for those loads and collapse their pipeline);
//   warps 4-7   epilogue: tcgen05.ld of the accumulators (TMEM lane quarter warp % 4), 16-byte
//               stores of the partial block;
//   warps 8-15  converters: read FP32 S in 128-row x 64-column items (one BF16 tile of one
//               k-block each), store the tile (round to nearest even, 128-byte swizzled K-major
//               layout, the layout the MMA descriptors read), and add each row's dot products with
//               V to FP32 row sums held in registers.  After an item's stores they arrive at a
//               named barrier the signaler waits on (barriers do not wait for loads in flight), in
//               FU_SLOTS rotating slots, each freed again by the signaler.  The signaler publishes
//               the items in groups of FU_PUB, one fence per group.  A prefetch to L2 runs a
//               few items ahead of their loads.
// The kernel is launched at 128 registers a thread and the warpgroups re-divide them
// (setmaxnreg): the converters take 184, enough for three items of loads in flight.
//
// Schedule.  The lower triangle is covered by the quad units of gram_tc_kernel (U units, each two
// 128-row blocks against two).  Every unit has c = w G strided slots: slot s takes the k-blocks
// s, s + c, s + 2c, ...  CTA gi (gi < U w) runs unit gi mod U, slot group sg = gi / U, and its G
// tasks t = 0 .. G-1 take slot sg + t w; the G tasks add into one FP32 partial block (each task
// is its own FP32 accumulation chain of at most 1024 k-blocks).  At step tau = t NK + j
// (NK = ceil(nkb / c)) the whole grid consumes the w contiguous k-blocks t w + j c + [0, w): one
// narrow window of m, kappa = tau w + sg in consumption order.  The converters produce the same
// k-blocks in the same order: with Q = grid / T, CTA b < Q T converts row tile I = b mod T of the
// k-blocks kappa = b / T, b / T + Q, b / T + 2Q, ...; its threads' rows never change, so b = S V
// accumulates in registers.  A converter does not start an item more than `lead` steps (kLead
// plus the span of its load pipeline) ahead of its own CTA's producer, which keeps the
// written-but-unread tiles (a few MB) in L2 and bounds how far the two roles drift apart.
//
// Progress.  All CTAs are co-resident (cooperative launch).  A producer waiting at step tau needs
// only items of step tau, and a converter is held back only while it is more than `lead` steps
// ahead of a producer that has work left, with none of the items whose loads it holds (or that
// it wrote and whose publication group is still open) needed before then; so the item of the
// smallest unfinished step can always be converted and published, and every wait ends.  Every wait is still bounded (2 s); on a timeout the CTA records DFS_ERR_TIMEOUT,
// stops its roles, waits for its copies and MMAs in flight and frees TMEM.
//
// b: converter CTA (I, q) writes rows I * 128 ... of partial q of Rpart (Q partials of n x KQ
// FP64, each row added in a fixed order by one thread), which pass_reduce / the n-space kernel sum
// in partial order, so b is deterministic.
#define DFS_SRC_ID 4
#include <climits>

#include "gram_tc.cuh"

namespace dfs {

namespace {

constexpr int FU_CONV_WARPS = 8;
constexpr int FU_CONV_THREADS = FU_CONV_WARPS * 32;
constexpr int FU_ROW_STEP = FU_CONV_WARPS * 4;      // rows of an item one load instruction step covers
constexpr int FU_RPT = TC_BM / FU_ROW_STEP;         // rows of an item per converter thread
// Warp roles, four warpgroups: 0 producer, 1 MMA issuer, 2 signaler, 3 idle | 4-7 epilogue (TMEM lane
// quarter warp % 4) | 8-15 converters.  Launched at 128 registers a thread; the warpgroups then
// re-divide them (setmaxnreg): 64 for warpgroup 0, 80 for the epilogue, 184 for the converters,
// 128 (64 + 80) + 256 x 184 = 65536 = 512 x 128 in all.
constexpr int FU_SIG_WARP = 2;
constexpr int FU_FIRST_EPI_WARP = 4;
constexpr int FU_FIRST_CONV_WARP = 8;
constexpr int FU_THREADS = FU_FIRST_CONV_WARP * 32 + FU_CONV_THREADS;
constexpr int FU_LAUNCH_REGS = 128;
constexpr int FU_REGS_WG0 = 64, FU_REGS_EPI = 80, FU_REGS_CONV = 184;
static_assert(128 * (FU_REGS_WG0 + FU_REGS_EPI) + FU_CONV_THREADS * FU_REGS_CONV <= FU_THREADS * FU_LAUNCH_REGS,
              "the register split must fit the launch's registers");
// Items the signaler publishes per gpu-scope fence (a fence waits for the stores it covers to
// reach L2; one fence per item held the converters back: 1.456 -> 1.442 ms at n=1024, m=2^20).
constexpr int FU_PUB = 4;
constexpr int FU_SLOTS = FU_PUB > 2 ? FU_PUB : 2;        // items a converter may run ahead of the signaler
// named barriers: 1 = converters' start; 2 .. 2 + FU_SLOTS - 1 = item written (converters arrive,
// the signaler waits); the next FU_SLOTS = slot free again (the signaler arrives, converters wait)
constexpr int FU_BAR_START = 1, FU_BAR_FULL = 2, FU_BAR_EMPTY = 2 + FU_SLOTS;
static_assert(FU_BAR_EMPTY + FU_SLOTS <= 16, "named barrier ids");
constexpr bool kVAtIssue(int kq) { return kq == 1; }  // V loaded with the item (else when converted)
constexpr int FU_HANDSHAKE = FU_CONV_THREADS + 32;
constexpr int FU_FLAG_WINDOW = 8;  // ready counts the producer reads ahead at once
// Items ahead of the one being converted whose lines a converter pulls into L2 (prefetch: no
// registers, no shared memory), so that its own loads, a couple of items ahead, hit L2: the HBM
// stream then has about FU_PREFETCH x 32 KB in flight per SM.
constexpr int FU_PREFETCH = 5;
constexpr int kFoldItems = 16;  // items between FP64 folds of a converter's FP32 row sums
constexpr int FU_ITEM_COLS = 64;  // FP32 columns per item (one 128-byte BF16 k-block row)
// items whose loads a converter thread keeps in registers: the one being converted and the next
// two (the L2 prefetch covers the HBM latency; the converters hold 184 registers a thread)
__host__ __device__ constexpr int fu_depth(int kq) { return kq > 0 ? 3 : 3; }
constexpr int kLead = 12;         // steps a converter may run ahead of its CTA's producer

struct FuSmem {
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t accf;
    uint64_t acce;
    uint64_t done;
    uint32_t tmem_base;
    int abort;
    int never;
    int gram_tau;  // the step the producer is at; INT_MAX once it has no work left
    double rsum[TC_BM * 4];  // the converters' FP64 row sums of b (128 rows x up to 4 right-hand sides)
};

constexpr size_t FU_SMEM_BYTES = 1024 + (size_t)TC_STAGES * TC_STAGE_BYTES + sizeof(FuSmem);

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void red_relaxed_gpu_add(int* p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Wait until *flag >= target (acquire).  Gives up after limit_ns or when the device status or the
// CTA's abort flag is set; returns false then.
__device__ __forceinline__ bool wait_count_bounded(const int* flag, int target, const DevStatus* st,
                                                   volatile int* abort, uint64_t limit_ns) {
    if (ld_acquire_gpu(flag) >= target) return true;
    const uint64_t t0 = tc::globaltimer_ns();
    while (true) {
        __nanosleep(32);
        if (ld_acquire_gpu(flag) >= target) return true;
        if (*abort || *reinterpret_cast<const volatile int*>(&st->status)) return false;
        if (tc::globaltimer_ns() - t0 > limit_ns) return false;
    }
}


// Position kappa = tau w + sg in the consumption order of the k-blocks, walked without divisions:
// tau = t NK + j, k-block sg + t w + j c.
struct FuCursor {
    int tau, sg, t, j;
    __device__ __forceinline__ void init(int kappa, int w, int NK) {
        tau = kappa / w;
        sg = kappa - tau * w;
        t = tau / NK;
        j = tau - t * NK;
    }
    __device__ __forceinline__ int kb(int w, int c) const { return sg + t * w + j * c; }
    __device__ __forceinline__ void advance(int step, int w, int NK) {
        sg += step;
        while (sg >= w) {
            sg -= w;
            ++tau;
            if (++j == NK) {
                j = 0;
                ++t;
            }
        }
    }
};

}  // namespace

// KQ: right-hand sides of b = S V (1, 2 or 4).
template <int KQ>
__global__ void __launch_bounds__(FU_THREADS, 1)
gram_fused_kernel(const float* __restrict__ S, int n, int64_t m, int64_t lds, const float* __restrict__ V,
                  int64_t ldv, int k, int v_vec, double* __restrict__ Rpart, unsigned char* __restrict__ Sp, int T,
                  int U, int w, int G, int NK, int nkb, int lead, float* __restrict__ part,
                  int* __restrict__ ready, DevStatus* st) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* stage_mem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    FuSmem* sm = reinterpret_cast<FuSmem*>(stage_mem + TC_STAGES * TC_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = w * G;
    const int ngroups = U * w;
    const bool has_gram = (int)blockIdx.x < ngroups;
    // converter role: CTA b < Q T converts row tile I = b mod T of the k-blocks q0, q0 + Q, ... of
    // the consumption order kappa = tau w + sg (nslots = w G NK of them, the ones with kb >= nkb
    // are not real)
    const int Q = (int)gridDim.x / T;
    const bool conv = (int)blockIdx.x < Q * T;
    const int I = (int)blockIdx.x % T, q0 = (int)blockIdx.x / T;
    const int nslots = w * G * NK;
    const int my_items = conv && q0 < nslots ? (nslots - 1 - q0) / Q + 1 : 0;

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
        sm->gram_tau = has_gram ? 0 : INT_MAX;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) tc::tmem_alloc(&sm->tmem_base, TC_TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm->tmem_base;
    volatile int* abort = &sm->abort;
    volatile int* never = &sm->never;
    volatile int* gram_tau = &sm->gram_tau;
    const uint64_t wait_ns = wait_limit(st);
    const int fault = test_fault(st);
    // Each warpgroup's branch first re-divides the registers (every warp of a warpgroup takes the
    // same step).
    if (warp < FU_FIRST_EPI_WARP) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(FU_REGS_WG0));
        if (warp == 0) {
            if (lane == 0 && has_gram) {
                // ---------------- tile producer ----------------
                int stage = 0;
                uint32_t phase = 0;
                uint32_t last_parity[TC_STAGES];
                bool issued[TC_STAGES];
                for (int s = 0; s < TC_STAGES; ++s) issued[s] = false;
                bool ok = true;
                const int gi = blockIdx.x;
                int I2, J2;
                tc_unit_ij(gi % U, I2, J2);
                const int sg = gi / U;
                const int i0 = 2 * I2, j0 = 2 * J2;
                const bool diag = J2 == I2;
                const uint32_t bytes = (uint32_t)TC_TILE_BYTES * (diag ? 2u : 4u);
                for (int t = 0; ok && t < G; ++t) {
                    const int slot = sg + t * w;
                    const int nk = slot < nkb ? (nkb - 1 - slot) / c + 1 : 0;
                    int known = 0;  // steps j < known have all their tiles written
                    for (int j = 0; j < nk; ++j) {
                        *gram_tau = t * NK + j;
                        const int64_t kb = slot + (int64_t)j * c;
                        if (!tc::mbar_wait_bounded(&sm->empty[stage], phase ^ 1u, abort, wait_ns)) {
                            ok = false;
                            break;
                        }
                        if (j >= known) {
                            // read the ready counts of the next steps at once (relaxed loads in flight
                            // together, one acquire fence), then wait on the first alone if need be
                            int v[FU_FLAG_WINDOW];
    #pragma unroll
                            for (int q = 0; q < FU_FLAG_WINDOW; ++q)
                                v[q] = j + q < nk ? ld_relaxed_gpu(ready + kb + (int64_t)q * c) : 0;
                            fence_acq_rel_gpu();
                            int cnt = 0;
    #pragma unroll
                            for (int q = 0; q < FU_FLAG_WINDOW; ++q)
                                if (cnt == q && v[q] >= T) ++cnt;
                            if (cnt == 0) {
                                if (!wait_count_bounded(ready + kb, T, st, abort, wait_ns)) {
                                    ok = false;
                                    break;
                                }
                                cnt = 1;
                            }
                            known = j + cnt;
                        }
                        fence_proxy_async_global();
                        if (!DFS_IN_BOUNDS(st, kb < nkb && i0 + 1 < T && (diag || j0 + 1 < T))) {
                            *abort = 1;
                            ok = false;
                            break;
                        }
                        unsigned char* a = stage_mem + stage * TC_STAGE_BYTES;
                        unsigned char* b = a + 2 * TC_TILE_BYTES;
                        tc::mbar_arrive_expect_tx(&sm->full[stage], bytes);
                        tc::bulk_load(a, Sp + ((kb * T + i0) << 14), TC_TILE_BYTES, &sm->full[stage]);
                        tc::bulk_load(a + TC_TILE_BYTES, Sp + ((kb * T + i0 + 1) << 14), TC_TILE_BYTES, &sm->full[stage]);
                        if (!diag) {
                            tc::bulk_load(b, Sp + ((kb * T + j0) << 14), TC_TILE_BYTES, &sm->full[stage]);
                            tc::bulk_load(b + TC_TILE_BYTES, Sp + ((kb * T + j0 + 1) << 14), TC_TILE_BYTES,
                                          &sm->full[stage]);
                        }
                        issued[stage] = true;
                        last_parity[stage] = phase;
                        if (++stage == TC_STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
                *gram_tau = INT_MAX;  // no more steps: the converters run free
                if (!ok) {
                    *abort = 1;
                    set_status(st, DFS_ERR_TIMEOUT);
                }
                for (int s = 0; s < TC_STAGES; ++s)
                    if (issued[s] && !tc::mbar_wait_bounded(&sm->full[s], last_parity[s], never, kDefaultWaitNs))
                        set_status(st, DFS_ERR_TIMEOUT);
            }
        } else if (warp == kMmaWarp) {
            if (lane == 0 && has_gram) {
                // ---------------- MMA issuer ----------------
                constexpr uint32_t idesc_wide = tc::instr_desc_f32acc(tc::kFmtBF16, TC_BM, TC_BN);
                int stage = 0;
                uint32_t phase = 0;
                uint32_t acc_phase = 0;
                bool ok = true;
                const int gi = blockIdx.x;
                int I2, J2;
                tc_unit_ij(gi % U, I2, J2);
                const int sg = gi / U;
                const bool diag = J2 == I2;
                for (int t = 0; ok && t < G; ++t) {
                    const int slot = sg + t * w;
                    const int nk = slot < nkb ? (nkb - 1 - slot) / c + 1 : 0;
                    if (nk == 0) continue;  // the epilogue writes zeros for an empty task
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
                        const uint32_t bb = diag ? a0 : a0 + 2 * TC_TILE_BYTES;
    #pragma unroll
                        for (int kk = 0; kk < TC_ROW_BYTES / 32; ++kk)
                            tc::mma_ss<0>(tmem, tc::sw128_kmajor_desc(a0 + kk * 32), tc::sw128_kmajor_desc(bb + kk * 32),
                                          idesc_wide, (kt | kk) != 0);
    #pragma unroll
                        for (int kk = 0; kk < TC_ROW_BYTES / 32; ++kk)
                            tc::mma_ss<0>(tmem + (uint32_t)TC_BN, tc::sw128_kmajor_desc(a1a + kk * 32),
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
                tc::mma_commit(&sm->done);
                if (!tc::mbar_wait_bounded(&sm->done, 0, never, kDefaultWaitNs)) set_status(st, DFS_ERR_TIMEOUT);
            }
        } else if (warp == FU_SIG_WARP) {
            // ---------------- signaler ----------------
            // For every item of this CTA, in order: wait until the converters have written it (slot
            // li % FU_SLOTS) and free the slot for item li + FU_SLOTS; after each group of FU_PUB
            // items, one fence and the group's ready counts.  The barrier sequence is the
            // converters' exactly (every item, whatever its validity), so neither side can wait for
            // an arrival that never comes.
            if (conv) {
                FuCursor cur;
                cur.init(q0, w, NK);
                for (int sl = 0; sl < FU_SLOTS && sl < my_items; ++sl)
                    named_bar_arrive(FU_BAR_EMPTY + sl, FU_HANDSHAKE);
                for (int g0 = 0; g0 < my_items; g0 += FU_PUB) {
                    int kbs[FU_PUB];
#pragma unroll
                    for (int d = 0; d < FU_PUB; ++d) {
                        const int li = g0 + d;
                        kbs[d] = -1;
                        if (li < my_items) {
                            const int kb = cur.kb(w, c);
                            cur.advance(Q, w, NK);
                            named_bar_sync(FU_BAR_FULL + li % FU_SLOTS, FU_HANDSHAKE);
                            if (li + FU_SLOTS < my_items) named_bar_arrive(FU_BAR_EMPTY + li % FU_SLOTS, FU_HANDSHAKE);
                            // (test hook: CTA 0 withholds its first tile, so the Gram's waits for it run out)
                            const bool withhold = fault == DFS_TEST_FAULT_FUSED_GRAM && blockIdx.x == 0 && li == 0;
                            if (kb < nkb && !withhold) kbs[d] = kb;
                        }
                    }
                    if (lane == 0) {
                        // the converters' stores are ordered before the barriers; this thread's
                        // gpu-scope fence makes them visible before the counts it adds
                        fence_proxy_async_global();
                        fence_acq_rel_gpu();
#pragma unroll
                        for (int d = 0; d < FU_PUB; ++d)
                            if (kbs[d] >= 0) red_relaxed_gpu_add(ready + kbs[d], 1);
                    }
                }
            }
        }
    } else if (warp < FU_FIRST_CONV_WARP) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(FU_REGS_EPI));
        // ---------------- epilogue ----------------
        if (has_gram) {
            const int q = warp & 3;
            const int row = q * 32 + lane;
            uint32_t acc_phase = 0;
            const int gi = blockIdx.x;
            int I2, J2;
            tc_unit_ij(gi % U, I2, J2);
            const int sg = gi / U;
            const bool diag = J2 == I2;
            float* blk = part + (size_t)gi * TC_PART;
            for (int t = 0; t < G; ++t) {
                const int slot = sg + t * w;
                const int nk = slot < nkb ? (nkb - 1 - slot) / c + 1 : 0;
                const bool first = (t == 0);
                if (nk == 0) {
                    if (first)
                        for (int h = 0; h < 2; ++h)
                            for (int jj = 0; jj < TC_BN; jj += 4)
                                *reinterpret_cast<float4*>(blk + (size_t)(h * TC_BM + row) * TC_BN + jj) =
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
                    const int ncols = (h == 0 && diag) ? TC_BM : TC_BN;
                    const uint32_t tbase = tmem + (uint32_t)(h * TC_BN) + ((uint32_t)(q * 32) << 16);
                    float* dst = blk + (size_t)(h * TC_BM + row) * TC_BN;
#pragma unroll 1
                    for (int cc = 0; cc < ncols / 32; ++cc) {
                        uint32_t v[32];
                        tc::tmem_ld_32x32b_x32(tbase + (uint32_t)(cc * 32), v);
                        tc::tmem_ld_wait();
                        float4* d4 = reinterpret_cast<float4*>(dst + cc * 32);
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            float4 o = make_float4(__uint_as_float(v[4 * jj]), __uint_as_float(v[4 * jj + 1]),
                                                   __uint_as_float(v[4 * jj + 2]), __uint_as_float(v[4 * jj + 3]));
                            if (!first) {
                                const float4 p = d4[jj];
                                o.x += p.x;
                                o.y += p.y;
                                o.z += p.z;
                                o.w += p.w;
                            }
                            d4[jj] = o;
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&sm->acce);
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(FU_REGS_CONV));
        if (conv) {
            // ---------------- converters ----------------
            // This CTA converts row tile I (rows I * 128 ...) of the k-blocks q0, q0 + Q, q0 + 2Q, ... of
            // the consumption order.  Thread (converter warp cw, lane) owns rows
            // r_e = cw * 4 + lane / 8 + FU_ROW_STEP e (e < FU_RPT) of the tile and the FP32 segments
            // s = lane % 8 and s + 8 (16 bytes each) of every item's 64 columns: each load instruction
            // of a warp covers four whole 128-byte row halves.  The rows never change, so their dot
            // products with V accumulate in FP32 registers across items, folded into FP64 every
            // kFoldItems items.
            const int ct = threadIdx.x - FU_FIRST_CONV_WARP * 32;
            const int cw = ct >> 5;
            const int rg = lane >> 3, cs = lane & 7;
            const float* rowp[FU_RPT];
            bool row_ok[FU_RPT];
            int soff[FU_RPT][2];  // byte offsets of the thread's 8-byte BF16 pieces within a tile
#pragma unroll
            for (int e = 0; e < FU_RPT; ++e) {
                const int r = cw * 4 + rg + FU_ROW_STEP * e;
                const int i = I * TC_BM + r;
                row_ok[e] = i < n;
                rowp[e] = S + (int64_t)(row_ok[e] ? i : 0) * lds;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int sgm = cs + 8 * h;  // FP32 segment = 8 bytes of BF16 in the 128-byte row
                    soff[e][h] = r * 128 + ((((sgm >> 1) ^ (r & 7))) << 4) + ((sgm & 1) << 3);
                }
            }
            const int nkb_full = (int)(m / FU_ITEM_COLS);  // k-blocks with all 64 columns inside m

            bool ok = true;
            constexpr int FU_DEPTH = fu_depth(KQ);
            uint4 buf[FU_DEPTH][2 * FU_RPT];
            int desc[FU_DEPTH];  // k-block of the buffered item, -1 if it is not a real one
            constexpr int VQ = kVAtIssue(KQ) ? KQ : 1;
            float4 vbuf[FU_DEPTH][2][VQ];
            float acc[FU_RPT][KQ];
#pragma unroll
            for (int e = 0; e < FU_RPT; ++e)
#pragma unroll
                for (int q = 0; q < KQ; ++q) acc[e][q] = 0.f;
            double* rsum = sm->rsum;  // row r, right-hand side q at r * KQ + q; lane cs == 0 of the row adds
            for (int e = ct; e < TC_BM * KQ; e += FU_CONV_THREADS) rsum[e] = 0.0;
            named_bar_sync(FU_BAR_START, FU_CONV_THREADS);
            FuCursor cur, pcur;
            cur.init(q0, w, NK);
            pcur.init(q0, w, NK);
            // Pull the next item's 128 rows x 256 bytes into L2: thread ct takes row ct / 2, half ct % 2.
            auto prefetch = [&]() {
                const int kb = pcur.kb(w, c);
                pcur.advance(Q, w, NK);
                const int i = I * TC_BM + (ct >> 1);
                const int64_t j0 = (int64_t)kb * FU_ITEM_COLS + (ct & 1) * 32;
                if (kb < nkb && i < n && j0 < m) prefetch_l2(S + (int64_t)i * lds + j0);
            };
            // Issue the loads of the next item into b and vb (zeros past n and m, and for items that
            // are not real), after holding back while more than `lead` steps ahead of this CTA's
            // producer (lane 0 waits, the warp takes its verdict: `ok` stays warp-uniform).
            auto issue = [&](uint4 (&b)[2 * FU_RPT], int& dkb, float4 (&vb)[2][VQ]) {
                const int kb = cur.kb(w, c);
                const int tau = cur.tau;
                cur.advance(Q, w, NK);
                const bool valid = kb < nkb && tau < G * NK;
                if (valid && ok && *gram_tau < tau - lead) {
                    int good = 1;
                    if (lane == 0) {
                        const uint64_t t0 = tc::globaltimer_ns();
                        while (*gram_tau < tau - lead) {
                            __nanosleep(64);
                            if (*abort || *reinterpret_cast<const volatile int*>(&st->status) ||
                                tc::globaltimer_ns() - t0 > wait_ns) {
                                good = 0;
                                break;
                            }
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, good, 0) != 0;
                }
                dkb = (valid && ok) ? kb : -1;
                const int64_t col = (int64_t)kb * FU_ITEM_COLS;
                if (valid && ok && kb < nkb_full) {
                    // the usual case: every column inside m
#pragma unroll
                    for (int e = 0; e < FU_RPT; ++e)
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            b[2 * e + h] = row_ok[e] ? __ldcs(reinterpret_cast<const uint4*>(rowp[e] + col + (cs + 8 * h) * 4))
                                                     : make_uint4(0u, 0u, 0u, 0u);
                } else {
#pragma unroll
                    for (int e = 0; e < FU_RPT; ++e)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int64_t j0 = col + (cs + 8 * h) * 4;
                            uint4 x = make_uint4(0u, 0u, 0u, 0u);
                            if (valid && ok && row_ok[e]) {
                                const float* p = rowp[e];
                                if (j0 < m) x.x = __float_as_uint(p[j0]);
                                if (j0 + 1 < m) x.y = __float_as_uint(p[j0 + 1]);
                                if (j0 + 2 < m) x.z = __float_as_uint(p[j0 + 2]);
                                if (j0 + 3 < m) x.w = __float_as_uint(p[j0 + 3]);
                            }
                            b[2 * e + h] = x;
                        }
                }
                if constexpr (kVAtIssue(KQ)) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int64_t j0 = col + (cs + 8 * h) * 4;
#pragma unroll
                        for (int q = 0; q < VQ; ++q) {
                            const float* vr = V + (int64_t)q * ldv;
                            float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (valid && ok && q < k) {
                                if (v_vec && j0 + 4 <= m) {
                                    t4 = __ldg(reinterpret_cast<const float4*>(vr + j0));
                                } else {
                                    if (j0 < m) t4.x = __ldg(vr + j0);
                                    if (j0 + 1 < m) t4.y = __ldg(vr + j0 + 1);
                                    if (j0 + 2 < m) t4.z = __ldg(vr + j0 + 2);
                                    if (j0 + 3 < m) t4.w = __ldg(vr + j0 + 3);
                                }
                            }
                            vb[h][q] = t4;
                        }
                    }
                }
            };
            // Convert and store one item, and add its products to the row sums.
            auto process = [&](const uint4 (&b)[2 * FU_RPT], int dkb, const float4 (&vbi)[2][VQ]) {
                if (dkb < 0) return;
                float4 vb[2][KQ];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        if constexpr (kVAtIssue(KQ)) {
                            vb[h][q] = vbi[h][q < VQ ? q : 0];
                        } else {
                            const int64_t j0 = (int64_t)dkb * FU_ITEM_COLS + (cs + 8 * h) * 4;
                            const float* vr = V + (int64_t)q * ldv;
                            float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (q < k) {
                                if (v_vec && j0 + 4 <= m) {
                                    t4 = __ldg(reinterpret_cast<const float4*>(vr + j0));
                                } else {
                                    if (j0 < m) t4.x = __ldg(vr + j0);
                                    if (j0 + 1 < m) t4.y = __ldg(vr + j0 + 1);
                                    if (j0 + 2 < m) t4.z = __ldg(vr + j0 + 2);
                                    if (j0 + 3 < m) t4.w = __ldg(vr + j0 + 3);
                                }
                            }
                            vb[h][q] = t4;
                        }
                    }
                unsigned char* tile = Sp + (((int64_t)dkb * T + I) << 14);
                const bool tile_ok = DFS_IN_BOUNDS(st, dkb < nkb && I < T);
#pragma unroll
                for (int e = 0; e < FU_RPT; ++e) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint4 x = b[2 * e + h];
                        const float x0 = __uint_as_float(x.x), x1 = __uint_as_float(x.y), x2 = __uint_as_float(x.z),
                                    x3 = __uint_as_float(x.w);
#pragma unroll
                        for (int q = 0; q < KQ; ++q)
                            acc[e][q] = fmaf(x3, vb[h][q].w, fmaf(x2, vb[h][q].z, fmaf(x1, vb[h][q].y, fmaf(x0, vb[h][q].x, acc[e][q]))));
                        const __nv_bfloat162 lo = __floats2bfloat162_rn(x0, x1);
                        const __nv_bfloat162 hi = __floats2bfloat162_rn(x2, x3);
                        uint2 o;
                        o.x = *reinterpret_cast<const uint32_t*>(&lo);
                        o.y = *reinterpret_cast<const uint32_t*>(&hi);
                        if (tile_ok) *reinterpret_cast<uint2*>(tile + soff[e][h]) = o;
                    }
                }
            };
            // FP32 row sums -> FP64: reduce over the 8 lanes of a row, lane cs == 0 keeps the total
            auto fold = [&]() {
#pragma unroll
                for (int e = 0; e < FU_RPT; ++e)
#pragma unroll
                    for (int q = 0; q < KQ; ++q) {
                        float a = acc[e][q];
                        a += __shfl_xor_sync(0xffffffffu, a, 1);
                        a += __shfl_xor_sync(0xffffffffu, a, 2);
                        a += __shfl_xor_sync(0xffffffffu, a, 4);
                        if (cs == 0) rsum[(cw * 4 + rg + FU_ROW_STEP * e) * KQ + q] += (double)a;
                        acc[e][q] = 0.f;
                    }
            };

            for (int p = 0; p < FU_PREFETCH; ++p) prefetch();
#pragma unroll
            for (int d = 0; d < FU_DEPTH - 1; ++d) issue(buf[d], desc[d], vbuf[d]);
            int since_fold = 0;
            for (int base = 0; base < my_items; base += FU_DEPTH) {
#pragma unroll
                for (int d = 0; d < FU_DEPTH; ++d) {
                    const int li = base + d;
                    prefetch();
                    issue(buf[(d + FU_DEPTH - 1) % FU_DEPTH], desc[(d + FU_DEPTH - 1) % FU_DEPTH],
                          vbuf[(d + FU_DEPTH - 1) % FU_DEPTH]);
                    if (li < my_items) {
                        process(buf[d], desc[d], vbuf[d]);
                        // hand the item to the signaler: wait until its slot is free, then arrive
                        named_bar_sync(FU_BAR_EMPTY + li % FU_SLOTS, FU_HANDSHAKE);
                        named_bar_arrive(FU_BAR_FULL + li % FU_SLOTS, FU_HANDSHAKE);
                        if (++since_fold == kFoldItems) {
                            since_fold = 0;
                            fold();
                        }
                    }
                }
            }
            fold();
            // this CTA's share of b: rows of tile I, partial q0 of Q (written whole, every launch; a
            // row's sums are only touched by its own lane cs == 0)
            if (cs == 0) {
#pragma unroll
                for (int e = 0; e < FU_RPT; ++e) {
                    const int r = cw * 4 + rg + FU_ROW_STEP * e;
                    const int i = I * TC_BM + r;
                    if (i < n && DFS_IN_BOUNDS(st, q0 < Q))
#pragma unroll
                        for (int q = 0; q < KQ; ++q) Rpart[((size_t)q0 * n + i) * KQ + q] = rsum[r * KQ + q];
                }
            }
            if (!ok) {
                *abort = 1;
                set_status(st, DFS_ERR_TIMEOUT);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// ---- host side ------------------------------------------------------------------------------

// The fused form applies to FP32 S with BF16 tiles, at most 4 right-hand sides, and a Gram
// schedule that fits one wave of the grid (U units x w slot groups <= SMs, i.e. n <= 4096 on 152
// SMs).  Fills plan (a GramTcPlan that gram_tc_finalize reads as usual) and returns 1, else 0.
// The kernel's register split assumes it was built at FU_LAUNCH_REGS registers a thread: a
// smaller launch count would leave the converters' setmaxnreg.inc waiting for registers that do
// not exist, so the fused form is only offered when the built kernel reports exactly that count.
static const void* fused_kernel_for(int kq) {
    return kq == 1 ? (const void*)gram_fused_kernel<1>
                   : (kq == 2 ? (const void*)gram_fused_kernel<2> : (const void*)gram_fused_kernel<4>);
}
static bool fused_kernel_regs_ok(int kq) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, fused_kernel_for(kq)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.numRegs == FU_LAUNCH_REGS && a.maxThreadsPerBlock >= FU_THREADS;
}

int gram_fused_plan(int s_dtype, int64_t n, int64_t m, int kq, int num_sms, size_t smem_optin, GramTcPlan* plan) {
    if (s_dtype != DFS_F32 || kq > 4 || n < 1 || m < 1) return 0;
    if (smem_optin < FU_SMEM_BYTES) return 0;
    if (!fused_kernel_regs_ok(kq == 1 ? 1 : (kq == 2 ? 2 : 4))) return 0;
    GramTcPlan p{};
    p.kind = 0;
    p.packed = 1;
    p.n_tiles = (int)round_up(ceil_div(n, TC_BM), 2);
    p.h2 = 0;
    const int U = tc_num_units(p.n_tiles, 0);
    if (U > num_sms) return 0;
    p.npairs = U;
    const int64_t nkb = ceil_div(m, FU_ITEM_COLS);
    // the kernel walks the k-blocks with 32-bit indices (w G NK <= nkb + 2 c)
    if (nkb + 4 * (int64_t)num_sms >= (int64_t)1 << 30) return 0;
    int w = num_sms / U;
    if (w > nkb) w = (int)nkb;
    if (w < 1) w = 1;
    int G = 1;
    while ((int64_t)w * G * 1024 < nkb) ++G;
    p.c = w * G;
    p.group = G;
    p.ntasks = U * p.c;
    p.nkb = nkb;
    p.partial_bytes = (size_t)(U * w) * TC_PART * sizeof(float);
    *plan = p;
    return 1;
}

size_t gram_fused_ready_bytes(const GramTcPlan& plan) { return (size_t)plan.nkb * sizeof(int); }

cudaError_t launch_gram_fused(const GramTcPlan& plan, int kq, const void* S, int64_t n, int64_t m, int64_t lds,
                              const void* V, int64_t ldv, int k, double* Rpart, void* Sp, void* P, int* ready,
                              DevStatus* st, int num_sms, cudaStream_t stream, int* parts) {
    if (kq != 1 && kq != 2 && kq != 4) return cudaErrorInvalidValue;
    if (k > kq || (k > 0 && V == nullptr) || Sp == nullptr || P == nullptr || ready == nullptr)
        return cudaErrorInvalidValue;
    const int U = plan.npairs, G = plan.group, w = plan.c / plan.group;
    if (U * w > num_sms) return cudaErrorInvalidValue;
    const int NK = (int)ceil_div(plan.nkb, plan.c);
    cudaError_t e = cudaMemsetAsync(ready, 0, gram_fused_ready_bytes(plan), stream);
    if (e != cudaSuccess) return e;
    const int v_vec = (V != nullptr && (reinterpret_cast<uintptr_t>(V) % 16 == 0) && (ldv % 4 == 0)) ? 1 : 0;
    const float* s = static_cast<const float*>(S);
    const float* v = static_cast<const float*>(V);
    unsigned char* sp = static_cast<unsigned char*>(Sp);
    float* part = static_cast<float*>(P);
    int T = plan.n_tiles;
    int ni = (int)n;
    int nkb = (int)plan.nkb;
    // A converter holds the loads of fu_depth - 1 items it has not yet written while it waits to
    // issue the next, and up to FU_PUB - 1 written items may still wait for the rest of their
    // publication group; its consecutive items are Q / w steps apart, so those items lie at most
    // `span` steps behind it.  With lead >= span an item the producer waits for is never one held
    // back that way (the progress argument above).
    const int Q = num_sms / T;
    const int span = (int)ceil_div((int64_t)(fu_depth(kq) - 1 + FU_PUB - 1) * Q, w) + 1;
    int lead = kLead + span;
    void* args[] = {(void*)&s,  (void*)&ni, (void*)&m,   (void*)&lds, (void*)&v,    (void*)&ldv,
                    (void*)&k,  (void*)&v_vec, (void*)&Rpart, (void*)&sp, (void*)&T,  (void*)&U,
                    (void*)&w,  (void*)&G,  (void*)&NK,  (void*)&nkb, (void*)&lead, (void*)&part,
                    (void*)&ready, (void*)&st};
    const void* kern = fused_kernel_for(kq);
    if (!fused_kernel_regs_ok(kq)) return cudaErrorNotSupported;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FU_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FU_THREADS, FU_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    e = cudaLaunchCooperativeKernel(kern, dim3(num_sms), dim3(FU_THREADS), args, FU_SMEM_BYTES, stream);
    count_launch();
    if (parts) *parts = Q;
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace dfs
