/*
 * dfs.h -- C ABI of libdfs: Cholesky solve of the damped Fisher system on GB300 (sm_103a).
 *
 * Method: Chen, Xie, Wang, "Efficient Numerical Algorithm for Large-Scale Damped
 * Natural Gradient Descent", arXiv 2310.17556.
 *   Eq. 1        (S^T S + lambda I) x = v, S is n x m (m >> n), lambda > 0.
 *   Algorithm 1  W = S S^T + lambda I~;  L = Chol(W);  Q = L^{-1} S;  x = (v - Q^T Q v) / lambda.
 *   Section 2    Q is never formed: Q^T Q v = S^T L^{-T} L^{-1} S v, evaluated right to left
 *                with two triangular solves.
 *   Appendix A   for lambda > 0 the result is the unique solution of Eq. 1.
 *
 * Conventions shared by every entry point
 *   - Every function returns a dfs_status.  The library never aborts.  It prints only when
 *     the environment variable DFS_LOG is set (to anything but "0"): then each error message
 *     it records for dfs_last_error also goes to stderr.
 *   - Matrices are row-major with an explicit leading dimension (in elements).
 *     S: n rows of length m, row stride lds >= m (each sample row is contiguous).
 *     V, X: k rows of length m (one right-hand side per row), strides ldv, ldx >= m.
 *     W, L: n x n, row stride ldw >= n; only the lower triangle is read or written.
 *     Y, B (n-space vectors): n rows of k values, row stride ldb >= k.
 *   - Element types: S is FP64, FP32 or BF16 (dfs_dtype).  V and X are FP64 when S is
 *     FP64 and FP32 otherwise.  n-space results follow the precision of the call.
 *   - Pointers named "device" are CUDA device memory owned by the caller; the library
 *     keeps no pointer to them after the call returns.  "stream" is a cudaStream_t
 *     (NULL = legacy default stream); all GPU work of a call is ordered on it.
 *   - Argument errors return DFS_ERR_INVALID_ARG before any GPU work is queued:
 *     NULL pointers, n < 1, m < 1, k < 1, a leading dimension below its minimum,
 *     lambda not finite or <= 0, an S pointer not 16-byte aligned, or lds * sizeof(S
 *     element) not a multiple of 16 bytes (S rows are read with 16-byte vector loads
 *     and tensor-memory-accelerator copies).
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef DFS_H
#define DFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DFS_VERSION 100

typedef enum {
    DFS_OK = 0,
    DFS_ERR_INVALID_ARG = 1,   /* rejected before launch */
    DFS_ERR_NOT_SPD = 2,       /* a Cholesky pivot was <= 0 or NaN (the Cholesky of Algorithm 1) */
    DFS_ERR_NOT_CONVERGED = 3, /* refinement stopped above tolerance; X holds the last iterate */
    DFS_ERR_NONFINITE = 4,     /* NaN/Inf met in W or in the solution */
    DFS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    DFS_ERR_NO_MEMORY = 6,     /* workspace allocation failed */
    DFS_ERR_CUDA = 7,          /* a CUDA runtime call failed (text in dfs_last_error) */
    DFS_ERR_UNSUPPORTED = 8,   /* valid request this build cannot serve (e.g. no sm_103a device) */
    DFS_ERR_BOUNDS = 9         /* debug build only (libdfs_debug.so, -DDFS_DEBUG_BOUNDS): a device
                                  index check failed and its access was skipped; dfs_last_error
                                  names the site */
} dfs_status;

typedef enum {
    DFS_F64 = 0,   /* double */
    DFS_F32 = 1,   /* float */
    DFS_BF16 = 2   /* bfloat16 (S only) */
} dfs_dtype;

/* Arithmetic of the Gram step W = S S^T (the Gram of Algorithm 1), the O(n^2 m) contraction. */
typedef enum {
    DFS_PREC_AUTO = 0,   /* FP64 for FP64 S; BF16 tensor Gram + refinement otherwise */
    DFS_PREC_FP64 = 1,   /* FP64 everywhere (S must be FP64) */
    DFS_PREC_FP32 = 2,   /* plain FP32 path: FP32 FFMA Gram, FP32 solves, no refinement */
    DFS_PREC_BF16 = 3,   /* tcgen05 BF16 Gram (FP32 accumulate) + n-space refinement */
    DFS_PREC_TF32 = 4,   /* tcgen05 TF32 Gram (FP32 accumulate) + n-space refinement */
    DFS_PREC_BF16X3 = 5, /* FP32 S only: S = H + L, H = bf16(S), L = bf16(S - H); tcgen05 BF16 Gram
                            of W = H H^T + L H^T + (L H^T)^T (L L^T, ~2^-16 relative, dropped): the
                            work of three BF16 Grams, ~2^-16 relative accuracy; + refinement */
    DFS_PREC_FP8 = 6     /* FP32 or BF16 S: each row scaled by a power of two r_i (max |s_ij| / r_i
                            <= 448) and rounded to e4m3; tcgen05 kind::f8f6f4 Gram, W_ik scaled by
                            r_i r_k; one extra read of S for the row maxima; + refinement */
} dfs_precision;

/* entries of dfs_info.ms and of dfs_step_times' output */
#define DFS_STEP_TIMES 9

/* dfs_options.flags */
#define DFS_FLAG_STEP_TIMING 1  /* record CUDA events around the steps; dfs_info.ms is filled */
#define DFS_FLAG_FP64_PANEL 2   /* factor the 32 x 32 diagonal blocks of the Cholesky in FP64
                                   (FP32 and mixed paths; the FP64 path always does).  Off by
                                   default: GB300's FP64 rate (about 1/64 of FP32) makes the
                                   factorisation ~4.6x slower at n = 1024 (1.42 ms against
                                   0.31 ms), each block is stored back in FP32, and the
                                   trailing updates are FP32 in any case */
#define DFS_FLAG_CENTER 4       /* stochastic reconfiguration (Section 4): the S argument holds O, the
                                   log-derivatives of the wave function, and the system solved is
                                   Eq. 1 with S = (O - O_bar) / sqrt(n), O_bar the mean of O over the
                                   n rows.  O is never modified or copied: W = P (O O^T / n) P +
                                   lambda I with P = I - 1 1^T / n, b = P O v / sqrt(n), and each
                                   pass over O reads P y / sqrt(n) (the triangular solves run on the
                                   reduce + substitution kernels).  dfs_solve and dfs_solve_host. */
/* Right-hand sides per group: the solve runs its passes over S on groups of at most g columns of
 * V (g = 1, 2, 4 or 8).  More per group means fewer passes over S, but each pass does more work
 * per strip; DFS_FLAG_RHS_GROUP(0) (the default) lets the library choose (the kernels' limit,
 * or a dfs_autotune choice for the problem's class). */
#define DFS_FLAG_RHS_GROUP(g) (((g) & 15) << 8)
#define DFS_FLAG_TWO_KERNEL_GRAM 8 /* BF16 Gram on FP32 S: run the first pass over S (b = S v and the
                                   BF16 tiles) and the Gram as two kernels instead of the one fused
                                   kernel that overlaps them (the default where it applies: n <= 4096
                                   on 152 SMs, up to 4 right-hand sides per group) */

typedef struct {
    int precision;   /* dfs_precision */
    int max_iter;    /* refinement passes after the first solve (mixed paths); <0 = default 8 */
    double tol;      /* stop when the estimated relative error left in x <= tol; <=0 = 1e-7 */
    int flags;       /* DFS_FLAG_* bits, 0 for none */
} dfs_options;

typedef struct {
    int status;             /* final dfs_status of the device work */
    int precision_used;     /* dfs_precision actually run */
    int iters;              /* refinement passes run (0 on the FP32/FP64 paths) */
    int failed_pivot;       /* first non-positive pivot index, -1 if none */
    int passes;             /* full refinement passes over S (iters, less a final correction read
                               from the packed BF16 tiles) */
    double rel_correction;  /* estimated relative error left in x (0 if no refinement) */
    double rel_residual_n;  /* last ||r_n|| / ||S v||, r_n = S v - (S S^T + lambda I) y */
    float ms[DFS_STEP_TIMES]; /* with DFS_FLAG_STEP_TIMING (CUDA events on the call's stream):
                               [0] Gram kernel (the fused first-pass kernel when it runs),
                               [1] Gram finalize + Cholesky, [2] first n-space solve (S v pass,
                               two triangular solves), [3] the rest (refinement or the x pass),
                               [4] whole call, [5] S v pass kernel alone (0 in the fused form), [6] first
                               pass over S after the solves (refinement or x pass) alone,
                               [7] Cholesky kernel alone, [8] the correction from the packed BF16
                               tiles alone (0 when it did not run); zeros otherwise */
} dfs_info;

typedef struct dfs_handle_s* dfs_handle;

/* Create a handle bound to CUDA device `device`.  The handle owns a device workspace that
 * grows on demand (cudaMalloc) and is freed by dfs_destroy.  Errors: INVALID_ARG (NULL
 * out-pointer), CUDA (bad device), UNSUPPORTED (device is not compute capability 10.3). */
dfs_status dfs_create(dfs_handle* handle, int device);
dfs_status dfs_destroy(dfs_handle handle);

/* Number of CUDA kernels this library has launched in the calling process (all handles). */
int64_t dfs_kernel_launches(void);

/* Static text for a status code; never NULL. */
const char* dfs_status_string(int status);
/* Last error message recorded on this handle (empty string if none); owned by the handle. */
const char* dfs_last_error(dfs_handle handle);

/* Grow the workspace now so later calls up to these sizes allocate nothing (needed before
 * stream capture of dfs_solve).  Sizes are maxima over the calls that will follow. */
dfs_status dfs_reserve(dfs_handle handle, int64_t n_max, int64_t m_max, int64_t k_max,
                       int precision);

/* Full solve of Eq. 1 for k right-hand sides (Algorithm 1 with Q inlined, Section 2).
 *   S (device, n x m, lds), V (device, k x m, ldv) -> X (device, k x m, ldx).
 *   X must not overlap S; X may equal V (in place).
 *   opt may be NULL (defaults: precision AUTO, max_iter 8, tol 1e-7).
 * Asynchronous on `stream` when info == NULL: the return value then only covers argument
 * checks and launches; device-detected errors are read with dfs_sync_info.  When info !=
 * NULL the call synchronizes `stream`, fills *info and returns the device status. */
dfs_status dfs_solve(dfs_handle handle, const void* S, int s_dtype, int64_t n, int64_t m,
                     int64_t lds, const void* V, int64_t k, int64_t ldv, double lambda,
                     void* X, int64_t ldx, const dfs_options* opt, void* stream,
                     dfs_info* info);

/* Same solve with S, V and X in HOST memory (pinned memory gives full copy speed).  The
 * call copies S and V to handle-owned device buffers, solves, copies X back and
 * synchronizes `stream` before returning.  info may be NULL. */
dfs_status dfs_solve_host(dfs_handle handle, const void* S, int s_dtype, int64_t n, int64_t m,
                          int64_t lds, const void* V, int64_t k, int64_t ldv, double lambda,
                          void* X, int64_t ldx, const dfs_options* opt, void* stream,
                          dfs_info* info);

/* dfs_solve_host without the wait: the copies and the solve are queued and the call returns.
 * S and V must be PINNED host memory (pageable memory makes the copies synchronous) and must stay
 * unchanged, and X must not be read, until `stream` has finished the call's work (dfs_sync_info
 * or a stream synchronize).  The uploads run on a copy stream of the handle into one of two
 * device staging slots that alternate between calls, so consecutive calls overlap one call's
 * host -> device copy with the previous call's solve (the link is the bound of a host-to-host
 * solve); the solve and the download of X run on `stream` in call order.  A failed pivot or
 * other device error is reported by the next dfs_sync_info, which describes the last call's
 * solve only. */
dfs_status dfs_solve_host_async(dfs_handle handle, const void* S, int s_dtype, int64_t n, int64_t m,
                                int64_t lds, const void* V, int64_t k, int64_t ldv, double lambda,
                                void* X, int64_t ldx, const dfs_options* opt, void* stream);

/* Complex stochastic reconfiguration (Section 4, full Fisher matrix F = S^dagger S): solve
 * (S^dagger S + lambda I) X = V for complex S = S_re + i S_im and k complex right-hand sides.
 * S_re, S_im: DEVICE planes, n x m row-major with the same lds and dtype (FP32, BF16 or FP64, the
 * dfs_solve contract); V_re, V_im, X_re, X_im: DEVICE planes of k rows of length m (ldv, ldx),
 * FP64 for FP64 S, else FP32.  Algorithm 1 with Hermitian conjugates, on the stacked real matrix
 * Z = [S_re; S_im] (2n x m): the Gram is Z Z^T (Re W and Im W are sums and differences of its
 * blocks), every pass over S reads Z once with two real right-hand sides per complex one, and the
 * n-space steps factor and solve the real 2n system [[Re W, -Im W], [Im W, Re W]].  When S_im is
 * row n of the same allocation as S_re (S_im == S_re + n lds elements) Z is used in place;
 * otherwise the call stacks the planes in a handle-owned buffer (the bytes of the two planes).
 * Every precision of dfs_solve applies; up to 4 complex right-hand sides share a pass (larger k
 * runs in groups).  2n <= 65536.  Synchronizes `stream` before returning; info may be NULL.
 * DFS_FLAG_CENTER is not available here (DFS_ERR_UNSUPPORTED).  The real-part Fisher matrix
 * F = Re[S^dagger S] needs no entry point: it is dfs_solve on the 2n x m matrix with the rows of
 * S_re followed by those of S_im. */
dfs_status dfs_solve_complex(dfs_handle handle, const void* S_re, const void* S_im, int s_dtype,
                             int64_t n, int64_t m, int64_t lds, const void* V_re, const void* V_im,
                             int64_t k, int64_t ldv, double lambda, void* X_re, void* X_im,
                             int64_t ldx, const dfs_options* opt, void* stream, dfs_info* info);

/* Synchronize `stream` and report the device status of the last dfs_solve on this handle. */
dfs_status dfs_sync_info(dfs_handle handle, void* stream, dfs_info* info);

/* Mean step times in ms (layout of dfs_info.ms) over the solves run with DFS_FLAG_STEP_TIMING
 * since the previous call, at most the last 64; waits for the last of their events.
 * *count (may be NULL) receives how many solves were averaged (0: mean_ms all zero). */
dfs_status dfs_step_times(dfs_handle handle, float* mean_ms, int* count);

/* One independent problem of a batch (all pointers device memory, same dtype rules). */
typedef struct {
    const void* S; int64_t n, m, lds;
    const void* V; int64_t k, ldv;
    double lambda;
    void* X; int64_t ldx;
} dfs_problem;

/* Solve `count` independent problems of uneven (n, m) (Eq. 1 for each; Algorithm 1 per
 * problem).  `problems` is a host array; every problem obeys dfs_solve's rules, S of type s_dtype.
 * Problems are dealt longest first (estimated cost n^2 m + 4 n m k) to up to 8 lanes (see
 * dfs_set_batch_lanes), each with its own stream and workspace, forked from and joined back into `stream`; with one problem the
 * solve runs on `stream` itself.
 * status_out (host, `count` ints, may be NULL) receives each problem's device status, in
 * `problems` order; when it is non-NULL the call synchronizes `stream` and returns the first
 * problem's error.  With status_out NULL nothing synchronizes; the statuses stay on the device
 * for dfs_batched_status.
 * Allocation: lanes, their workspaces and the status array are created or grown on demand,
 * unless dfs_plan_batched was called before for problems of the same or larger sizes.  During
 * stream capture any such growth fails with DFS_ERR_NO_MEMORY: plan first, then capture. */
dfs_status dfs_solve_batched(dfs_handle handle, const dfs_problem* problems, int count,
                             int s_dtype, const dfs_options* opt, void* stream,
                             int* status_out);

/* Prepare dfs_solve_batched for this list without launching anything: validate it (the same
 * argument errors as dfs_solve_batched), create the lanes it will use with their streams and
 * events, size each lane's workspace for the problems the longest-first schedule deals it, and
 * size the device status array.  After it, dfs_solve_batched on a list with the same count, the
 * same (or smaller) n, m, k per position and the same s_dtype and precision allocates nothing
 * and can be captured into a CUDA graph.  *workspace_bytes (may be NULL) receives the device
 * bytes held for the batch: the lanes' workspaces plus the status array.  Only the problems'
 * sizes, lambda and pointers' alignment are read; S, V and X are not touched. */
dfs_status dfs_plan_batched(dfs_handle handle, const dfs_problem* problems, int count,
                            int s_dtype, const dfs_options* opt, size_t* workspace_bytes);

/* Device statuses of the last dfs_solve_batched on this handle, in `problems` order:
 * synchronizes `stream` (the stream the batch ran on, or a later one) and copies `count`
 * ints (count <= the batch's count) to host memory status_out.  Returns DFS_OK, or the first
 * non-zero status among them. */
dfs_status dfs_batched_status(dfs_handle handle, int* status_out, int count, void* stream);

/* Concurrency of dfs_solve_batched on this handle: up to `lanes` (1..16) lanes run at once, and
 * each lane's kernels size their grids for 1/share (share 1..16) of the SMs, so that several
 * small problems' latency-bound kernels share the GPU instead of queueing behind each other.
 * The default is 8 lanes, share 1.  Takes effect at the next dfs_plan_batched or
 * dfs_solve_batched (plan again before capturing a batch into a graph).  DFS_ERR_INVALID_ARG
 * for values out of range. */
dfs_status dfs_set_batch_lanes(dfs_handle handle, int lanes, int share);
dfs_status dfs_get_batch_lanes(dfs_handle handle, int* lanes, int* share);

/* Choose the batch concurrency (lanes, share) for this list of problems by timing it: each of a
 * fixed set of candidates runs the batch once untimed and twice timed on `stream` (the problems'
 * X are overwritten; S and V are only read), and the fastest is set on the handle as by
 * dfs_set_batch_lanes.  cache_path (may be NULL) names a text file of JSON lines
 *   {"gpu": <device name>, "batch": <key>, "lanes": L, "share": S, "ms": t}
 * where the key encodes count, s_dtype, the resolved precision and a hash of the sorted (n, m, k)
 * of the problems: a line for this GPU and key is used without timing (*ms_out = 0), otherwise
 * the winner is appended.  lanes_out, share_out, ms_out (may be NULL) receive the choice and its
 * mean batch time in ms.  Synchronizes `stream`; not allowed during stream capture
 * (DFS_ERR_INVALID_ARG).  Errors of a timed run are returned as dfs_solve_batched's; a problem
 * that stops above its tolerance does not stop the tuning. */
dfs_status dfs_autotune_batched(dfs_handle handle, const dfs_problem* problems, int count,
                                int s_dtype, const dfs_options* opt, const char* cache_path,
                                void* stream, int* lanes_out, int* share_out, float* ms_out);

/* ---- single steps of Algorithm 1 (for composition and testing) ---------------------- */

/* Gram: W = S S^T + lambda I~, lower triangle only, written to W (device, n x n, ldw).
 * W is FP64 for precision FP64, FP32 otherwise.  precision FP32 = FFMA; BF16/TF32/BF16X3
 * run the tcgen05 tensor-core kernel (lambda is added in FP32 after the contraction). */
dfs_status dfs_gram(dfs_handle handle, const void* S, int s_dtype, int64_t n, int64_t m,
                    int64_t lds, double lambda, int precision, void* W, int64_t ldw,
                    void* stream);

/* Cholesky of Algorithm 1: in-place lower factor W = L L^T (device, n x n, ldw, w_dtype FP32 or
 * FP64).  Blocked right-looking, the kernel dfs_solve runs: FP64 W entirely in FP64, FP32 W with
 * its 32 x 32 diagonal blocks in FP32 (as dfs_solve without DFS_FLAG_FP64_PANEL).  Synchronizes
 * `stream`.  Returns NOT_SPD (and *failed_pivot, may be NULL) on a pivot <= 0 or NaN. */
dfs_status dfs_cholesky(dfs_handle handle, void* W, int w_dtype, int64_t n, int64_t ldw,
                        void* stream, int64_t* failed_pivot);

/* Triangular solves of Section 2 with the factor from dfs_cholesky (device L, n x n, ldl):
 * trans = 0 solves L A = B, trans = 1 solves L^T Y = B, in place on B (device, n x k, ldb),
 * same dtype as L. */
dfs_status dfs_trsm(dfs_handle handle, const void* L, int l_dtype, int64_t n, int64_t ldl,
                    void* B, int64_t k, int64_t ldb, int trans, void* stream);

/* The streaming pass over S (one read of S), with Y (device, n x k FP64, ldy):
 *   U = V - S^T Y           (Y == NULL means Y = 0)
 *   X = U / lambda          (if X != NULL; Algorithm 1's update of x with Q inlined)
 *   R = S U - lambda Y      (if R != NULL; device n x k FP64, ldr: the n-space residual
 *                            S v - (S S^T + lambda I~) y of Appendix A's identity)
 * V, X as in dfs_solve. */
dfs_status dfs_fisher_pass(dfs_handle handle, const void* S, int s_dtype, int64_t n, int64_t m,
                           int64_t lds, const void* V, int64_t k, int64_t ldv, const double* Y,
                           int64_t ldy, double lambda, void* X, int64_t ldx, double* R,
                           int64_t ldr, void* stream);

/* ---- throughput probes --------------------------------------------------------------- */

/* Measured peak rate (flop/s, 2 per fused multiply-add) of the current device's SIMT units, the
 * roofline denominator of the kernels that run on them (the FP32 path's Gram, the FP64 path):
 * independent FMA chains on every SM for ~0.1-0.3 s.  Changes no device setting.  Allocates a
 * small output buffer.  Synchronous. */
#define DFS_PEAK_FFMA32 1
#define DFS_PEAK_DFMA64 2
dfs_status dfs_measure_peak(int kind, double* flops_per_s);

/* ---- test hook: make one bounded device wait run out ---------------------------------- */

/* Every device-side wait of the library (on a flag, a peer CTA or an mbarrier) gives up after a
 * limit (2 s by default), records DFS_ERR_TIMEOUT in the call's device status, releases what it
 * holds and returns; the next call on the handle starts afresh.  This hook lets a test exercise
 * that path without faulting anything: it sets the limit for the following calls on `handle`
 * (wait_limit_ns <= 0: back to 2 s) and names one signal that a kernel then withholds (the
 * waits for it run out):
 *   DFS_TEST_FAULT_CHOLESKY      the Cholesky never publishes tile (2, 1) as finished (n > 64);
 *   DFS_TEST_FAULT_CLUSTER_PASS  in a refinement pass run as clusters (FP32 S, n <= 4096), rank 1
 *                                of the first cluster withholds its first strip's partial sums;
 *   DFS_TEST_FAULT_FUSED_GRAM    the fused first pass (BF16 Gram, FP32 S) withholds one tile.
 * DFS_TEST_FAULT_NONE (0) switches it off.  Not for production use. */
#define DFS_TEST_FAULT_NONE 0
#define DFS_TEST_FAULT_CHOLESKY 1
#define DFS_TEST_FAULT_CLUSTER_PASS 2
#define DFS_TEST_FAULT_FUSED_GRAM 3
dfs_status dfs_set_test_fault(dfs_handle handle, int fault, int64_t wait_limit_ns);

/* ---- no-allocation variant ---------------------------------------------------------- */

/* Size of the fixed device scratch used by dfs_fisher_pass_noalloc (8 MiB per device). */
#define DFS_NOALLOC_SCRATCH_BYTES (8u << 20)

/* The pass of dfs_fisher_pass (same arguments, same results up to rounding order) with no
 * handle and no device-memory allocation.  The paper has no counterpart: this is for callers
 * that cannot allocate device memory around the call, e.g. one whose device memory is fully
 * reserved by its own pool allocator, or one that cannot afford the implicit device-wide
 * synchronisation that cudaMalloc / cudaFree may perform.
 *
 * Device: the calling thread's current device; S, V, Y, X, R must live on it.
 * Scratch: a fixed array of DFS_NOALLOC_SCRATCH_BYTES in the library's device image holds the
 *   per-CTA partial sums and the status word.  It is reserved when the library's CUDA module
 *   is loaded on the device, not by this call.  The first call with a given device current
 *   looks up the array's address (cudaGetSymbolAddress) and the device's SM count and
 *   shared-memory limit; make that first call before any stream capture.
 * Size limit: with R != NULL the pass needs about (grid * n * kq + 2 * grid * kq) * 8 bytes of
 *   scratch, grid = one CTA per SM when n <= 1024 (up to four per SM above), kq = right-hand
 *   sides per pass (the next power of two >= k, capped by shared memory, halved here until
 *   the partials fit).  On a 152-SM GB300 that is n <= 1024 with 4 RHS per pass, or n up to
 *   about 6800 (FP32 / BF16 S) one RHS at a time.  A call that does not fit even with one RHS
 *   per pass launches nothing and returns DFS_ERR_NO_MEMORY; *scratch_bytes (host, may be
 *   NULL) receives the bytes the call needs (or needed).
 * Concurrency: all calls on one device share the one scratch array.  Calls whose work
 *   overlaps on the device (different streams with no ordering between them, or several host
 *   threads) race on it and give wrong results: order them on one stream or with events.
 * Errors: DFS_ERR_INVALID_ARG / DFS_ERR_UNSUPPORTED as dfs_fisher_pass (no message string:
 *   there is no handle), DFS_ERR_CUDA if the set-up query or a launch fails.  Asynchronous
 *   on `stream`. */
dfs_status dfs_fisher_pass_noalloc(const void* S, int s_dtype, int64_t n, int64_t m, int64_t lds,
                                   const void* V, int64_t k, int64_t ldv, const double* Y,
                                   int64_t ldy, double lambda, void* X, int64_t ldx, double* R,
                                   int64_t ldr, void* stream, int64_t* scratch_bytes);

/* The device status of the no-allocation calls queued on `stream`, which the call itself cannot
 * return without waiting for its work: waits for `stream`, then copies the status word of the
 * current device's fixed scratch into *status_out (host): DFS_OK, or DFS_ERR_TIMEOUT when a
 * bounded device wait of the pass ran out (X and R are then incomplete).  Allocates nothing.
 * The word belongs to the last no-allocation call on the device, whatever its stream.
 * DFS_ERR_INVALID_ARG if status_out is NULL or no no-allocation call has set up the device;
 * DFS_ERR_CUDA if the copy fails. */
dfs_status dfs_fisher_pass_noalloc_status(int* status_out, void* stream);

/* The test hook of dfs_set_test_fault for the no-allocation calls on the current device (the
 * fault DFS_TEST_FAULT_CLUSTER_PASS applies to them). */
dfs_status dfs_fisher_pass_noalloc_test_fault(int fault, int64_t wait_limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* DFS_H */
