// Internal launcher declarations of libdfs (one .cu file per step of Algorithm 1).
#pragma once

#include "common.cuh"

namespace dfs {

// ---- Gram, SIMT (gram_simt.cu) ----
int gram_simt_tile(int acc_f64);
void gram_simt_plan(int64_t n, int64_t m, int acc_f64, int num_sms, int* nsplit, int64_t* chunk);
size_t gram_simt_partial_bytes(int64_t n, int acc_f64, int nsplit);
cudaError_t launch_gram_simt(int s_dtype, int acc_f64, const void* S, int64_t n, int64_t m, int64_t lds,
                             int nsplit, int64_t chunk, void* P, cudaStream_t stream);
cudaError_t launch_gram_finalize(int acc_f64, int w_f64, int BM, const void* P, int nsplit, int64_t n,
                                 int64_t n_out, double lambda, void* W, int64_t ldw, cudaStream_t stream);

// ---- Gram, tcgen05 tensor cores (gram_tc.cu) ----
// kind: 0 = BF16 MMA, 1 = TF32 MMA.
struct GramTcPlan {
    int kind;
    int packed;       // operands come from the packed tiles of the S v pass
    int n_tiles;      // T: 128-row blocks of S (of the stacked [H; L] operand for kind 2)
    int h2;           // kind 2: T_h / 2 super-rows of H (the units with J2 >= h2 are skipped); else 0
    int npairs;       // quad units (two 128-row blocks x two 128-column blocks)
    int c;            // tasks per cost unit (a unit of cost k gets c k tasks)
    int ntasks;       // tasks (k-split pieces of the units)
    int group;        // tasks per CTA group; ntasks / group partial blocks (256 x 256 FP32)
    int64_t nkb;      // 128-byte k-blocks along m
    size_t partial_bytes;
};
int gram_tc_supported(int s_dtype, int kind);
GramTcPlan gram_tc_plan(int s_dtype, int kind, int64_t n, int64_t m, int num_sms);
cudaError_t launch_gram_tc(const GramTcPlan& plan, int s_dtype, const void* S, int64_t n, int64_t m, int64_t lds,
                           const void* Sp, void* P, DevStatus* st, cudaStream_t stream);
cudaError_t launch_gram_tc_finalize(const GramTcPlan& plan, const void* P, int64_t n, int64_t n_out, double lambda,
                                    void* W, int64_t ldw, cudaStream_t stream, const float* rscale = nullptr);

// ---- first pass + Gram as one kernel (gram_fused.cu) ----
// FP32 S, BF16 tiles, kq <= 4 right-hand sides, one-wave schedule; returns 0 where it does not apply.
int gram_fused_plan(int s_dtype, int64_t n, int64_t m, int kq, int num_sms, size_t smem_optin, GramTcPlan* plan);
size_t gram_fused_ready_bytes(const GramTcPlan& plan);
// b = S V into Rpart (num_sms rows of n x kq FP64; *parts = num_sms), the BF16 tiles into Sp, the
// Gram partial blocks into P (read by launch_gram_tc_finalize); `ready` is per-k-block scratch.
// k = 0 (V unused): the tiles and the Gram only.
cudaError_t launch_gram_fused(const GramTcPlan& plan, int kq, const void* S, int64_t n, int64_t m, int64_t lds,
                              const void* V, int64_t ldv, int k, double* Rpart, void* Sp, void* P, int* ready,
                              DevStatus* st, int num_sms, cudaStream_t stream, int* parts);

// ---- Cholesky (cholesky.cu) ----
// fp64_panel: factor the 32 x 32 diagonal blocks in FP64 (else in the storage type).
// flags: cholesky_flag_bytes(n_pad) of device scratch (zeroed by the launcher).
size_t cholesky_flag_bytes(int64_t n_pad);
// share > 1: the kernel takes 1 / share of the resident-CTA capacity (concurrent factorisations).
cudaError_t launch_cholesky(int w_f64, void* W, int64_t ld, int64_t n_pad, void* Linv, int* flags, DevStatus* st,
                            cudaStream_t stream, int fp64_panel = 1, int share = 1);
cudaError_t launch_diag_inverse(int w_f64, const void* L, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                                cudaStream_t stream);

// ---- n-space step: reduction of the pass partials + both triangular solves (nspace.cu) ----
constexpr int NS_MODE_REDUCE = 1;    // right-hand side = sum of Rpart (else read from B)
constexpr int NS_MODE_LAMBDA_Y = 2;  // subtract lambda Y
constexpr int NS_MODE_FWD = 4;       // L a = r
constexpr int NS_MODE_BWD = 8;       // L^T z = a
int nspace_slots(int n_pad, int KQ, int elem, size_t smem_limit);  // >= 2 when the kernel applies
cudaError_t launch_nspace(int f64, int kq, const void* W, int64_t ld, int n_pad, const void* Linv, int mode,
                          const double* Rpart, int nparts, int n, int k, const double* Y, double lambda, const void* B,
                          int64_t ldb, double* R, void* Z, int64_t ldz, const double* U2part, double* U2,
                          size_t smem_limit, DevStatus* st, int honor_stop, cudaStream_t stream);

// ---- triangular solves (trsv.cu) ----
size_t trsv_smem_bytes(int n_pad, int KQ, int elem, int nst);
cudaError_t launch_mirror_lower(int f64, void* L, int64_t ld, int n_pad, cudaStream_t stream);
int trsv_max_group(int n_pad, int elem, size_t smem_limit);
cudaError_t launch_trsv(int f64, int trans, const void* L, int64_t ld, int n_pad, const void* Linv, void* B,
                        int64_t ldb, int k, int kq, const DevStatus* st, int honor_stop, cudaStream_t stream);

// ---- streaming passes over S (pass.cu) ----
struct PassPlan {
    int rpt;      // rows per thread kept in registers by the refinement pass (0: re-read mode)
    int grid;     // CTAs of fisher_pass_kernel
    int sv_grid;  // CTAs of sv_pack_kernel
    int cs;       // > 0: the refinement pass runs as clusters of cs CTAs (pass_cluster.cu)
    int crpt;     // rows per thread of the cluster form
    int ncl;      // clusters
    int nparts;   // partial rows of R (Rpart) the refinement pass writes
    int uparts;   // partial rows of the U^2 / dX^2 sums (U2part) it writes
    int two;      // 1: the pass runs as sty_cols_kernel (X) then sv_rows_kernel (R) (large n)
};
int pass_cluster_plan(int s_dtype, int n, int KQ, int num_sms, int64_t m, size_t smem_limit, int* cs_out,
                      int* rpt_out);
cudaError_t launch_pass_cluster(int ncl, int cs, int rpt, int kq, const void* S, int n, int64_t m, int64_t lds,
                                const void* V, int64_t ldv, int k, const double* Y, int64_t ldy, double lambda,
                                void* X, int64_t ldx, double* Rpart, double* U2part, int dmode, const DevStatus* st,
                                int honor_stop, cudaStream_t stream);
size_t pass_smem_bytes(int n, int KQ, int s_dtype);
int pass_max_group(int n, int s_dtype, size_t smem_limit);
int pass_grid(int n, int KQ, int s_dtype, int num_sms, int64_t m);
// allow_two = 0: keep the one-kernel pass (the two-kernel form needs an X output to carry U)
PassPlan pass_make_plan(int n, int KQ, int s_dtype, int num_sms, int64_t m, size_t smem_limit, int allow_two = 1);
int pass_partial_rows(const PassPlan& p);  // rows of the partial buffers (max of both grids)
// pack: 0 none, 1 BF16 tiles, 2 TF32 tiles, 3 stacked BF16 H / L tiles, 4 row-scaled e4m3 tiles
// (rinv: the inverse row scales from launch_row_scale) (see sv_pack_kernel)
cudaError_t launch_row_scale(int s_dtype, const void* S, int n, int n_pad, int64_t m, int64_t lds, float* rs,
                             const DevStatus* st, cudaStream_t stream);
int64_t pack_kblocks(int s_dtype, int pack, int64_t m);
size_t pack_bytes(int s_dtype, int pack, int64_t n, int64_t m);
cudaError_t launch_sv_pack(const PassPlan& plan, int s_dtype, int kq, int pack, const void* S, int n, int64_t m,
                           int64_t lds, const void* V, int64_t ldv, int k, double* Rpart, void* Sp,
                           const DevStatus* st, cudaStream_t stream, const float* rinv = nullptr,
                           int* parts = nullptr);  // *parts: the partial rows of R written (for the reduce)
// dmode: 0 = no change measurement, 1 = also sum (X_new - X_old)^2 with X_old read from X,
// 2 = same with X_old = V / lambda.  U2part holds 2 * kq doubles per CTA: sum U^2, sum dX^2.
cudaError_t launch_pass(const PassPlan& plan, int s_dtype, int kq, const void* S, int n, int64_t m, int64_t lds,
                        const void* V, int64_t ldv, int k, const double* Y, int64_t ldy, double lambda, void* X,
                        int64_t ldx, double* Rpart, double* U2part, int dmode, const DevStatus* st, int honor_stop,
                        cudaStream_t stream);
cudaError_t launch_pass_reduce(int f64, const double* Rpart, int nparts, int n, int n_out, int KQ, int k,
                               const double* Y, int64_t ldy, double lambda, double* R, int64_t ldr, void* Rt,
                               const double* U2part, double* U2, const DevStatus* st, int honor_stop,
                               cudaStream_t stream);

// ---- centred score matrices, S = (O - O_bar) / sqrt(n) (center.cu) ----
// W (lower, rows < n, holding G = O O^T without lambda) <- P G P / n + lambda I; scratch holds
// center_gram_scratch_doubles(n) doubles.
cudaError_t launch_center_gram(int f64, void* W, int64_t ld, int n, double* scratch, double lambda,
                               cudaStream_t stream);
size_t center_gram_scratch_doubles(int64_t n);
// mode 0: R <- P R / sqrt(n) - lambda Y (Y may be null), Z <- R; mode 1: Yc <- P Y / sqrt(n).
// R, Y, Yc, Z: n_pad x KQ row-major (KQ <= 8).
cudaError_t launch_center_vec(int f64, int mode, int n, int n_pad, int KQ, int k, double* R, const double* Y,
                              double lambda, void* Z, double* Yc, const DevStatus* st, int honor_stop,
                              cudaStream_t stream);

// ---- complex scores (complex.cu): the glue of the native complex solve on Z = [Re S; Im S] ----
// r = R(S) u - lambda y (or b = S v without Y) from the pass partials over Z (KQP columns, the
// complex RHS q in columns q and kc + q) into R (FP64) and Zb (solve type), n_pad x KQN; folds the
// per-part stopping sums U2part (uparts x 2 KQP) into U2c (uparts x 2 KQN) when U2part is given
cudaError_t launch_complex_combine(int f64, const double* P, int nparts, int n, int kc, int KQP, const double* Y,
                                   double lambda, double* R, void* Zb, int KQN, int n_pad, const double* U2part,
                                   int uparts, double* U2c, const DevStatus* st, int honor_stop, cudaStream_t stream);
// the pass's y (2n x KQP, FP64) from the real n-space y (rows 0..2n-1, stride KQN)
cudaError_t launch_complex_yexp(const double* Y, int KQN, int n, int kc, int KQP, double* Yp, const DevStatus* st,
                                int honor_stop, cudaStream_t stream);
// the same from an FP32 n-space correction into rows_out x KQP FP32 (the packed-tile correction's dy)
cudaError_t launch_complex_dyexp(const float* Z, int KQN, int n, int kc, int KQP, float* dy, int rows_out,
                                 const DevStatus* st, int honor_stop, cudaStream_t stream);
// R(W) + lambda I~ (lower, n_pad x n_pad, ld) from the stacked Gram G = Z Z^T (lower, same shape)
cudaError_t launch_complex_assemble(int f64, const void* G, int64_t ld, int n, int n_pad, double lambda, void* W,
                                    cudaStream_t stream);

// ---- refinement control and small utilities (refine.cu, util.cu) ----
// wait_ns: limit of the call's bounded device waits (0: the 2 s default); fault: a test hook's
// DFS_TEST_FAULT_* (0 normally)
cudaError_t launch_status_reset(DevStatus* st, cudaStream_t stream, unsigned long long wait_ns = 0, int fault = 0);
cudaError_t launch_group_reset(DevStatus* st, cudaStream_t stream);
cudaError_t launch_status_save(const DevStatus* st, int* dst, cudaStream_t stream);
cudaError_t launch_refine_init(int f64, const void* Z, int n_pad, int KQ, double* Y, const double* R,
                               double* bnorm2, DevStatus* st, cudaStream_t stream);
// after a pass (or the tile correction, fast = 1): U2 = sum of U2part, the error estimate and the
// stop decision (refine.cu)
cudaError_t launch_refine_check(const double* U2part, int nparts, double* U2, int KQ, int k, double lambda, double tol,
                                int it, int max_iter, int fast, DevStatus* st, cudaStream_t stream);
// after the n-space solve of a step that did not stop: y += dy and the n-space residual norm
cudaError_t launch_refine_update(int f64, const void* Z, const double* R, int n_pad, int KQ, int k, double* Y,
                                 const double* bnorm2, DevStatus* st, cudaStream_t stream);
// x -= S^T dy / lambda from the packed BF16 tiles (pass.cu), with the per-part sums of the passes;
// grid = the SM count; the parts it writes (at most tile_correct_parts(num_sms)) are returned by
// the launch through *parts
int tile_correct_parts(int num_sms);
bool tile_correct_fits(int n_rows, int kq, size_t smem_limit);
cudaError_t launch_tile_correct(int kq, const void* Sp, int n, int n_rows, int64_t m, int64_t nkb, const float* Z,
                                int k, double lambda, float* X, int64_t ldx, double* U2part, const DevStatus* st,
                                int grid, cudaStream_t stream, int* parts);
cudaError_t launch_pad_copy_in(int f64, const void* src, int64_t lds, int64_t n, void* dst, int64_t n_pad,
                               cudaStream_t stream);
cudaError_t launch_copy_lower_out(int f64, const void* src, int64_t n_pad, void* dst, int64_t ldd, int64_t n,
                                  cudaStream_t stream);
cudaError_t launch_copy_rhs_in(int f64, const void* src, int64_t lds, int64_t n, int k, void* dst, int KQ,
                               int64_t n_pad, cudaStream_t stream);
cudaError_t launch_copy_rhs_out(int f64, const void* src, int KQ, int64_t n, int k, void* dst, int64_t ldd,
                                cudaStream_t stream);

}  // namespace dfs
