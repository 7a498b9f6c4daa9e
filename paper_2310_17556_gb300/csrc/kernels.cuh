// Internal launcher declarations of libdfs (one .cu file per step of Algorithm 1).
#pragma once

#include "common.cuh"

namespace dfs {

// ---- step 1, SIMT Gram (gram_simt.cu) ----
int gram_simt_tile(int acc_f64);
void gram_simt_plan(int64_t n, int64_t m, int acc_f64, int num_sms, int* nsplit, int64_t* chunk);
size_t gram_simt_partial_bytes(int64_t n, int acc_f64, int nsplit);
cudaError_t launch_gram_simt(int s_dtype, int acc_f64, const void* S, int64_t n, int64_t m, int64_t lds,
                             int nsplit, int64_t chunk, void* P, cudaStream_t stream);
cudaError_t launch_gram_finalize(int acc_f64, int w_f64, int BM, const void* P, int nsplit, int64_t n,
                                 int64_t n_out, double lambda, void* W, int64_t ldw, cudaStream_t stream);

// ---- step 1, tcgen05 tensor-core Gram (gram_tc.cu) ----
// kind: 0 = BF16 (S converted on chip), 1 = TF32, 2 = split BF16 x3.
struct GramTcPlan {
    int kind;
    int n_tiles;      // 128-row tiles of S (rows padded to 128)
    int nsplit;       // split-m chunks
    int64_t chunk;    // columns per chunk (multiple of the k-block)
    int ngroups;      // output work groups per chunk
    size_t partial_bytes;
};
int gram_tc_supported(int s_dtype, int kind);
GramTcPlan gram_tc_plan(int s_dtype, int kind, int64_t n, int64_t m, int num_sms);
cudaError_t launch_gram_tc(const GramTcPlan& plan, int s_dtype, const void* S, int64_t n, int64_t m, int64_t lds,
                           void* P, DevStatus* st, cudaStream_t stream);
cudaError_t launch_gram_tc_finalize(const GramTcPlan& plan, const void* P, int64_t n, int64_t n_out, double lambda,
                                    void* W, int64_t ldw, cudaStream_t stream);

// ---- step 2, Cholesky (cholesky.cu) ----
cudaError_t launch_cholesky(int w_f64, void* W, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                            cudaStream_t stream);
cudaError_t launch_diag_inverse(int w_f64, const void* L, int64_t ld, int64_t n_pad, void* Linv, DevStatus* st,
                                cudaStream_t stream);

// ---- triangular solves (trsv.cu) ----
size_t trsv_smem_bytes(int n_pad, int KQ, int elem);
int trsv_max_group(int n_pad, int elem, size_t smem_limit);
cudaError_t launch_trsv(int f64, int trans, const void* L, int64_t ld, int n_pad, const void* Linv, void* B,
                        int64_t ldb, int k, int kq, const DevStatus* st, int honor_stop, cudaStream_t stream);

// ---- streaming pass over S (pass.cu) ----
size_t pass_smem_bytes(int n, int KQ, int s_dtype);
int pass_max_group(int n, int s_dtype, size_t smem_limit);
int pass_grid(int n, int KQ, int s_dtype, int num_sms, int64_t m);
cudaError_t launch_pass(int s_dtype, int kq, const void* S, int n, int64_t m, int64_t lds, const void* V,
                        int64_t ldv, int k, const double* Y, int64_t ldy, double lambda, void* X, int64_t ldx,
                        double* Rpart, double* U2part, int grid, const DevStatus* st, int honor_stop,
                        cudaStream_t stream);
cudaError_t launch_pass_reduce(int f64, const double* Rpart, int nparts, int n, int n_out, int KQ, int k,
                               const double* Y, int64_t ldy, double lambda, double* R, int64_t ldr, void* Rt,
                               const double* U2part, double* U2, const DevStatus* st, int honor_stop,
                               cudaStream_t stream);

// ---- refinement control and small utilities (refine.cu, util.cu) ----
cudaError_t launch_status_reset(DevStatus* st, cudaStream_t stream);
cudaError_t launch_group_reset(DevStatus* st, cudaStream_t stream);
cudaError_t launch_status_save(const DevStatus* st, int* dst, cudaStream_t stream);
cudaError_t launch_refine_init(int f64, const void* Z, int n_pad, int KQ, double* Y, const double* R,
                               double* bnorm2, DevStatus* st, cudaStream_t stream);
cudaError_t launch_refine_control(int f64, const void* Z, const double* R, int n_pad, int KQ, int k, double* Y,
                                  const double* U2, const double* bnorm2, double lambda, double tol, int it,
                                  int max_iter, DevStatus* st, cudaStream_t stream);
cudaError_t launch_pad_copy_in(int f64, const void* src, int64_t lds, int64_t n, void* dst, int64_t n_pad,
                               cudaStream_t stream);
cudaError_t launch_copy_lower_out(int f64, const void* src, int64_t n_pad, void* dst, int64_t ldd, int64_t n,
                                  cudaStream_t stream);
cudaError_t launch_copy_rhs_in(int f64, const void* src, int64_t lds, int64_t n, int k, void* dst, int KQ,
                               int64_t n_pad, cudaStream_t stream);
cudaError_t launch_copy_rhs_out(int f64, const void* src, int KQ, int64_t n, int k, void* dst, int64_t ldd,
                                cudaStream_t stream);

}  // namespace dfs
