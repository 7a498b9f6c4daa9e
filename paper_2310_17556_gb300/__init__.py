"""Cholesky solve of the damped Fisher system on GB300 (arXiv 2310.17556, Algorithm 1).

(S^T S + lambda I) x = v for a wide score matrix S (n x m, m >> n), with every step in
hand-written sm_103a CUDA kernels behind the C ABI of include/dfs.h (libdfs.so).  This
package is the thin Python binding: same entry-point names, torch tensors in and out.
"""

from .api import (  # noqa: F401
    DfsError,
    Handle,
    NotConvergedError,
    default_handle,
    dfs_cholesky,
    dfs_fisher_pass,
    dfs_fisher_pass_noalloc,
    dfs_fisher_pass_noalloc_status,
    dfs_fisher_pass_noalloc_test_fault,
    dfs_set_test_fault,
    dfs_gram,
    dfs_measure_peak,
    dfs_kernel_launches,
    dfs_reserve,
    dfs_solve,
    dfs_solve_batched,
    dfs_plan_batched,
    dfs_batched_status,
    dfs_set_batch_lanes,
    dfs_get_batch_lanes,
    dfs_autotune_batched,
    dfs_solve_host,
    dfs_solve_host_async,
    dfs_solve_complex,
    dfs_step_times,
    dfs_sync_info,
    dfs_trsm,
)
