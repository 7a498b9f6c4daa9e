"""dfs_fisher_pass_noalloc (fixed device scratch, no allocation) against the FP64 oracle and
against dfs_fisher_pass, and its device status.

Collected last on purpose: the no-allocation entry point must give the handle-based pass's
results both in a fresh process and after every other test has run on the device.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_2310_17556_gb300 as dfs
from paper_2310_17556_gb300 import workloads as wl
from paper_2310_17556_gb300._lib import (DFS_ERR_NO_MEMORY, DFS_ERR_TIMEOUT, DFS_NOALLOC_SCRATCH_BYTES, DFS_OK,
                                         DFS_TEST_FAULT_CLUSTER_PASS, DFS_TEST_FAULT_NONE)

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _inputs(n, m, k, dtype, seed, with_y):
    S = wl.gaussian(n, m, seed, device=DEV, dtype=dtype)
    vdt = torch.float64 if dtype == torch.float64 else torch.float32
    V = wl.rhs(m, k, seed + 1, device=DEV, dtype=vdt)
    Y = None
    if with_y:
        g = torch.Generator(device=DEV)
        g.manual_seed(seed + 2)
        Y = torch.randn((n, k), generator=g, device=DEV, dtype=torch.float64) * 0.1
    return S, V, Y


def _close(a, b, rtol):
    scale = b.abs().max().item() + 1e-300
    err = (a.double() - b.double()).abs().max().item()
    assert err <= rtol * scale, f"max |diff| {err:.3e} > {rtol:.1e} * {scale:.3e}"


@pytest.mark.parametrize("n,m,k,dtype,with_y", [
    (1024, 200_003 + 1, 1, torch.float32, True),    # register-resident strips, ragged tail
    (300, 65_536, 3, torch.float32, False),          # three RHS in one pass (kq = 4)
    (1024, 131_072, 2, torch.bfloat16, True),
    (257, 40_000, 1, torch.float64, True),
    (1500, 50_000, 1, torch.float32, True),          # n > 1024: strips re-read from L2
])
def test_noalloc_matches_handle_pass_twice(n, m, k, dtype, with_y):
    S, V, Y = _inputs(n, m, k, dtype, 4100 + n, with_y)
    lam = 1e-2
    X_ref, R_ref = dfs.dfs_fisher_pass(S, V, lam, Y=Y)
    rtol_x = 1e-12 if dtype == torch.float64 else 1e-6
    rtol_r = 1e-12 if dtype == torch.float64 else 1e-6
    for _ in range(2):  # two calls in a row reuse the same fixed scratch
        X = torch.full_like(V, float("nan"))
        R = torch.full((n, k), float("nan"), device=DEV, dtype=torch.float64)
        dfs.dfs_fisher_pass_noalloc(S, V, lam, Y=Y, X=X, R=R)
        torch.cuda.synchronize()
        assert torch.isfinite(X).all() and torch.isfinite(R).all()
        _close(X, X_ref, rtol_x)
        _close(R, R_ref, rtol_r)


def test_noalloc_x_only_and_r_only():
    S, V, Y = _inputs(512, 100_000, 1, torch.float32, 77, True)
    X_ref, R_ref = dfs.dfs_fisher_pass(S, V, 0.5, Y=Y)
    X = torch.empty_like(V)
    dfs.dfs_fisher_pass_noalloc(S, V, 0.5, Y=Y, X=X)
    R = torch.empty((512, 1), device=DEV, dtype=torch.float64)
    dfs.dfs_fisher_pass_noalloc(S, V, 0.5, Y=Y, R=R)
    torch.cuda.synchronize()
    _close(X, X_ref, 1e-6)
    _close(R, R_ref, 1e-6)


def test_noalloc_rejects_oversize_partials():
    # n = 8192 FP32 with R: about 2 CTAs per SM x 8192 rows x 8 bytes of partials per CTA, well
    # above the fixed scratch even with one RHS per pass.
    n, m = 8192, 16_384
    S = torch.zeros((n, m), device=DEV, dtype=torch.float32)
    V = torch.ones((1, m), device=DEV, dtype=torch.float32)
    R = torch.empty((n, 1), device=DEV, dtype=torch.float64)
    with pytest.raises(dfs.DfsError) as ei:
        dfs.dfs_fisher_pass_noalloc(S, V, 1.0, R=R)
    assert ei.value.status == DFS_ERR_NO_MEMORY
    assert str(DFS_NOALLOC_SCRATCH_BYTES) in str(ei.value)
    # the same call without R needs only the small per-CTA sums and runs
    X = torch.empty_like(V)
    dfs.dfs_fisher_pass_noalloc(S, V, 1.0, X=X)
    torch.cuda.synchronize()
    assert torch.equal(X, V)


def _np64(t):
    return t.detach().to("cpu").to(torch.float64).numpy()


@pytest.mark.parametrize("n,m,k,dtype", [(1024, 100_004, 1, torch.float32), (300, 40_000, 3, torch.float32),
                                         (257, 20_000, 2, torch.float64)])
def test_noalloc_matches_the_oracle(n, m, k, dtype):
    """X = (V - S^T Y) / lambda and R = S (V - S^T Y) - lambda Y (Appendix A's n-space residual)
    against the oracle's FP64 restatement, on the stored values."""
    S, V, Y = _inputs(n, m, k, dtype, 4300 + n, True)
    lam = 1e-2
    X = torch.empty_like(V)
    R = torch.empty((n, k), device=DEV, dtype=torch.float64)
    dfs.dfs_fisher_pass_noalloc(S, V, lam, Y=Y, X=X, R=R)
    assert dfs.dfs_fisher_pass_noalloc_status() == DFS_OK
    S64, V64, Y64 = _np64(S), _np64(V), _np64(Y)
    X_ref = (V64.T - S64.T @ Y64).T / lam
    R_ref = oracle.residual_n_space(S64, V64.T, Y64, lam)
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    assert np.abs(_np64(X) - X_ref).max() <= tol * np.abs(X_ref).max()
    assert np.abs(_np64(R) - R_ref).max() <= 10 * tol * np.abs(R_ref).max()


def test_noalloc_two_kernel_form():
    """n > 2048 with X given and a 4096-column chunk for every SM: the pass runs as its two
    row-shared kernels (x, then R from x), whose partials are laid out differently.  Against
    dfs_fisher_pass, and against FP64 sums (torch, column chunks) of the same formulas."""
    n, m, k, lam = 2056, 622_592, 1, 1e-2
    S, V, Y = _inputs(n, m, k, torch.bfloat16, 4400, True)
    X_ref, R_ref = dfs.dfs_fisher_pass(S, V, lam, Y=Y)
    X = torch.empty_like(V)
    R = torch.empty((n, k), device=DEV, dtype=torch.float64)
    for _ in range(2):
        X.fill_(float("nan"))
        R.fill_(float("nan"))
        dfs.dfs_fisher_pass_noalloc(S, V, lam, Y=Y, X=X, R=R)
        assert dfs.dfs_fisher_pass_noalloc_status() == DFS_OK
        _close(X, X_ref, 1e-6)
        _close(R, R_ref, 1e-6)
    U = torch.empty((k, m), device=DEV, dtype=torch.float64)
    R64 = -lam * Y.clone()
    for c0 in range(0, m, 1 << 17):
        Sc = S[:, c0:c0 + (1 << 17)].double()
        U[:, c0:c0 + (1 << 17)] = V[:, c0:c0 + (1 << 17)].double() - (Sc.T @ Y).T
        R64 += Sc @ U[:, c0:c0 + (1 << 17)].T
    _close(X, U / lam, 1e-6)
    _close(R, R64, 1e-5)


def test_noalloc_allocates_no_device_memory():
    S, V, Y = _inputs(1024, 200_000, 1, torch.float32, 4500, True)
    X = torch.empty_like(V)
    R = torch.empty((1024, 1), device=DEV, dtype=torch.float64)
    dfs.dfs_fisher_pass_noalloc(S, V, 1e-2, Y=Y, X=X, R=R)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        dfs.dfs_fisher_pass_noalloc(S, V, 1e-2, Y=Y, X=X, R=R)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert dfs.dfs_fisher_pass_noalloc_status() == DFS_OK


def test_noalloc_status_reports_a_wait_that_ran_out():
    """The call cannot return the device's verdict without waiting for its work: the status
    companion reads it from the fixed scratch.  With rank 1 of the first cluster withholding its
    partial sums (test hook, 5 ms wait limit) the other ranks' waits run out: DFS_ERR_TIMEOUT.
    The next call, hook off, is whole again."""
    n, m, lam = 1024, 100_000, 1e-2
    S, V, Y = _inputs(n, m, 1, torch.float32, 4600, True)
    X = torch.empty_like(V)
    R = torch.empty((n, 1), device=DEV, dtype=torch.float64)
    try:
        dfs.dfs_fisher_pass_noalloc_test_fault(DFS_TEST_FAULT_CLUSTER_PASS, 5_000_000)
        dfs.dfs_fisher_pass_noalloc(S, V, lam, Y=Y, X=X, R=R)
        assert dfs.dfs_fisher_pass_noalloc_status() == DFS_ERR_TIMEOUT
    finally:
        dfs.dfs_fisher_pass_noalloc_test_fault(DFS_TEST_FAULT_NONE, 0)
    dfs.dfs_fisher_pass_noalloc(S, V, lam, Y=Y, X=X, R=R)
    assert dfs.dfs_fisher_pass_noalloc_status() == DFS_OK
    X_ref, R_ref = dfs.dfs_fisher_pass(S, V, lam, Y=Y)
    _close(X, X_ref, 1e-6)
    _close(R, R_ref, 1e-6)
