"""Failure detection on the device, in forms that fault and hang nothing.

Every device-side wait of the library is bounded: when a wait runs out the kernel records
DFS_ERR_TIMEOUT, releases what it holds and returns, and the next call on the handle works.  The
test hook (dfs_set_test_fault) makes one kernel withhold one signal and shortens the limit to a
few milliseconds, so that the bounded waits for that signal run out.  Refinement that stops above
its tolerance reports DFS_ERR_NOT_CONVERGED, which the binding raises unless the caller allows it.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2310_17556_gb300 import DfsError, NotConvergedError, workloads as wl
from paper_2310_17556_gb300._lib import (DFS_ERR_NOT_CONVERGED, DFS_ERR_TIMEOUT, DFS_TEST_FAULT_CHOLESKY,
                                         DFS_TEST_FAULT_CLUSTER_PASS, DFS_TEST_FAULT_FUSED_GRAM,
                                         DFS_TEST_FAULT_NONE)

from test_gpu_parity import aligned, assert_mixed, dev, fp32_tol, np64, rel_err, solve_ref

pytestmark = pytest.mark.gpu

dfs = pytest.importorskip("paper_2310_17556_gb300")

SHORT_NS = 5_000_000  # 5 ms


@pytest.mark.parametrize("fault,prec,n,m", [
    (DFS_TEST_FAULT_CHOLESKY, "fp32", 512, 20000),       # the Cholesky's flag waits
    (DFS_TEST_FAULT_CHOLESKY, "fp32", 2304, 20000),      # the same with the per-warp trailing tiles
    (DFS_TEST_FAULT_CLUSTER_PASS, "bf16", 1024, 65536),  # the refinement pass's cluster exchange
    (DFS_TEST_FAULT_FUSED_GRAM, "bf16", 1024, 65536),    # the fused first pass's tile waits
])
def test_withheld_signal_times_out_and_the_handle_recovers(fault, prec, n, m):
    lam = 1e-2
    S = aligned(wl.gaussian(n, m, seed=1500 + fault, device=dev()))
    V = wl.rhs(m, 1, seed=1501 + fault, device=dev())
    h = dfs.Handle()
    try:
        dfs.dfs_set_test_fault(fault, SHORT_NS, handle=h)
        with pytest.raises(DfsError) as e:
            dfs.dfs_solve(S, V, lam, precision=prec, handle=h)
        assert e.value.status == DFS_ERR_TIMEOUT, e.value
        # the context is intact and the handle starts afresh
        dfs.dfs_set_test_fault(DFS_TEST_FAULT_NONE, 0, handle=h)
        X, info = dfs.dfs_solve(S, V, lam, precision=prec, handle=h)
        assert info["status"] == 0, info
        if prec == "fp32":
            assert rel_err(np64(X), solve_ref(S, V, lam)) <= fp32_tol(S, lam)
        else:
            assert_mixed(S, V, lam, X)
    finally:
        h.close()
    torch.cuda.synchronize()


def test_not_converged_raises_and_returns_the_last_iterate():
    """One refinement pass cannot confirm convergence (the stopping rule needs the rate of two
    successive changes): DFS_ERR_NOT_CONVERGED, raised as NotConvergedError carrying x and the
    info; with allow_not_converged the same call returns them.  The iterate is the one pass's x,
    better than x_0 = v / lambda and short of the converged 1e-6."""
    n, m, lam = 512, 40000, 1e-3
    S = aligned(wl.gaussian(n, m, seed=1600, device=dev()))
    V = wl.rhs(m, 1, seed=1601, device=dev())
    with pytest.raises(NotConvergedError) as e:
        dfs.dfs_solve(S, V, lam, precision="fp8", max_iter=1)
    assert e.value.status == DFS_ERR_NOT_CONVERGED
    assert e.value.info["status"] == DFS_ERR_NOT_CONVERGED and e.value.info["iters"] == 1
    X, info = dfs.dfs_solve(S, V, lam, precision="fp8", max_iter=1, allow_not_converged=True)
    assert info["status"] == DFS_ERR_NOT_CONVERGED
    assert torch.equal(X, e.value.X)
    ref = solve_ref(S, V, lam)
    err = rel_err(np64(X), ref)
    err0 = rel_err(np64(V) / lam, ref)
    assert np.isfinite(err) and err < err0, (err, err0)
    # the same problem converges when refinement may continue
    X2, info2 = dfs.dfs_solve(S, V, lam, precision="fp8", max_iter=20)
    assert info2["status"] == 0
    assert_mixed(S, V, lam, X2)


def test_unknown_test_fault_is_rejected():
    with pytest.raises(DfsError):
        dfs.dfs_set_test_fault(99, 0)
