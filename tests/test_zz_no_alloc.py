"""dfs_fisher_pass_noalloc (fixed device scratch, no allocation) against dfs_fisher_pass.

Collected last on purpose: the no-allocation entry point must give the handle-based pass's
results both in a fresh process and after every other test has run on the device.
"""

import pytest
import torch

import paper_2310_17556_gb300 as dfs
from paper_2310_17556_gb300 import workloads as wl
from paper_2310_17556_gb300._lib import DFS_ERR_NO_MEMORY, DFS_NOALLOC_SCRATCH_BYTES

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
