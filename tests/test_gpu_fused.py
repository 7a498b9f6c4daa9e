"""The fused first pass over FP32 S (b = S v, the BF16 tensor-core tiles and the tcgen05 Gram of
Algorithm 1 in one kernel) against the FP64 oracle, and against the two-kernel form it replaces.

The BF16 Gram of FP32 S is the Gram of bf16(S) (round to nearest even), accumulated in FP32 by the
tensor cores, so the step test compares it with the oracle's Gram of the rounded values: only the
FP32 accumulation may differ (at most one unit of 2^-23 per accumulating MMA step, m / 16 steps,
relative to max W).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2310_17556_gb300 import workloads as wl

from test_gpu_parity import aligned, assert_mixed, dev, np64

pytestmark = pytest.mark.gpu

dfs = pytest.importorskip("paper_2310_17556_gb300")


@pytest.mark.parametrize("n,m", [
    (1024, 65536 + 36),   # the headline's 8 row tiles, ragged last k-block
    (100, 1000),          # one super-row, padding rows
    (130, 64),            # a single k-block
    (257, 33333),         # ragged n and m
    (777, 12345),
    (2056, 38912),        # 18 row tiles, three slot groups
    (3072, 16384),        # one slot group (U = 78)
    (4096, 4100),         # the largest one-wave schedule (U = 136)
])
def test_fused_gram_step_is_the_gram_of_bf16_rounded_s(n, m):
    lam = 0.25
    S = aligned(wl.gaussian(n, m, seed=1100 + n, device=dev()))
    W = dfs.dfs_gram(S, lam, precision="bf16")
    Sb = np64(S.to(torch.bfloat16))
    Wr = oracle.gram(Sb, lam)
    lo = np.tril(np.ones((n, n), bool))
    err = np.abs(np64(W) - Wr)[lo].max() / np.abs(Wr).max()
    assert err <= m / 16 * 2.0 ** -23 + 1e-7, err
    assert np.all(np64(W)[~lo] == 0.0)


@pytest.mark.parametrize("n,m,k,lam", [
    (1024, 65536, 1, 1e-3),
    (257, 33336, 3, 1e-3),     # four right-hand sides per group
    (777, 12345, 2, 1e-2),     # two
    (2056, 38912, 4, 1e-2),
    (130, 64, 1, 0.3),
    (3072, 16384, 1, 1e-2),
])
def test_fused_solve_matches_oracle_and_two_kernel_form(n, m, k, lam):
    S = aligned(wl.gaussian(n, m, seed=1200 + n, device=dev()))
    V = wl.rhs(m, k, seed=1201 + n, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16")
    assert info["status"] == 0, info
    ref = oracle.solve(np64(S), np64(V).T, lam).T
    assert_mixed(S, V, lam, X, ref=ref)
    X2, info2 = dfs.dfs_solve(S, V, lam, precision="bf16", two_kernel_gram=True)
    assert info2["status"] == 0, info2
    assert_mixed(S, V, lam, X2, ref=ref)
    assert info["iters"] == info2["iters"], (info, info2)


def test_fused_first_iterate_matches_two_kernel_form():
    """With one refinement pass, x_1 = (v - S^T y_0) / lambda comes straight from y_0 = W~^-1 b, so it
    carries the fused kernel's b and Gram: it must agree with the two-kernel form's x_1 up to their
    FP32 summation order (the two Grams differ by ~1e-6 relative), far below what a lost k-block or
    row of b or W would move it (>= 1e-3).  SVD-structured S with sigma_max^2 / lambda < 1 keeps
    the row-space error of x_1 proportional to that of y_0."""
    n, m, lam = 1024, 131072 + 64, 1e-3
    S, _, _, _ = wl.svd_structured(n, m, seed=1300, sigma_min=1e-3, device=dev())
    V = wl.rhs(m, 2, seed=1301, device=dev())
    X1, i1 = dfs.dfs_solve(S, V, lam, precision="bf16", max_iter=1, allow_not_converged=True)
    X2, i2 = dfs.dfs_solve(S, V, lam, precision="bf16", max_iter=1, two_kernel_gram=True,
                           allow_not_converged=True)
    S64 = np64(S)
    d = S64 @ (np64(X1) - np64(X2)).T
    base = S64 @ np64(X2).T
    rel = np.linalg.norm(d, axis=0) / np.linalg.norm(base, axis=0)
    assert rel.max() <= 1e-5, rel
    # and both first iterates are BF16-Gram accurate only: refinement has work left
    ref = oracle.solve(S64, np64(V).T, lam)
    e = oracle.errors(S64, np64(V).T, lam, np64(X1).T, ref)
    assert 1e-9 < e["e_range"] < 1e-1, e


def test_fused_solve_is_deterministic():
    """b's row sums and the Gram partials are added in a fixed order: two solves agree bit for bit."""
    n, m, lam = 1024, 262144, 1e-2
    S = wl.gaussian(n, m, seed=1400, device=dev())
    V = wl.rhs(m, 1, seed=1401, device=dev())
    X1, _ = dfs.dfs_solve(S, V, lam, precision="bf16")
    X2, _ = dfs.dfs_solve(S, V, lam, precision="bf16")
    assert torch.equal(X1, X2)
