"""Column ranges of S as ranks: the algebra of an m-sharded solve, checked on one GPU.

Eq. 1's system splits over the parameters: with S = [S_1 ... S_P] (column blocks) and v split the
same way, W = S S^T = sum_p S_p S_p^T, b = S v = sum_p S_p v_p, and the n-space residual of
Appendix A's identity r = S (v - S^T y) - lambda y = sum_p S_p (v_p - S_p^T y) - lambda y; only
x_p = (v_p - S_p^T y) / lambda stays local.  A run over P ranks would all-reduce the partials and
repeat the small n-space steps (Cholesky, triangular solves) on every rank.  Here each column range
is a "rank": the library's step entry points run on each range, the partials are summed on the
device, and the sums must match the single-range results and the FP64 oracle.

Tolerances: Gram sums against the full-range Gram within the FP32 accumulation of the kernels
(2e-5 of max|W| for the FFMA Gram; for the BF16 tensor Gram, whose operands are rounded the same
way on both sides, twice the tensor core's FP32 accumulation bound m/16 * 2^-23 of max|W|: 3e-4);
pass partials within 2e-6 relative (FP32 products folded into FP64, as in the single-step pass
test); the refined sharded solve within 1e-6 of the oracle.
"""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2310_17556_gb300 import workloads as wl

from test_gpu_parity import aligned, dev, np64

pytestmark = pytest.mark.gpu

dfs = pytest.importorskip("paper_2310_17556_gb300")

N, M, K, LAM = 300, 3 * 4096 + 1234, 2, 1e-2
CUTS = (0, 4104, 8200, M)  # three ragged ranges; starts keep 16-byte alignment for FP32 and BF16 S


def ranges():
    return list(zip(CUTS[:-1], CUTS[1:]))


def inputs(dtype):
    S = aligned(wl.gaussian(N, M, seed=231, device=dev(), dtype=dtype))
    V = wl.rhs(M, K, seed=232, device=dev())
    return S, V


def lower(W):
    return torch.tril(W.double())


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype,precision,tol", [
    (torch.float32, "fp32", 2e-5),
    (torch.float32, "bf16", 3e-4),
    (torch.bfloat16, "bf16", 3e-4),
])
def test_gram_partials_sum_to_full_gram(dtype, precision, tol):
    S, _ = inputs(dtype)
    P = len(ranges())
    Wsum = torch.zeros(N, N, device=dev(), dtype=torch.float64)
    for a, b in ranges():
        Wsum += lower(dfs.dfs_gram(S[:, a:b], LAM, precision=precision))
    # every range added lambda once; the sharded Gram adds it once
    Wsum -= (P - 1) * LAM * torch.eye(N, device=dev(), dtype=torch.float64)
    Wfull = lower(dfs.dfs_gram(S, LAM, precision=precision))
    scale = float(Wfull.abs().max())
    assert float((Wsum - Wfull).abs().max()) <= tol * scale
    ref = np.tril(oracle.gram(np64(S), LAM))
    assert np.abs(np64(Wsum) - ref).max() <= (tol if precision == "fp32" else 1e-2) * np.abs(ref).max()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_pass_partials_sum_to_full_pass(dtype):
    S, V = inputs(dtype)
    P = len(ranges())
    Y = torch.randn(N, K, device=dev(), dtype=torch.float64, generator=torch.Generator(device=dev()).manual_seed(233))
    Y *= 0.3 / math.sqrt(N / 150)
    Xfull, Rfull = dfs.dfs_fisher_pass(S, V, LAM, Y)
    Rsum = torch.zeros_like(Rfull)
    Xcat = torch.empty_like(Xfull)
    bsum = torch.zeros_like(Rfull)
    for a, b in ranges():
        Xp, Rp = dfs.dfs_fisher_pass(S[:, a:b], V[:, a:b].contiguous(), LAM, Y)
        Rsum += Rp
        Xcat[:, a:b] = Xp
        _, bp = dfs.dfs_fisher_pass(S[:, a:b], V[:, a:b].contiguous(), LAM, None, want_x=False)
        bsum += bp
    Rsum += (P - 1) * LAM * Y  # each range subtracted lambda y once; r subtracts it once
    s, v, y = np64(S), np64(V).T, np64(Y)
    r_ref = oracle.residual_n_space(s, v, y, LAM)
    assert rel(np64(Rsum), np64(Rfull)) <= 2e-6
    assert rel(np64(Rsum), r_ref) <= 2e-6
    assert rel(np64(bsum), s @ v) <= 2e-6
    assert rel(np64(Xcat), np64(Xfull)) <= 2e-6
    assert rel(np64(Xcat), ((v - s.T @ y) / LAM).T) <= 2e-6


def test_sharded_solve_over_ranges_matches_oracle():
    """Algorithm 1 with the refinement of the mixed path, the O(n^2 m) and O(nm) work done per
    range and only n-space quantities combined: BF16 Gram partials, one factorisation, then passes
    whose partial residuals are summed before each triangular-solve correction."""
    S, V = inputs(torch.float32)
    P = len(ranges())
    W = torch.zeros(N, N, device=dev(), dtype=torch.float32)
    for a, b in ranges():
        W += torch.tril(dfs.dfs_gram(S[:, a:b], LAM, precision="bf16"))
    W -= (P - 1) * LAM * torch.eye(N, device=dev(), dtype=torch.float32)
    L, piv = dfs.dfs_cholesky(W)
    assert piv == -1

    def nspace_solve(r):
        z = r.to(torch.float32).contiguous()
        dfs.dfs_trsm(L, z, trans=False)
        dfs.dfs_trsm(L, z, trans=True)
        return z.double()

    def sharded_pass(Y):
        R = torch.zeros(N, K, device=dev(), dtype=torch.float64)
        X = torch.empty_like(V)
        for a, b in ranges():
            Xp, Rp = dfs.dfs_fisher_pass(S[:, a:b], V[:, a:b].contiguous(), LAM, Y)
            R += Rp
            X[:, a:b] = Xp
        if Y is not None:
            R += (P - 1) * LAM * Y
        return X, R

    _, b = sharded_pass(None)
    Y = nspace_solve(b)
    for _ in range(4):
        X, R = sharded_pass(Y)
        Y = Y + nspace_solve(R)
    X, _ = sharded_pass(Y)
    ref = oracle.solve(np64(S), np64(V).T, LAM).T
    err = np.linalg.norm(np64(X) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert float(err.max()) <= 1e-6
