"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and end to end.

Inputs come from the seeded generators; the oracle gets the exact stored values (widened to
FP64).  Tolerances:
  * FP64 path: e_rel <= 1e-10 (FP64 arithmetic throughout; cond(A) <= ~1e3 here).
  * FP32 path: e_rel <= 1e-5 (the plain-FP32 bar); Gram entries within 2e-5 * max|W|.
  * mixed paths (tensor Gram + refinement): e_rel <= 1e-6.
"""

import json
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2310_17556_gb300 import DfsError, workloads as wl

pytestmark = pytest.mark.gpu

dfs = pytest.importorskip("paper_2310_17556_gb300")


def dev():
    return torch.device("cuda", 0)


def np64(t):
    return t.detach().to("cpu").to(torch.float64).numpy()


def solve_ref(S, V, lam):
    """Oracle x for S (n, m) and V (k, m) torch tensors; returns (k, m) float64."""
    return oracle.solve(np64(S), np64(V).T, lam).T


def aligned(t):
    """Same values with a row stride that is a multiple of 16 bytes (the C ABI's S contract)."""
    per = 16 // t.element_size()
    m = t.shape[1]
    lds = -(-m // per) * per
    if lds == m:
        return t.contiguous()
    buf = torch.zeros((t.shape[0], lds), device=t.device, dtype=t.dtype)
    buf[:, :m] = t
    return buf[:, :m]


def fp32_tol(S, lam):
    """The plain FP32 path (no refinement) carries FP32 rounding of W and of its factor, amplified
    by cond(W) = (sigma_max^2 + lambda) / (sigma_min^2 + lambda) (sigma_min = 0 when m < n).  The
    1e-5 bar is for cond(W) <= 10 (the SVD-structured workload has cond(W) <= 11); beyond that the
    bar grows in proportion."""
    sv = np.linalg.svd(np64(S), compute_uv=False)
    smin = sv[-1] if S.shape[1] >= S.shape[0] else 0.0
    cond = (sv[0] ** 2 + lam) / (smin ** 2 + lam)
    return 1e-5 * max(1.0, cond / 10.0)


def sigma_max_sq(S64):
    """Largest eigenvalue of S S^T (FP64, from the n x n or m x m Gram)."""
    G = S64 @ S64.T if S64.shape[0] <= S64.shape[1] else S64.T @ S64
    return float(np.linalg.eigvalsh(G)[-1])


def row_space_amplification(S64, V64, lam):
    """A = sigma_max (sigma_max^2 + lam) / lam * ||v|| / ||S v||, per right-hand side (V64 is (k, m)).

    For any x with ||x - x*|| <= eps ||x*||, e_range <= A eps: ||S d|| <= sigma_max ||d||, S x* = y*
    with (S S^T + lam I) y* = S v, so ||y*|| >= ||S v|| / (sigma_max^2 + lam), and ||x*|| <= ||v|| / lam.
    A is large where sigma_max^2 / lam is (Gaussian scores at small lam); there e_rel, diluted by
    the v / lam part of x*, says little about the row space and e_range is the sharper check."""
    s_max = math.sqrt(sigma_max_sq(S64))
    SV = S64 @ V64.T
    return s_max * (s_max ** 2 + lam) / lam * np.linalg.norm(V64, axis=1) / np.linalg.norm(SV, axis=0)


STOP_TOL = 1e-7  # the solver's default stopping tolerance (estimated relative error of x)


def range_bar(S64, V64, lam, base=1e-6):
    """e_range bar of the refined paths: 1e-6, or the row-space error that twice the stopping
    tolerance allows through the amplification A (whichever is larger)."""
    return max(base, 2.0 * STOP_TOL * float(row_space_amplification(S64, V64, lam).max()))


def assert_mixed(S, V, lam, X, ref=None, e_rel_tol=1e-6, e_range_tol=1e-6):
    """Mixed paths after refinement: e_rel <= 1e-6, and the error inside the row space of S (where
    e_rel is diluted by the v / lam part of x*) within range_bar."""
    S64, V64, X64 = np64(S), np64(V), np64(X)
    if ref is None:
        ref = oracle.solve(S64, V64.T, lam).T
    e = oracle.errors(S64, V64.T, lam, X64.T, ref.T)
    assert e["e_rel"] <= e_rel_tol, e
    bar = range_bar(S64, V64, lam, e_range_tol)
    assert e["e_range"] <= bar, (e, bar)
    return e


def rel_err(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.linalg.norm(x - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


# ---------------------------------------------------------------------------- end to end


@pytest.mark.parametrize("n,m,k,lam", [(256, 16384, 1, 1e-3), (100, 3001, 3, 1e-2), (130, 999, 2, 0.5)])
def test_fp64_path_matches_oracle(n, m, k, lam):
    S = aligned(wl.gaussian(n, m, seed=11 + n, device=dev(), dtype=torch.float64))
    V = wl.rhs(m, k, seed=12 + n, device=dev(), dtype=torch.float64)
    X, info = dfs.dfs_solve(S, V, lam, precision="fp64")
    assert info["status"] == 0 and info["precision"] == "fp64"
    assert rel_err(np64(X), solve_ref(S, V, lam)) <= 1e-10


def test_fp64_orthonormal_rows_closed_form():
    n, m, lam = 256, 16384, 1e-3
    S = wl.orthonormal_rows(n, m, seed=3, device=dev(), dtype=torch.float64)
    v = wl.rhs(m, 1, seed=4, device=dev(), dtype=torch.float64)
    X, info = dfs.dfs_solve(S, v, lam, precision="fp64")
    s, vv = np64(S), np64(v)[0]
    x_cf = (vv - s.T @ (s @ vv) / (1 + lam)) / lam
    assert rel_err(np64(X)[0], x_cf) <= 1e-10


@pytest.mark.parametrize("n,m,k,lam", [
    (1024, 65536, 1, 1e-2),   # several 128-tiles, full strips
    (257, 33333, 3, 1e-3),    # ragged n and m
    (100, 5000, 8, 1e-1),     # n below one tile, 8 RHS
    (300, 100, 1, 1e-2),      # m < n
    (1, 777, 2, 0.3),         # n = 1
    (64, 4096, 11, 1e-2),     # k > 8: two RHS groups
])
def test_fp32_path_matches_oracle(n, m, k, lam):
    S = aligned(wl.gaussian(n, m, seed=21 + n, device=dev()))
    V = wl.rhs(m, k, seed=22 + n, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="fp32")
    assert info["status"] == 0 and info["precision"] == "fp32"
    assert rel_err(np64(X), solve_ref(S, V, lam)) <= fp32_tol(S, lam)


def test_fp32_path_svd_structured_small():
    n, m = 256, 65536
    S, U, s, Vf = wl.svd_structured(n, m, seed=5, sigma_min=1e-3, device=dev())
    v = wl.rhs(m, 1, seed=6, device=dev())
    for lam in (1e-2, 1e-4):
        X, info = dfs.dfs_solve(S, v, lam, precision="fp32")
        assert rel_err(np64(X), solve_ref(S, v, lam)) <= 1e-5


def test_bf16_storage_fp32_path():
    n, m, lam = 200, 20000, 1e-2
    S = wl.gaussian(n, m, seed=7, device=dev(), dtype=torch.bfloat16)
    V = wl.rhs(m, 2, seed=8, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="fp32")
    assert rel_err(np64(X), solve_ref(S, V, lam)) <= 1e-5


@pytest.mark.parametrize("dtype,prec,n,m,k,lam", [
    (torch.bfloat16, "bf16", 1153, 12347, 3, 1e-2),   # ragged rows and columns; V rows not 16-byte aligned
    (torch.float32, "bf16", 1500, 20001, 2, 1e-2),    # FP32 S beyond 1024 rows, packed
    (torch.float32, "fp32", 2000, 9001, 1, 1e-2),     # FP32 S beyond 1024 rows, no packing
    (torch.bfloat16, "fp32", 300, 5003, 4, 1e-2),     # BF16 S, no packing, four RHS
    (torch.bfloat16, "bf16", 64, 70, 1, 0.3),         # one row block, a ragged second k-block
])
def test_row_blocked_sv_solves(dtype, prec, n, m, k, lam):
    """b = S v by 128-row blocks (BF16 S, and FP32 S beyond 1024 rows), packing the BF16 Gram
    tiles on the way for the mixed path: solves match the oracle at the path's tolerance."""
    S = aligned(wl.gaussian(n, m, seed=41 + n, device=dev(), dtype=dtype))
    V = wl.rhs(m, k, seed=42 + n, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision=prec)
    assert info["status"] == 0 and info["precision"] == prec
    if prec == "bf16":
        assert_mixed(S, V, lam, X)
    else:
        assert rel_err(np64(X), solve_ref(S, V, lam)) <= fp32_tol(S, lam)


def test_padded_leading_dimension_and_in_place():
    n, m, lam = 70, 1001, 1e-2
    big = wl.gaussian(n, 1024, seed=9, device=dev())
    S = big[:, :m]  # lds = 1024 > m
    Vb = wl.rhs(1008, 2, seed=10, device=dev())
    V = Vb[:, :m]
    ref = solve_ref(S, V, lam)
    X, _ = dfs.dfs_solve(S, V, lam, X=V, precision="fp32")  # X aliases V
    assert X.data_ptr() == V.data_ptr()
    assert rel_err(np64(V), ref) <= 1e-5


@pytest.mark.parametrize("n,m,k,lam", [
    (1024, 65536, 1, 1e-2),
    (257, 33336, 3, 1e-3),
    (100, 5000, 8, 1e-1),
    (300, 128, 2, 0.5),       # m < n (lambda large enough that v - S^T y does not cancel badly)
    (1, 1000, 1, 0.3),
])
def test_tf32_refined_path_matches_oracle(n, m, k, lam):
    S = aligned(wl.gaussian(n, m, seed=81 + n, device=dev()))
    V = wl.rhs(m, k, seed=82 + n, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="tf32")
    assert info["status"] == 0 and info["precision"] == "tf32"
    assert info["iters"] >= 1
    assert_mixed(S, V, lam, X)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_fp64_diagonal_panel_variant(prec):
    n, m, lam = 700, 50000, 1e-3
    S = wl.gaussian(n, m, seed=89, device=dev())
    V = wl.rhs(m, 2, seed=90, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision=prec, fp64_panel=True)
    assert info["status"] == 0
    if prec == "fp32":
        assert rel_err(np64(X), solve_ref(S, V, lam)) <= fp32_tol(S, lam)
    else:
        assert_mixed(S, V, lam, X)


def test_long_rows_gram():
    # long rows (1.2 MB): many k-blocks per task, the progress throttle is exercised
    n, m, lam = 300, 300000, 1e-2
    S = wl.gaussian(n, m, seed=91, device=dev())
    for prec, tol in (("tf32", 3e-3),):
        W = dfs.dfs_gram(S, lam, precision=prec)
        Wr = oracle.gram(np64(S), lam)
        lo = np.tril(np.ones((n, n), bool))
        assert np.abs(np64(W) - Wr)[lo].max() / np.abs(Wr).max() <= tol
    Sb = S.to(torch.bfloat16)
    W = dfs.dfs_gram(Sb, lam, precision="bf16")
    Wr = oracle.gram(np64(Sb), lam)
    # BF16 products are exact; the tensor core's FP32 accumulation error grows with the
    # per-task contraction length (here ~m/8 terms)
    assert np.abs(np64(W) - Wr)[lo].max() / np.abs(Wr).max() <= 1e-5 + 3e-10 * m
    V = wl.rhs(m, 1, seed=92, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="tf32")
    assert info["status"] == 0
    assert_mixed(S, V, lam, X)


def test_tf32_refined_svd_structured():
    n, m = 512, 131072
    S, U, s, Vf = wl.svd_structured(n, m, seed=83, sigma_min=1e-3, device=dev())
    v = wl.rhs(m, 2, seed=84, device=dev())
    for lam in (1e-2, 1e-4):
        X, info = dfs.dfs_solve(S, v, lam, precision="tf32")
        assert info["status"] == 0
        assert_mixed(S, v, lam, X)


def test_refined_path_in_place():
    n, m, lam = 200, 30000, 1e-3
    S = wl.gaussian(n, m, seed=87, device=dev())
    V = wl.rhs(m, 3, seed=88, device=dev())
    V0 = V.clone()
    ref = solve_ref(S, V, lam)
    X, info = dfs.dfs_solve(S, V, lam, X=V, precision="tf32")
    assert X.data_ptr() == V.data_ptr() and info["status"] == 0
    assert_mixed(S, V0, lam, V, ref=ref)


def test_bf16_storage_bf16_tensor_path():
    n, m, lam = 384, 40000, 1e-2
    S = aligned(wl.gaussian(n, m, seed=85, device=dev(), dtype=torch.bfloat16))
    V = wl.rhs(m, 2, seed=86, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16")
    assert info["status"] == 0 and info["precision"] == "bf16"
    assert_mixed(S, V, lam, X)


# ---------------------------------------------------------------------------- single steps


@pytest.mark.parametrize("dtype,prec,n,m,tol", [
    (torch.float32, "fp32", 300, 10001, 2e-5), (torch.float64, "fp64", 130, 3000, 1e-12),
    (torch.bfloat16, "fp32", 129, 4099, 2e-5),
    # TF32 keeps 10 mantissa bits (truncated): per-entry error up to ~2^-10 of sum |s_i s_j|
    (torch.float32, "tf32", 300, 10001, 3e-3), (torch.float32, "tf32", 1000, 70000, 3e-3),
    (torch.float32, "tf32", 77, 64, 3e-3), (torch.float32, "tf32", 384, 20000, 3e-3),
    (torch.float32, "tf32", 2100, 4000, 3e-3), (torch.float32, "tf32", 1153, 100, 3e-3),
    # BF16 inputs are exact and their products exact in FP32, so only the tensor core's FP32
    # accumulation errs: at most one unit of 2^-23 (truncating adds) per accumulating MMA step, of
    # which there are at most m / 16, relative to sum |s_i s_j| <= max W  ->  tol = m / 16 * 2^-23
    (torch.bfloat16, "bf16", 600, 33000, 33000 / 16 * 2.0 ** -23),
    (torch.bfloat16, "bf16", 130, 64, 2e-6), (torch.bfloat16, "bf16", 1153, 3000, 3000 / 16 * 2.0 ** -23),
    # BF16x3: s = H + L + E with |s - H| <= 2^-8 |s| and |E| <= 2^-16 |s|; dropping L L^T and E leaves
    # at most 3 * 2^-16 of sum |s_i s_j| per entry, plus the FP32 accumulation of the three products
    (torch.float32, "bf16x3", 600, 33000, 3 * 2.0 ** -16 + 3 * 33000 / 16 * 2.0 ** -23),
    (torch.float32, "bf16x3", 77, 64, 3 * 2.0 ** -16 + 1e-6),
    (torch.float32, "bf16x3", 1153, 3000, 3 * 2.0 ** -16 + 3 * 3000 / 16 * 2.0 ** -23),
    (torch.float32, "bf16x3", 2100, 4000, 3 * 2.0 ** -16 + 3 * 4000 / 16 * 2.0 ** -23)])
def test_gram_step(dtype, prec, n, m, tol):
    lam = 0.25
    S = aligned(wl.gaussian(n, m, seed=31, device=dev(), dtype=dtype))
    W = dfs.dfs_gram(S, lam, precision=prec)
    Wr = oracle.gram(np64(S), lam)
    lo = np.tril(np.ones((n, n), bool))
    err = np.abs(np64(W) - Wr)[lo].max() / np.abs(Wr).max()
    assert err <= tol
    assert np.all(np64(W)[~lo] == 0.0)  # upper triangle untouched (zeros from the caller)


@pytest.mark.parametrize("n,m", [(300, 20000), (1024, 8192), (1100, 6000)])
def test_bf16x3_gram_cross_terms(n, m):
    """Rows h_i = bf16(g + z_i / 2) share a common component g (so every Gram entry is O(m)) and
    carry a per-row low part: s_i = h_i (1 + c_i 2^-9), |c_i| < 1, so bf16(s_i) = h_i and the low
    BF16 part is ~c_i 2^-9 h_i.  Then (L H^T)[i][k] ~ c_i 2^-9 W_ik, and W needs both cross terms,
    c_i and c_k: a dropped or mis-transposed L H^T term is off by ~1e-3 W_ik, twenty times the
    tolerance, which covers the dropped L L^T (2^-18) and the FP32 accumulation."""
    g = torch.Generator(device=dev()).manual_seed(97)
    base = torch.randn(m, generator=g, device=dev())
    z = torch.randn(n, m, generator=g, device=dev())
    h = (base[None, :] + 0.5 * z).to(torch.bfloat16).float()
    c = (torch.rand(n, generator=g, device=dev()) * 1.8 - 0.9)
    S = aligned((h * (1.0 + c[:, None] * 2.0 ** -9)).contiguous())
    lam = 0.5
    W = dfs.dfs_gram(S, lam, precision="bf16x3")
    Wr = oracle.gram(np64(S), lam)
    lo = np.tril(np.ones((n, n), bool))
    err = np.abs(np64(W) - Wr)[lo].max() / np.abs(Wr).max()
    assert err <= 5e-5 + m / 1024 * 2.0 ** -23 * 16, err
    # the same matrix in plain BF16 misses the low parts: its error is of the size the test detects
    Wb = dfs.dfs_gram(S, lam, precision="bf16")
    assert np.abs(np64(Wb) - Wr)[lo].max() / np.abs(Wr).max() >= 4e-4


def _fp8_gram_model(S64, lam):
    """W of the FP8 Gram as the arithmetic defines it, computed independently of the kernels:
    r_i = the smallest power of two with max_j |s_ij| <= 448 r_i, q = e4m3(s / r_i) (round to
    nearest even; torch's float8_e4m3fn cast), W = r_i r_k sum_j q_ij q_kj + lam I, in FP64."""
    amax = np.abs(S64).max(axis=1)
    f, e = np.frexp(amax / 448.0)
    e = np.where(f == 0.5, e - 1, e)
    r = np.where(amax > 0, np.ldexp(1.0, e), 1.0)
    q = torch.from_numpy(S64 / r[:, None]).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    return (r[:, None] * (q @ q.T)) * r[None, :] + lam * np.eye(S64.shape[0]), q, r


@pytest.mark.parametrize("dtype,n,m", [(torch.float32, 300, 20000), (torch.float32, 1024, 8192),
                                       (torch.float32, 77, 100), (torch.bfloat16, 384, 12000),
                                       (torch.float32, 1500, 3000)])
def test_fp8_gram_step_matches_quantisation_model(dtype, n, m):
    S = wl.gaussian(n, m, seed=201, device=dev(), dtype=torch.float32)
    S[1] *= 1e-3          # rows of very different scale get their own power of two
    S[2] *= 37.0
    S[3] = 0.0            # a zero row: scale 1, zeros in W
    S = aligned(S.to(dtype))
    lam = 0.25
    W = dfs.dfs_gram(S, lam, precision="fp8")
    S64 = np64(S)
    Wm, q, r = _fp8_gram_model(S64, lam)
    lo = np.tril(np.ones((n, n), bool))
    # the MMAs multiply e4m3 values exactly; the tensor core's FP32 accumulation is the only
    # difference from the model: at most 2^-23 per accumulating step (K = 32), relative to
    # r_i r_k sum |q_i q_k|
    # r_i r_k sum |q_i q_k|, plus the FP32 rounding of W itself (2^-24 |W|: it holds lambda on the
    # diagonal, which dwarfs the small rows' sums there)
    ref = (r[:, None] * (np.abs(q) @ np.abs(q).T)) * r[None, :]
    err = ((np.abs(np64(W) - Wm) - 2.0 ** -24 * np.abs(Wm)) / np.maximum(ref, 1e-300))[lo]
    assert err.max() <= m / 32 * 2.0 ** -23 + 1e-6, err.max()
    assert np.all(np64(W)[~lo] == 0.0)
    # and against the exact Gram, the e4m3 rounding bound: |s - r q| <= 2^-4 |s| + 2^-10 r
    Wr = oracle.gram(S64, lam)
    bound = 2 * 2.0 ** -4 + 2.0 ** -8
    assert np.abs(np64(W) - Wr)[lo].max() <= bound * np.abs(Wr).max()


def _sr_inputs(n, m, k, seed, dtype=torch.float32):
    """O = Gaussian scores plus a per-column offset of the same size as their spread (so the
    centring matters), V Gaussian."""
    O = wl.gaussian(n, m, seed=seed, device=dev())
    g = torch.Generator(device=dev()).manual_seed(seed + 1)
    O += torch.randn(m, generator=g, device=dev())[None, :] / math.sqrt(n)
    return aligned(O.to(dtype)), wl.rhs(m, k, seed=seed + 2, device=dev())


@pytest.mark.parametrize("prec,n,m,k,lam", [("fp32", 300, 20000, 2, 1e-2), ("bf16", 1024, 65536, 1, 1e-3),
                                            ("bf16", 129, 5000, 3, 1e-2), ("tf32", 257, 33336, 2, 1e-3),
                                            ("fp8", 500, 40000, 1, 1e-2), ("bf16x3", 300, 9000, 2, 1e-4),
                                            ("bf16", 2100, 9000, 2, 1e-2)])
def test_sr_centred_solve_matches_oracle(prec, n, m, k, lam):
    """Section 4's SR scores: dfs_solve(O, ..., center=True) solves Eq. 1 for S = (O - O_bar) /
    sqrt(n), compared with the oracle's solve of its own sr_scores(O).  The plain FP32 path centres
    its FP32 Gram, which adds rounding of the size of the offset's share of O O^T (about u (1 +
    mu^2 / sigma^2) relative, mu ~ sigma here): 3x its usual bar."""
    O, V = _sr_inputs(n, m, k, seed=300 + n)
    X, info = dfs.dfs_solve(O, V, lam, precision=prec, center=True, max_iter=20)
    assert info["status"] == 0, info
    S64 = oracle.sr_scores(np64(O))
    ref = oracle.solve(S64, np64(V).T, lam).T
    tol = 3 * fp32_tol(torch.from_numpy(S64), lam) if prec == "fp32" else 1e-6
    assert rel_err(np64(X), ref) <= tol
    if prec != "fp32":
        e = oracle.errors(S64, np64(V).T, lam, np64(X).T, ref.T)
        assert e["e_range"] <= range_bar(S64, np64(V), lam), e
    # without centring the same call solves the uncentred system: a different answer
    X0, _ = dfs.dfs_solve(O, V, lam, precision=prec, max_iter=20)
    assert rel_err(np64(X0), ref) > 10 * tol


@pytest.mark.parametrize("lam", [1e-4, 1e-2])
def test_refinement_final_correction_from_bf16_tiles(lam):
    """The headline shape at small m: the second refinement step reads the packed BF16 tiles instead
    of S (one full pass over S in all), and x still meets the mixed path's 1e-6."""
    n, m = 1024, 65536
    S, U, sig, Vf = wl.svd_structured(n, m, seed=91, sigma_min=1e-3, device=dev())
    v = wl.rhs(m, 1, seed=92, device=dev())
    X, info = dfs.dfs_solve(S, v, lam, precision="bf16")
    assert info["status"] == 0 and info["iters"] == 2 and info["passes"] == 1, info
    assert_mixed(S, v, lam, X)
    # without the tiles' correction (TF32 tiles) the same solve runs two full passes
    X2, info2 = dfs.dfs_solve(S, v, lam, precision="tf32")
    assert info2["passes"] == info2["iters"] >= 1, info2


def test_refinement_step3_correction_from_bf16_tiles():
    """A batch-like problem (m/n near 70, eight right-hand sides) whose step-2 correction from the
    tiles misses the tolerance: the full pass recomputes x_2, and step 3 then ends on a correction
    from the tiles again instead of a third full pass.  x still meets the mixed path's 1e-6."""
    n, m, lam = 900, 62776, 0.0156
    S = wl.gaussian(n, m, seed=94, device=dev())
    V = wl.rhs(m, 8, seed=95, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16")
    assert info["status"] == 0 and info["passes"] < info["iters"], info
    assert_mixed(S, V, lam, X)


def test_nspace_sixteen_cta_cluster():
    """n = 5000 (n_pad 5120): eight ranks cannot hold their diagonal inverses in shared memory,
    so the n-space solves run as a 16-CTA cluster; the solve still matches the oracle."""
    n, m, lam = 5000, 12000, 1e-2
    S = wl.gaussian(n, m, seed=97, device=dev())
    V = wl.rhs(m, 1, seed=98, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16")
    assert info["status"] == 0, info
    assert_mixed(S, V, lam, X)


def test_solve_is_capturable_in_a_cuda_graph():
    """dfs_solve's launch sequence has no host round trip: captured once into a CUDA graph and
    replayed, it gives the same x as the stream-launched solve, bit for bit, and the device status."""
    n, m, lam = 512, 65536, 1e-3
    S = wl.gaussian(n, m, seed=95, device=dev())
    V = wl.rhs(m, 1, seed=96, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16")  # also sizes the workspace
    Xg = torch.empty_like(V)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    dfs.dfs_step_times()
    with torch.cuda.graph(g, stream=s):
        dfs.dfs_solve(S, V, lam, X=Xg, precision="bf16", sync=False, timing=True)
    for _ in range(2):
        Xg.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(Xg, X)
        assert dfs.dfs_sync_info()["status"] == 0
    # the step events are graph nodes: the replays recorded them
    ms, count = dfs.dfs_step_times()
    assert count == 1 and ms[0] > 0 and ms[4] >= ms[0]


def test_host_async_pipeline_matches_oracle():
    """Three queued host-memory solves with different S, V (the staging slots alternate, so the
    third reuses the first's): each X matches its oracle solve after one synchronize."""
    probs = []
    for j in range(3):
        n, m, lam = 300 + 37 * j, 20000 + 1000 * j, 1e-2
        S = wl.gaussian(n, m, seed=800 + j)
        V = wl.rhs(m, 2, seed=810 + j)
        Sh = torch.empty(S.shape, dtype=S.dtype, pin_memory=True)
        Sh.copy_(S)
        Vh = torch.empty(V.shape, dtype=V.dtype, pin_memory=True)
        Vh.copy_(V)
        Xh = torch.empty(V.shape, dtype=V.dtype, pin_memory=True)
        probs.append((Sh, Vh, lam, Xh))
    for Sh, Vh, lam, Xh in probs:
        dfs.dfs_solve_host_async(Sh, Vh, lam, Xh, precision="bf16")
    torch.cuda.synchronize()
    assert dfs.dfs_sync_info()["status"] == 0
    for Sh, Vh, lam, Xh in probs:
        assert_mixed(Sh, Vh, lam, Xh)


def _complex_inputs(n, m, k, seed, dtype=torch.float32):
    A = wl.gaussian(n, m, seed=seed, device=dev()) / math.sqrt(2)
    B = wl.gaussian(n, m, seed=seed + 1, device=dev()) / math.sqrt(2)
    vdt = torch.float64 if dtype == torch.float64 else torch.float32
    Vr = wl.rhs(m, k, seed=seed + 2, device=dev()).to(vdt)
    Vi = wl.rhs(m, k, seed=seed + 3, device=dev()).to(vdt)
    return aligned(A.to(dtype)), aligned(B.to(dtype)), Vr, Vi


@pytest.mark.parametrize("prec,n,m,k,lam,dtype", [("bf16", 512, 40000, 2, 1e-3, torch.float32),
                                                  ("fp32", 200, 9000, 1, 1e-2, torch.float32),
                                                  ("fp64", 64, 3000, 2, 1e-2, torch.float64),
                                                  ("bf16", 300, 20000, 1, 1e-2, torch.bfloat16),
                                                  ("fp8", 257, 30000, 1, 1e-2, torch.float32)])
def test_complex_solve_matches_oracle(prec, n, m, k, lam, dtype):
    """Section 4, complex SR with F = S^dagger S: dfs_solve_complex against the oracle's complex
    Algorithm 1 (Hermitian conjugates, complex128), on the stored planes."""
    A, B, Vr, Vi = _complex_inputs(n, m, k, seed=400 + n, dtype=dtype)
    Xr, Xi, info = dfs.dfs_solve_complex(A, B, Vr, Vi, lam, precision=prec)
    assert info["status"] == 0, info
    S = np64(A) + 1j * np64(B)
    ref = oracle.solve_complex(S, (np64(Vr) + 1j * np64(Vi)).T, lam).T
    X = np64(Xr) + 1j * np64(Xi)
    err = float(np.max(np.linalg.norm(X - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    if prec == "fp32":
        sv = np.linalg.svd(S, compute_uv=False)
        tol = 1e-5 * max(1.0, (sv[0] ** 2 + lam) / (sv[-1] ** 2 + lam) / 10)
    else:
        tol = 1e-12 if prec == "fp64" else 1e-6
    assert err <= tol, err


@pytest.mark.parametrize("prec,n,m,k,lam,dtype", [("bf16", 300, 20004, 6, 1e-2, torch.float32),  # groups of 4 + 2
                                                  ("bf16", 1100, 30000, 3, 1e-2, torch.float32),  # 2n > 2048: 2 + 1
                                                  ("fp32", 129, 5000, 3, 1e-2, torch.float32),
                                                  ("fp64", 100, 2000, 5, 1e-2, torch.float64),
                                                  ("bf16", 64, 64, 1, 0.3, torch.bfloat16),
                                                  ("bf16", 512, 65536, 1, 1e-3, torch.float32),  # fused first pass
                                                  ("bf16", 257, 33336, 2, 1e-3, torch.float32)])
def test_complex_solve_on_stacked_planes(prec, n, m, k, lam, dtype):
    """The planes as rows 0..n-1 and n..2n-1 of one array (used in place, no stacking copy), with
    more complex right-hand sides than one pass takes (groups), ragged n and 2n beyond the
    8-right-hand-side pass; against the oracle's complex Algorithm 1."""
    A, B, Vr, Vi = _complex_inputs(n, m, k, seed=470 + n, dtype=dtype)
    Z = torch.cat([A, B], dim=0)
    Ar, Bi = Z[:n], Z[n:]
    assert Bi.data_ptr() == Ar.data_ptr() + n * Ar.stride(0) * Ar.element_size()
    Xr, Xi, info = dfs.dfs_solve_complex(Ar, Bi, Vr, Vi, lam, precision=prec)
    assert info["status"] == 0, info
    S = np64(A) + 1j * np64(B)
    ref = oracle.solve_complex(S, (np64(Vr) + 1j * np64(Vi)).T, lam).T
    X = np64(Xr) + 1j * np64(Xi)
    err = float(np.max(np.linalg.norm(X - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    if prec == "fp32":
        sv = np.linalg.svd(S, compute_uv=False)
        tol = 1e-5 * max(1.0, (sv[0] ** 2 + lam) / (sv[-1] ** 2 + lam) / 10)
    else:
        tol = 1e-12 if prec == "fp64" else 1e-6
    assert err <= tol, err
    # the separate-plane call (stacked by the library) gives the same x bit for bit
    Xr2, Xi2, _ = dfs.dfs_solve_complex(A, B, Vr, Vi, lam, precision=prec)
    assert torch.equal(Xr, Xr2) and torch.equal(Xi, Xi2)
    if prec == "bf16" and dtype == torch.float32 and k <= 2:
        # b = S v, the tiles and the Gram of the first group as one kernel or as two: the same solve
        Xr3, Xi3, info3 = dfs.dfs_solve_complex(Ar, Bi, Vr, Vi, lam, precision=prec, two_kernel_gram=True)
        assert info3["status"] == 0, info3
        X3 = np64(Xr3) + 1j * np64(Xi3)
        assert float(np.max(np.linalg.norm(X3 - ref, axis=1) / np.linalg.norm(ref, axis=1))) <= 1e-6


def test_complex_real_part_fisher_is_the_stacked_real_solve():
    """Section 4, real-part SR (F = Re[S^dagger S]): dfs_solve on the rows of Re S followed by those
    of Im S matches the oracle's real solve of real_part_scores(S)."""
    A, B, Vr, _ = _complex_inputs(300, 20000, 1, seed=450)
    Sr = torch.cat([A, B], dim=0)
    X, info = dfs.dfs_solve(Sr, Vr, 1e-2, precision="bf16")
    assert info["status"] == 0
    Sr64 = oracle.real_part_scores(np64(A) + 1j * np64(B))
    ref = oracle.solve(Sr64, np64(Vr).T, 1e-2).T
    assert_mixed(torch.from_numpy(Sr64), Vr, 1e-2, X, ref=ref)


def test_fp8_nonfinite_row_reaches_the_cholesky():
    n, m = 200, 5000
    S = wl.gaussian(n, m, seed=203, device=dev())
    S[17, 123] = float("inf")
    V = wl.rhs(m, 1, seed=204, device=dev())
    with pytest.raises(DfsError) as e:
        dfs.dfs_solve(S, V, 1e-2, precision="fp8")
    assert e.value.status == 4  # DFS_ERR_NONFINITE


@pytest.mark.parametrize("dtype,n,m,k,lam", [(torch.float32, 1024, 65536, 1, 1e-2),
                                             (torch.float32, 257, 33336, 3, 1e-3),
                                             (torch.float32, 100, 5000, 8, 1e-1),
                                             (torch.bfloat16, 384, 40000, 2, 1e-2)])
def test_fp8_refined_path_matches_oracle(dtype, n, m, k, lam):
    S = aligned(wl.gaussian(n, m, seed=205 + n, device=dev(), dtype=dtype))
    V = wl.rhs(m, k, seed=206 + n, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="fp8", max_iter=20)
    assert info["status"] == 0 and info["precision"] == "fp8", info
    assert_mixed(S, V, lam, X)


@pytest.mark.parametrize("n,m,k,lam", [(1024, 65536, 1, 1e-4), (257, 33336, 3, 1e-3), (100, 5000, 8, 1e-1),
                                       (2100, 9000, 2, 1e-2)])
def test_bf16x3_refined_path_matches_oracle(n, m, k, lam):
    S = aligned(wl.gaussian(n, m, seed=181 + n, device=dev()))
    V = wl.rhs(m, k, seed=182 + n, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16x3")
    assert info["status"] == 0 and info["precision"] == "bf16x3", info
    assert_mixed(S, V, lam, X)


@pytest.mark.parametrize("dtype,n,tol", [(torch.float32, 300, 1e-5), (torch.float64, 200, 1e-12),
                                         (torch.float32, 1024, 1e-5), (torch.float32, 33, 1e-5),
                                         (torch.float32, 2500, 2e-5), (torch.float64, 1100, 1e-12),
                                         (torch.float32, 4096, 4e-5)])
def test_cholesky_step(dtype, n, tol):
    A = wl.gaussian(n, 3 * n, seed=41, device=dev(), dtype=torch.float64)
    Wr = (A @ A.T + 0.5 * torch.eye(n, device=dev(), dtype=torch.float64)).cpu().numpy()
    W = torch.tensor(Wr, device=dev(), dtype=dtype)
    Lr = oracle.cholesky_lower(np64(W))  # before the in-place factorisation
    L, piv = dfs.dfs_cholesky(W)
    assert piv == -1
    Lg = np.tril(np64(L))
    assert np.abs(Lg - Lr).max() / np.abs(Lr).max() <= tol
    assert (np.diag(Lg) > 0).all()


@pytest.mark.parametrize("n,bad,value,status", [(1024, 700, -1.0, 2), (1024, 1023, 0.0, 2),
                                                (600, 31, float("nan"), 4), (300, 0, -2.0, 2),
                                                (2304, 2200, -1.0, 2), (2304, 100, float("nan"), 4)])
def test_cholesky_failure_anywhere(n, bad, value, status):
    # every CTA of the factorisation must see the failure and stop (no wait runs out)
    A = wl.gaussian(n, 2 * n, seed=43, device=dev(), dtype=torch.float64)
    W = (A @ A.T + torch.eye(n, device=dev(), dtype=torch.float64)).float()
    W[bad, :bad] = 0.0
    W[bad, bad] = value
    with pytest.raises(DfsError) as e:
        dfs.dfs_cholesky(W)
    assert e.value.status == status
    assert f"pivot {bad}" in str(e.value)
    # the handle stays usable afterwards
    W2 = (A @ A.T + torch.eye(n, device=dev(), dtype=torch.float64)).float()
    L, piv = dfs.dfs_cholesky(W2)
    assert piv == -1 and torch.isfinite(L).all()


def test_cholesky_reports_failed_pivot():
    n = 100
    d = torch.ones(n, dtype=torch.float32)
    d[70] = -1.0
    W = torch.diag(d).to(dev())
    with pytest.raises(DfsError) as e:
        dfs.dfs_cholesky(W)
    assert e.value.status == 2
    assert "pivot 70" in str(e.value)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-12)])
@pytest.mark.parametrize("trans", [False, True])
def test_trsm_step(dtype, tol, trans):
    n, k = 333, 5
    g = torch.Generator().manual_seed(51)
    Lr = torch.tril(torch.randn(n, n, generator=g, dtype=torch.float64)) / math.sqrt(n) + 2 * torch.eye(n, dtype=torch.float64)
    B = torch.randn(n, k, generator=g, dtype=torch.float64)
    L = Lr.to(dev(), dtype)
    Bd = B.to(dev(), dtype).contiguous()
    out = dfs.dfs_trsm(L, Bd, trans=trans)
    Ln = np64(L)
    ref = oracle.back_substitution_transposed(Ln, B.numpy()) if trans else oracle.forward_substitution(Ln, B.numpy())
    assert np.abs(np64(out) - ref).max() / np.abs(ref).max() <= tol


@pytest.mark.parametrize("dtype,n,extra,k", [
    (torch.bfloat16, 2100, 1234, 3),   # ragged rows, odd m (X rows not 16-byte aligned), 3 of 4 RHS
    (torch.float32, 2049, 0, 2),       # one row past the threshold, whole 4096-column chunks
    (torch.float32, 2056, 4095, 1),    # a 4095-column last chunk
])
def test_fisher_pass_two_kernel_form(dtype, n, extra, k):
    """n > 2048 with a 4096-column chunk per SM: the pass runs as X = (V - S^T Y)/lambda by column
    chunks, then R = S U - lambda Y by 8-row blocks.  The reference goes by column blocks b, since
    u_b depends only on b's columns: X_b = (v_b - S_b^T y)/lambda and R = sum_b r_b + (B - 1) lambda y
    with r_b the oracle's n-space residual of block b."""
    sms = torch.cuda.get_device_properties(dev()).multi_processor_count
    m, lam = 4096 * sms + extra, 1e-2
    S = aligned(wl.gaussian(n, m, seed=63, device=dev(), dtype=dtype))
    V = wl.rhs(m, k, seed=64, device=dev())
    Y = torch.randn(n, k, device=dev(), dtype=torch.float64) * (0.3 / math.sqrt(n / 150))
    X, R = dfs.dfs_fisher_pass(S, V, lam, Y)
    y = np64(Y)
    x_ref = np.empty((k, m))
    r_ref = np.zeros((n, k))
    blocks = 0
    for c0 in range(0, m, 65536):
        c1 = min(m, c0 + 65536)
        s, v = np64(S[:, c0:c1]), np64(V[:, c0:c1]).T
        x_ref[:, c0:c1] = ((v - s.T @ y) / lam).T
        r_ref += oracle.residual_n_space(s, v, y, lam)
        blocks += 1
    r_ref += (blocks - 1) * lam * y
    assert rel_err(np64(X), x_ref) <= 2e-6
    assert np.abs(np64(R) - r_ref).max() / np.abs(r_ref).max() <= 1e-5


@pytest.mark.parametrize("dtype,n,m,k", [
    (torch.float32, 150, 12345, 3), (torch.bfloat16, 150, 12345, 3), (torch.float64, 150, 12345, 3),
    (torch.float32, 1024, 40000, 8),   # RHS beyond the cluster form's 4 per pass: classic kernel
    (torch.float32, 1024, 40001, 1),   # clusters of 2 CTAs x 512 rows, ragged last strip
    (torch.float32, 1100, 20003, 2),   # clusters of 3 (column split 22/21/21)
    (torch.float32, 2500, 9001, 4),    # clusters of 5
    (torch.float32, 4096, 5000, 1),    # clusters of 8 (the largest)
    (torch.float32, 4097, 3001, 1),    # beyond the cluster form: re-read kernel
    (torch.float32, 77, 100, 3),       # fewer strips than clusters
    (torch.bfloat16, 700, 70001, 1),
])
def test_fisher_pass_step(dtype, n, m, k):
    lam = 1e-2
    S = aligned(wl.gaussian(n, m, seed=61, device=dev(), dtype=dtype))
    vdt = torch.float64 if dtype == torch.float64 else torch.float32
    V = wl.rhs(m, k, seed=62, device=dev(), dtype=vdt)
    Y = torch.randn(n, k, device=dev(), dtype=torch.float64) * (0.3 / math.sqrt(n / 150))
    X, R = dfs.dfs_fisher_pass(S, V, lam, Y)
    s, v, y = np64(S), np64(V).T, np64(Y)
    u = v - s.T @ y
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert rel_err(np64(X), (u / lam).T) <= tol
    r_ref = oracle.residual_n_space(s, v, y, lam)
    assert np.abs(np64(R) - r_ref).max() / np.abs(r_ref).max() <= tol * 5
    # Y = None: R = S v (the right-hand side of the n-space system), X = v / lam
    X0, R0 = dfs.dfs_fisher_pass(S, V, lam, None)
    assert rel_err(np64(R0).T, (s @ v).T) <= tol
    assert rel_err(np64(X0), (v / lam).T) <= (1e-15 if dtype == torch.float64 else 1e-7)


# ---------------------------------------------------------------------------- arguments


def test_invalid_arguments_rejected():
    S = torch.zeros(8, 64, device=dev())
    V = torch.zeros(1, 64, device=dev())
    for lam in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(DfsError) as e:
            dfs.dfs_solve(S, V, lam)
        assert e.value.status == 1
    S2 = torch.zeros(8, 66, device=dev())[:, :63]  # lds = 66 floats: not a multiple of 16 bytes
    with pytest.raises(DfsError) as e:
        dfs.dfs_solve(S2, torch.zeros(1, 63, device=dev()), 1.0)
    assert e.value.status == 1
    with pytest.raises(DfsError) as e:
        dfs.dfs_solve(S.double(), V.double(), 1.0, precision="fp32")
    assert e.value.status == 1


def test_zero_score_matrix_gives_v_over_lambda():
    S = torch.zeros(40, 1000, device=dev())
    V = wl.rhs(1000, 1, seed=71, device=dev())
    X, info = dfs.dfs_solve(S, V, 0.125, precision="fp32")
    assert torch.equal(X, V / 0.125)


# ---------------------------------------------------------------------------- full size


def test_full_size_headline_workload_matches_oracle():
    """The benchmark's workload (n=1024, m=2^20, SVD-structured FP32 S, lambda=1e-4), in the launch
    configuration bench.py times: the BF16 mixed path and the plain FP32 path against one full
    FP64 oracle solve on the host (the metric's bar: rel. error <= 1e-6 mixed, <= 1e-5 FP32)."""
    n, m, lam = 1024, 1 << 20, 1e-4
    S, U, s, V = wl.svd_structured(n, m, seed=231017556 + 1, sigma_min=1e-3, device=dev(),
                                   dtype=torch.float32, factor_dtype=torch.float64)
    del U, V
    v = wl.rhs(m, 1, seed=231017556 + 8, device=dev())
    Xm, info = dfs.dfs_solve(S, v, lam, precision="bf16")
    assert info["status"] == 0 and info["iters"] >= 1
    Xf, info_f = dfs.dfs_solve(S, v, lam, precision="fp32")
    assert info_f["status"] == 0
    S64 = np64(S)
    v64 = np64(v)[0]
    del S
    torch.cuda.empty_cache()
    x_ref = oracle.solve(S64, v64, lam)
    em = oracle.errors(S64, v64, lam, np64(Xm)[0], x_ref)
    ef = oracle.errors(S64, v64, lam, np64(Xf)[0], x_ref)
    assert em["e_rel"] <= 1e-6, em
    assert ef["e_rel"] <= 1e-5, ef
    # the error inside the row space of S, where Algorithm 1's S^T y part lives (sigma_max^2 / lam
    # is about 10 here, so x's FP32 storage floor, ~3e-6, is not reached)
    assert em["e_range"] <= 1e-6, em
    assert ef["e_range"] <= 1e-5, ef


# ---------------------------------------------------------------------------- batched


def test_solve_batched_ragged():
    """Independent problems of uneven (n, m, lambda) in one call (the batching workload's shape mix,
    at sizes the oracle finishes quickly): each matches its own oracle solve; per-problem status."""
    shapes = wl.ragged_batch_shapes(6, seed=4242, n_lo=64, n_hi=400, m_lo=2e3, m_hi=6e4, lam_lo=1e-3, lam_hi=1e-1)
    probs, refs = [], []
    for j, (n, m, lam) in enumerate(shapes):
        m = (m + 3) // 4 * 4
        S = wl.gaussian(n, m, seed=500 + j, device=dev())
        V = wl.rhs(m, 2, seed=600 + j, device=dev())
        probs.append((S, V, lam))
        refs.append(solve_ref(S, V, lam))
    outs, status = dfs.dfs_solve_batched(probs, precision="bf16")
    assert status == [0] * len(probs)
    for (S, V, lam), X, ref in zip(probs, outs, refs):
        assert rel_err(np64(X), ref) <= 1e-6


def _ragged_problems(count, seed, k=2, n_hi=400, m_hi=6e4):
    shapes = wl.ragged_batch_shapes(count, seed=seed, n_lo=64, n_hi=n_hi, m_lo=2e3, m_hi=m_hi, lam_lo=1e-3,
                                    lam_hi=1e-1)
    probs = []
    for j, (n, m, lam) in enumerate(shapes):
        m = (m + 3) // 4 * 4
        probs.append((wl.gaussian(n, m, seed=seed + 10 + j, device=dev()), wl.rhs(m, k, seed=seed + 50 + j, device=dev()),
                      lam))
    return probs


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_solve_batched_lanes(prec):
    """Nine uneven problems: more than the concurrent lanes, so lanes run several problems each,
    longest first; every problem matches its own oracle solve."""
    probs = _ragged_problems(9, seed=7000)
    outs, status = dfs.dfs_solve_batched(probs, precision=prec)
    assert status == [0] * len(probs)
    for (S, V, lam), X in zip(probs, outs):
        if prec == "fp32":
            assert rel_err(np64(X), solve_ref(S, V, lam)) <= fp32_tol(S, lam)
        else:
            assert_mixed(S, V, lam, X)


@pytest.mark.parametrize("lanes,share", [(1, 1), (4, 2), (8, 4), (16, 8)])
def test_solve_batched_lane_counts_and_shares(lanes, share):
    """The batch's concurrency knobs change only how problems share the GPU: one lane (a plain loop
    on the caller's stream), and lanes whose kernels size their grids for a fraction of the SMs,
    each give every problem its oracle solution."""
    probs = _ragged_problems(9, seed=7050)
    h = dfs.Handle()
    try:
        dfs.dfs_set_batch_lanes(lanes, share, handle=h)
        assert dfs.dfs_get_batch_lanes(handle=h) == (lanes, share)
        outs, status = dfs.dfs_solve_batched(probs, precision="bf16", handle=h)
        assert status == [0] * len(probs)
        for (S, V, lam), X in zip(probs, outs):
            assert_mixed(S, V, lam, X)
    finally:
        h.close()


def test_batch_lanes_out_of_range_are_rejected():
    h = dfs.Handle()
    try:
        for lanes, share in [(0, 1), (17, 1), (8, 0), (8, 17)]:
            with pytest.raises(DfsError):
                dfs.dfs_set_batch_lanes(lanes, share, handle=h)
        assert dfs.dfs_get_batch_lanes(handle=h) == (8, 1)
    finally:
        h.close()


def test_autotune_batched_picks_a_candidate_and_caches_it(tmp_path):
    """The tuner times the batch under its candidates, sets the fastest, and appends it to the cache;
    a second handle reads the choice back without timing; the tuned batch solves correctly."""
    probs = [(S, V, lam, torch.empty_like(V)) for S, V, lam in _ragged_problems(12, seed=7060)]
    cache = tmp_path / "batch_tune.jsonl"
    h1, h2 = dfs.Handle(), dfs.Handle()
    try:
        r1 = dfs.dfs_autotune_batched(probs, precision="bf16", handle=h1, cache_path=str(cache))
        assert r1["ms"] > 0.0
        assert (r1["lanes"], r1["share"]) in {(8, 1), (8, 2), (8, 4), (8, 8), (16, 4), (16, 8), (4, 1), (4, 2)}
        assert dfs.dfs_get_batch_lanes(handle=h1) == (r1["lanes"], r1["share"])
        lines = cache.read_text().splitlines()
        assert len(lines) == 1
        rec = json.loads(lines[0])
        assert rec["gpu"] == torch.cuda.get_device_name(0)
        assert (rec["lanes"], rec["share"]) == (r1["lanes"], r1["share"])
        r2 = dfs.dfs_autotune_batched(probs, precision="bf16", handle=h2, cache_path=str(cache))
        assert r2 == {"lanes": r1["lanes"], "share": r1["share"], "ms": 0.0}
        assert len(cache.read_text().splitlines()) == 1
        # another batch has another key: timed and appended
        r3 = dfs.dfs_autotune_batched(probs[:5], precision="bf16", handle=h2, cache_path=str(cache))
        assert r3["ms"] > 0.0 and len(cache.read_text().splitlines()) == 2
        outs, status = dfs.dfs_solve_batched([p[:3] for p in probs], precision="bf16", handle=h1)
        assert status == [0] * len(probs)
        for (S, V, lam, _), X in zip(probs, outs):
            assert_mixed(S, V, lam, X)
    finally:
        h1.close()
        h2.close()


def test_solve_batched_failure_stays_in_its_problem():
    """A NaN in one problem's S fails that problem alone (its lane's status is reset before the
    next problem); the call reports it by index and every other problem is still solved."""
    probs = _ragged_problems(7, seed=7100)
    bad = 3
    probs[bad][0][5, 17] = float("nan")
    with pytest.raises(DfsError) as e:
        dfs.dfs_solve_batched(probs, precision="bf16")
    assert e.value.status == 4 and f"problem {bad}" in str(e.value)
    assert [st for j, st in enumerate(e.value.statuses) if j != bad] == [0] * (len(probs) - 1)
    outs = e.value.outs
    for j, ((S, V, lam), X) in enumerate(zip(probs, outs)):
        if j != bad:
            assert_mixed(S, V, lam, X)


def test_solve_batched_planned_is_capturable():
    """dfs_plan_batched creates the lanes and sizes their workspaces, so the batched solve then
    allocates nothing and captures into a CUDA graph.  Each replay gives the stream-launched
    results bit for bit, and leaves the per-problem statuses on the device."""
    shapes = [(300, 20000, 2, 1e-2), (129, 50001, 1, 1e-3), (513, 9000, 3, 1e-1)]
    probs = [(aligned(wl.gaussian(n, m, seed=300 + j, device=dev())), wl.rhs(m, k, seed=310 + j, device=dev()), lam)
             for j, (n, m, k, lam) in enumerate(shapes)]
    h = dfs.Handle()
    assert dfs.dfs_plan_batched(probs, precision="bf16", handle=h) > 0
    outs, status = dfs.dfs_solve_batched(probs, precision="bf16", handle=h)
    assert status == [0, 0, 0]
    Xg = [torch.empty_like(V) for _, V, _ in probs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        dfs.dfs_solve_batched([(S, V, lam, X) for (S, V, lam), X in zip(probs, Xg)], precision="bf16", handle=h,
                              sync=False)
    for _ in range(2):
        for X in Xg:
            X.zero_()
        g.replay()
        torch.cuda.synchronize()
        for X, ref in zip(Xg, outs):
            assert torch.equal(X, ref)
        assert dfs.dfs_batched_status(3, handle=h) == [0, 0, 0]
    assert_mixed(probs[1][0], probs[1][1], probs[1][2], Xg[1])


# ---------------------------------------------------------------------------- full-size configurations


def _residual_fp64(S, X, V, lam, chunk=1 << 18):
    """||S^T S x + lam x - v|| / ||v|| per RHS, in FP64 with torch (column chunks of S), as a check
    independent of the CUDA path: for SPD A = S^T S + lam I, e_rel <= cond(A) res."""
    n, m = S.shape
    k = V.shape[0]
    Sx = torch.zeros((n, k), device=S.device, dtype=torch.float64)
    for c0 in range(0, m, chunk):
        Sx += S[:, c0:c0 + chunk].double() @ X[:, c0:c0 + chunk].double().T
    num = torch.zeros(k, device=S.device, dtype=torch.float64)
    for c0 in range(0, m, chunk):
        r = (S[:, c0:c0 + chunk].double().T @ Sx).T + lam * X[:, c0:c0 + chunk].double() - V[:, c0:c0 + chunk].double()
        num += (r * r).sum(dim=1)
    return (num.sqrt() / V.double().norm(dim=1)).cpu().numpy()


def _sigma_max_sq(S, iters=30, chunk=1 << 18):
    """Rayleigh-quotient estimate of ||S||_2^2 (a lower bound) by power iteration on S S^T, FP32
    products over column chunks of S, with torch."""
    n, m = S.shape
    g = torch.Generator(device=S.device).manual_seed(7)
    u = torch.randn(n, device=S.device, dtype=torch.float32, generator=g)
    u /= u.norm()
    est = 0.0
    for _ in range(iters):
        w = torch.zeros(n, device=S.device, dtype=torch.float32)
        for c0 in range(0, m, chunk):
            Sc = S[:, c0:c0 + chunk].float()
            w += Sc @ (Sc.T @ u)
        est = float(torch.dot(u, w))
        u = w / w.norm()
    return est


@pytest.mark.slow
def test_full_size_n4096_m2p22_k4_mixed():
    """The precision configuration at its full size: n=4096, m=2^22 (64 GB of FP32 S), k=4,
    lambda=1e-4, BF16 Gram with refinement, S with log-spaced singular values 1/sqrt(n) .. 1e-4/sqrt(n)
    (low-memory generator: its SVD factors in FP32).  cond(A) = (1/n + lambda)/lambda ~ 3.4, so the
    FP64 residual bounds the relative error: e_rel <= cond(A) res <= 1e-6 asks res <= 1e-6/cond(A)."""
    n, m, k, lam = 4096, 1 << 22, 4, 1e-4
    S = wl.svd_structured_lowmem(n, m, seed=231017556 + 3, sigma_min=1e-4, device=dev())
    V = wl.rhs(m, k, seed=231017556 + 10, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16")
    assert info["status"] == 0 and info["iters"] >= 1, info
    assert info["rel_correction"] <= 1e-6, info
    cond = (1.0 / n + lam) / lam * 1.01  # 1 % for the FP32 orthogonality of the generated factors
    res = _residual_fp64(S, X, V, lam)
    assert res.max() <= 1e-6 / cond, res
    del S, V, X
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_full_size_n8192_m2p22_heavy_tailed_bf16():
    """The stress configuration: n=8192, m=2^22, BF16 S (64 GB) with Student-t entries and log-normal
    column scales, lambda=1e-5 (near-singular W), k=1.

    x is returned in FP32; its rounding delta_x alone (|delta_x_i| <= 2^-24 |x_i|) adds up to
    ||A delta_x|| <= ||A||_2 2^-24 ||x|| to the residual of Eq. 1, ||A||_2 = ||S||_2^2 + lambda, which
    here (||S||_2^2 ~ 1e4, ||x|| ~ ||v||/lambda) is far above 1.  So the check is that the FP64
    residual stays within twice that storage floor (the factor 2 covers the power-iteration estimate
    of ||S||_2^2 from below), i.e. that the solver's own error is below it; an unrefined
    BF16-factor answer misses this floor by orders of magnitude."""
    n, m, lam = 8192, 1 << 22, 1e-5
    S = wl.heavy_tailed(n, m, seed=231017556 + 5, device=dev(), dtype=torch.bfloat16)
    V = wl.rhs(m, 1, seed=231017556 + 12, device=dev())
    X, info = dfs.dfs_solve(S, V, lam, precision="bf16", max_iter=12, allow_not_converged=True)
    assert info["status"] in (0, 3), info  # converged, or stopped at the rounding floor
    assert torch.isfinite(X).all()
    res = _residual_fp64(S, X, V, lam)
    s2 = _sigma_max_sq(S)
    floor = 2.0 ** -24 * (s2 + lam) * (X.double().norm(dim=1) / V.double().norm(dim=1)).cpu().numpy()
    assert (res <= 2.0 * floor).all(), (res, floor, s2)
    del S, V, X
    torch.cuda.empty_cache()
