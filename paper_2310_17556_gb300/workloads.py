"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random-number generation and matrix construction only: none
of the solve's arithmetic.  Both the CUDA path's callers (tests, bench) and the
FP64 oracle's callers take their inputs from here, so the two sides see the
same bytes.

The paper (arXiv 2310.17556, Section 2) measures on score matrices S of shape
n x m with m >> n (n ~ 10^3 samples, m ~ 10^5..10^6 parameters) and names no
dataset, so every input is synthetic:

* ``gaussian``: S_ij ~ N(0, 1)/sqrt(n) (the 1/sqrt(n) scaling of Section 2's
  definition of S), v ~ N(0, 1).
* ``orthonormal_rows``: S = Q^T with Q the thin-QR factor of an m x n Gaussian,
  so S S^T = I and Algorithm 1 has a closed form.
* ``svd_structured``: S = U diag(sigma) V^T / sqrt(n), U Haar-orthogonal n x n,
  V m x n orthonormal (thin QR of a Gaussian), sigma log-spaced from 1 down to
  sigma_min; the factors are returned so Appendix C's closed form can be used.
* ``heavy_tailed``: Student-t (nu = 3) entries, each column scaled by a
  log-normal(0, 1) factor, divided by sqrt(n).
* ``ragged_batch``: many independent problems with n ~ U{64..1024},
  m ~ log-uniform [1e4, 5e5], lambda ~ log-uniform [1e-5, 1e-1].

Layout: S is n x m row-major (each sample row contiguous along m); the k
right-hand sides are stored as k rows of length m (a k x m row-major array),
so each RHS is contiguous.
"""

from __future__ import annotations

import math

import torch

SEED_BASE = 231017556


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _randn(shape, g, device, dtype=torch.float64):
    return torch.randn(shape, generator=g, device=device, dtype=dtype)


def rhs(m: int, k: int, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """k right-hand sides v ~ N(0, 1), as a k x m row-major tensor."""
    g = _gen(seed ^ 0x5EED, device)
    return _randn((k, m), g, device, torch.float32 if dtype != torch.float64 else torch.float64).to(dtype)


def gaussian(n: int, m: int, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """S_ij ~ N(0, 1)/sqrt(n), n x m row-major, rounded once to ``dtype``."""
    g = _gen(seed, device)
    base = torch.float64 if dtype == torch.float64 else torch.float32
    S = _randn((n, m), g, device, base)
    S.mul_(1.0 / math.sqrt(n))
    return S.to(dtype)


def _thin_q(G: torch.Tensor) -> torch.Tensor:
    """Q factor (positive diagonal R) of the thin QR of a tall m x n matrix G (m >= n).

    Cholesky-QR applied twice: R = chol(G^T G)^T, Q = G R^{-1}, repeated once on Q.  The n x n
    factorisations run on the host in FP64 (numpy); the tall products stay on G's device, so
    no device linear-algebra library is needed.  For a Gaussian G with m >> n, cond(G) ~ 1 and
    two rounds give orthonormality to FP64 rounding.
    """
    import numpy as np

    Q = G
    for _ in range(2):
        C = (Q.T @ Q).cpu().numpy()
        L = np.linalg.cholesky(C)
        Linv_t = np.linalg.inv(L).T  # R^{-1} with R = L^T
        Q = Q @ torch.from_numpy(np.ascontiguousarray(Linv_t)).to(device=Q.device, dtype=Q.dtype)
    return Q


def orthonormal_rows(n: int, m: int, seed: int, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """S = Q^T with Q (m x n) the thin-QR factor of an m x n Gaussian: S S^T = I."""
    assert n <= m
    g = _gen(seed, device)
    G = _randn((m, n), g, device, torch.float64)
    Q = _thin_q(G)
    return Q.T.contiguous().to(dtype)


def _haar_orthogonal(n: int, g, device) -> torch.Tensor:
    """Haar-distributed n x n orthogonal matrix: QR of a Gaussian with R's diagonal signs folded
    into Q (Mezzadri 2007), computed on the host in FP64."""
    import numpy as np

    G = _randn((n, n), g, device, torch.float64).cpu().numpy()
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return torch.from_numpy(Q * d[None, :]).to(device)


def svd_structured(n: int, m: int, seed: int, sigma_min: float = 1e-3, device="cpu",
                   dtype=torch.float32, factor_dtype=torch.float64):
    """S = U diag(sigma) V^T / sqrt(n) with known factors.

    Returns (S, U, s, V) where s = sigma / sqrt(n) are the singular values of the
    unrounded product, U is n x n, V is m x n (both in ``factor_dtype``).  S is
    rounded once to ``dtype`` after the product is formed in ``factor_dtype``.
    """
    assert n <= m
    g = _gen(seed, device)
    U = _haar_orthogonal(n, g, device).to(factor_dtype)
    G = _randn((m, n), g, device, torch.float64)
    V = _thin_q(G).to(factor_dtype)
    del G
    sigma = torch.logspace(0.0, math.log10(sigma_min), n, dtype=torch.float64, device=device)
    s = (sigma / math.sqrt(n)).to(factor_dtype)
    S = (U * s[None, :]) @ V.T
    return S.to(dtype), U, s, V


def svd_structured_lowmem(n: int, m: int, seed: int, sigma_min: float = 1e-4, device="cpu",
                          dtype=torch.float32, chunk: int = 1 << 18) -> torch.Tensor:
    """S = U diag(sigma) V^T / sqrt(n) with the spectrum of ``svd_structured`` (Haar U, sigma
    log-spaced 1 .. sigma_min), for sizes where an m x n FP64 factor does not fit or an FP64 QR
    would take minutes: V comes from CholeskyQR2 of an FP32 Gaussian m x n block (FP32 Gram
    matrices, formed column chunk by column chunk; Cholesky and inverse in FP64 on the host), so it
    is orthonormal to FP32 accuracy; the Gaussian block is well conditioned (its condition number
    tends to (1 + sqrt(n/m)) / (1 - sqrt(n/m))), which is what CholeskyQR needs.  Only S is returned;
    it is a different draw from ``svd_structured`` with the same seed."""
    import numpy as np

    assert n <= m
    g = _gen(seed, device)
    U = _haar_orthogonal(n, g, device)  # FP64, n x n
    V = torch.empty((m, n), device=device, dtype=torch.float32)
    for c0 in range(0, m, chunk):
        V[c0:c0 + chunk] = _randn((min(chunk, m - c0), n), g, device, torch.float32)
    for _ in range(2):
        C = torch.zeros((n, n), device=device, dtype=torch.float32)
        for c0 in range(0, m, chunk):
            C.addmm_(V[c0:c0 + chunk].T, V[c0:c0 + chunk])
        L = np.linalg.cholesky(C.double().cpu().numpy())
        Rinv = torch.from_numpy(np.ascontiguousarray(np.linalg.inv(L).T)).to(device=device, dtype=torch.float32)
        for c0 in range(0, m, chunk):
            V[c0:c0 + chunk] = V[c0:c0 + chunk] @ Rinv
    sigma = torch.logspace(0.0, math.log10(sigma_min), n, dtype=torch.float64, device=device)
    B = (U * (sigma / math.sqrt(n))[None, :]).float()  # U diag(sigma) / sqrt(n), n x n
    S = torch.empty((n, m), device=device, dtype=dtype)
    for c0 in range(0, m, chunk):
        S[:, c0:c0 + chunk] = (B @ V[c0:c0 + chunk].T).to(dtype)
    del V
    return S


def heavy_tailed(n: int, m: int, seed: int, device="cpu", dtype=torch.bfloat16) -> torch.Tensor:
    """Student-t (nu = 3) entries times a per-column log-normal(0, 1) factor, / sqrt(n).

    t = z / sqrt(chi2_3 / 3) with chi2_3 the sum of three squared standard normals.
    Built in row chunks so the FP32 temporaries stay small next to S itself.
    """
    g = _gen(seed, device)
    col = torch.exp(_randn((m,), g, device, torch.float32))
    S = torch.empty((n, m), device=device, dtype=dtype)
    rows = max(1, (1 << 26) // max(m, 1))
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        z = _randn((r1 - r0, m), g, device, torch.float32)
        c = torch.zeros_like(z)
        for _ in range(3):
            c.add_(_randn((r1 - r0, m), g, device, torch.float32).square_())
        z.div_(torch.sqrt(c / 3.0)).mul_(col[None, :]).mul_(1.0 / math.sqrt(n))
        S[r0:r1] = z.to(dtype)
        del z, c
    return S


def log_uniform(lo: float, hi: float, g: torch.Generator, size: int) -> torch.Tensor:
    u = torch.rand((size,), generator=g, dtype=torch.float64)
    return torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def ragged_batch_shapes(count: int, seed: int, n_lo=64, n_hi=1024, m_lo=1e4, m_hi=5e5,
                        lam_lo=1e-5, lam_hi=1e-1):
    """Shapes of a ragged batch: list of (n, m, lambda), drawn on the host."""
    g = _gen(seed, "cpu")
    ns = torch.randint(n_lo, n_hi + 1, (count,), generator=g)
    ms = log_uniform(m_lo, m_hi, g, count).round().long()
    lams = log_uniform(lam_lo, lam_hi, g, count)
    return [(int(a), int(b), float(c)) for a, b, c in zip(ns, ms, lams)]
