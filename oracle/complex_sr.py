"""Complex score matrices for stochastic reconfiguration (Section 4 of arXiv 2310.17556).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path.

Section 4: when the wave function is complex, S is complex and every transpose of Eq. 1 and of
Algorithm 1 becomes the Hermitian conjugate.  Two Fisher matrices are in use:

* the full complex one, F = S^dagger S: solve (S^dagger S + lambda I) x = v (``solve_complex``,
  Algorithm 1 with conjugate transposes, in complex128);
* its real part, F = Re[S^dagger S]: the same real algorithm applied to S replaced by the
  concatenation of Re S and Im S along the sample (n) dimension (``real_part_scores``).
"""

from __future__ import annotations

import numpy as np

__all__ = ["solve_complex", "real_part_scores"]


def _as_c128(a) -> np.ndarray:
    return np.asarray(a, dtype=np.complex128)


def _cholesky_lower_hermitian(W: np.ndarray) -> np.ndarray:
    """W = L L^dagger with L lower triangular and a real positive diagonal; column recurrence:
        L[j, j] = sqrt(W[j, j] - sum_{p<j} |L[j, p]|^2)
        L[i, j] = (W[i, j] - sum_{p<j} L[i, p] conj(L[j, p])) / L[j, j],  i > j."""
    n = W.shape[0]
    L = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        Lj = L[j, :j]
        d = (W[j, j] - np.vdot(Lj, Lj)).real
        if not (d > 0.0):
            raise ValueError(f"Cholesky pivot {j} is not positive ({d!r})")
        ljj = np.sqrt(d)
        L[j, j] = ljj
        if j + 1 < n:
            L[j + 1:, j] = (W[j + 1:, j] - L[j + 1:, :j] @ np.conj(Lj)) / ljj
    return L


def solve_complex(S, V, lam: float) -> np.ndarray:
    """x = (S^dagger S + lambda I)^{-1} v by Algorithm 1 with Hermitian conjugates (complex128).

    Steps, right to left as in Section 2: W = S S^dagger + lambda I~, L = Chol(W), b = S v,
    a = L^{-1} b (forward substitution), y = L^{-dagger} a (backward substitution with the
    conjugate transpose), x = (v - S^dagger y) / lambda.  S is n x m, V is (m,) or (m, k).
    """
    lam = float(lam)
    if not (lam > 0.0) or not np.isfinite(lam):
        raise ValueError("lambda must be a finite positive number")
    S = _as_c128(S)
    V = _as_c128(V)
    vec = V.ndim == 1
    V2 = V[:, None] if vec else V
    n = S.shape[0]
    W = S @ np.conj(S.T)
    W[np.arange(n), np.arange(n)] += lam
    L = _cholesky_lower_hermitian(W)
    b = S @ V2
    a = np.zeros_like(b)
    for i in range(n):
        a[i] = (b[i] - L[i, :i] @ a[:i]) / L[i, i]
    y = np.zeros_like(a)
    for i in range(n - 1, -1, -1):
        y[i] = (a[i] - np.conj(L[i + 1:, i]) @ y[i + 1:]) / L[i, i]
    x = (V2 - np.conj(S.T) @ y) / lam
    return x[:, 0] if vec else x


def real_part_scores(S) -> np.ndarray:
    """Section 4, real-part SR: S <- Concat[Re S, Im S] along the sample dimension (2n x m), so
    that S^T S = Re[S^dagger S]."""
    S = _as_c128(S)
    return np.concatenate([S.real, S.imag], axis=0)
