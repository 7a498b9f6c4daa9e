"""FP64 CPU oracle for the Cholesky solve of the damped Fisher system.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path
(``paper_2310_17556_gb300``) and imports nothing from it.

What it computes (Chen, Xie, Wang, "Efficient Numerical Algorithm for
Large-Scale Damped Natural Gradient Descent", arXiv 2310.17556):

* Eq. 1: find x with (S^T S + lambda I) x = v, S an n x m matrix, x and v
  m-vectors, lambda > 0 (Appendix A, Prop. 1: any lambda > 0 makes the
  system uniquely solvable).
* Algorithm 1, steps 1-4: W = S S^T + lambda I~ (n x n), L = Chol(W) lower
  triangular, Q = L^{-1} S, x = (v - Q^T Q v) / lambda.
* Section 2 (text after Algorithm 1): Q is never formed; Q^T Q v is
  evaluated right to left as S^T L^{-T} L^{-1} S v with two triangular
  solves.

Several right-hand sides are handled column by column: V has shape (m, k)
and the solution X has the same shape (the paper states one RHS; the
solution of each column is unique, so k columns are k independent solves).

Every step is written out in FP64 in the paper's order.  Library primitives
used as steps: the matrix product (numpy ``@``) and ``sqrt``.  The Cholesky
factorisation and the two substitutions are written out as the textbook
column/row recurrences, so that they can be checked by eye.

Parity status: every function here is pinned by tests that do not go through
this module (dense LAPACK solve of Eq. 1, exact rational Gauss-Jordan,
closed forms of Appendix B and C, orthonormal-row closed form, n = 1
Sherman-Morrison form, textbook Cholesky example).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "NotPositiveDefinite",
    "gram",
    "cholesky_lower",
    "forward_substitution",
    "back_substitution_transposed",
    "solve",
    "solve_steps",
    "apply_operator",
    "residual_n_space",
    "solve_batched",
    "sr_scores",
    "errors",
]


class NotPositiveDefinite(ValueError):
    """Raised when a Cholesky pivot is not strictly positive.

    Algorithm 1's Cholesky assumes W is symmetric positive definite (true for any
    lambda > 0 in exact arithmetic, Appendix A).  A non-positive pivot in
    floating point is reported, never repaired.
    """

    def __init__(self, pivot: int, value: float):
        super().__init__(f"Cholesky pivot {pivot} is not positive ({value!r})")
        self.pivot = pivot
        self.value = value


def _as_f64(a) -> np.ndarray:
    """Exactly widen a stored array (f16/bf16-as-f32/f32/f64) to FP64."""
    return np.asarray(a, dtype=np.float64)


def _as_columns(v: np.ndarray, m: int) -> tuple[np.ndarray, bool]:
    v = _as_f64(v)
    if v.ndim == 1:
        if v.shape[0] != m:
            raise ValueError(f"v has length {v.shape[0]}, expected m={m}")
        return v[:, None], True
    if v.shape[0] != m:
        raise ValueError(f"V has {v.shape[0]} rows, expected m={m}")
    return v, False


def gram(S, lam: float) -> np.ndarray:
    """Algorithm 1, Gram: W = S S^T + lambda I~, with I~ the n x n identity.

    Returns the full symmetric n x n FP64 matrix.
    """
    S = _as_f64(S)
    n = S.shape[0]
    W = S @ S.T
    W[np.arange(n), np.arange(n)] += float(lam)
    return W


def cholesky_lower(W) -> np.ndarray:
    """Algorithm 1, Cholesky: L = Chol(W), W = L L^T, L lower with a positive diagonal.

    Column-by-column (Cholesky-Crout) recurrence, read from the lower
    triangle of W only:
        L[j, j] = sqrt(W[j, j] - sum_{p<j} L[j, p]^2)
        L[i, j] = (W[i, j] - sum_{p<j} L[i, p] L[j, p]) / L[j, j],  i > j
    Raises NotPositiveDefinite at the first pivot <= 0 (or NaN).
    """
    W = _as_f64(W)
    n = W.shape[0]
    if W.shape != (n, n):
        raise ValueError("W must be square")
    L = np.zeros((n, n), dtype=np.float64)
    for j in range(n):
        Lj = L[j, :j]
        d = W[j, j] - np.dot(Lj, Lj)
        if not (d > 0.0):
            raise NotPositiveDefinite(j, float(d))
        ljj = np.sqrt(d)
        L[j, j] = ljj
        if j + 1 < n:
            L[j + 1:, j] = (W[j + 1:, j] - L[j + 1:, :j] @ Lj) / ljj
    return L


def forward_substitution(L, B) -> np.ndarray:
    """Solve L A = B for A, L lower triangular (first triangular solve, L^{-1} S v).

    Row recurrence: A[i] = (B[i] - sum_{p<i} L[i, p] A[p]) / L[i, i].
    B may be a vector or an (n, k) matrix.
    """
    L = _as_f64(L)
    B = _as_f64(B)
    vec = B.ndim == 1
    B2 = B[:, None] if vec else B
    n = L.shape[0]
    A = np.zeros_like(B2)
    for i in range(n):
        A[i] = (B2[i] - L[i, :i] @ A[:i]) / L[i, i]
    return A[:, 0] if vec else A


def back_substitution_transposed(L, A) -> np.ndarray:
    """Solve L^T Y = A for Y, L lower triangular (second solve, L^{-T} L^{-1} S v).

    Row recurrence from the bottom: Y[i] = (A[i] - sum_{p>i} L[p, i] Y[p]) / L[i, i].
    """
    L = _as_f64(L)
    A = _as_f64(A)
    vec = A.ndim == 1
    A2 = A[:, None] if vec else A
    n = L.shape[0]
    Y = np.zeros_like(A2)
    for i in range(n - 1, -1, -1):
        Y[i] = (A2[i] - L[i + 1:, i] @ Y[i + 1:]) / L[i, i]
    return Y[:, 0] if vec else Y


def solve_steps(S, V, lam: float) -> dict:
    """Algorithm 1 with Q inlined, evaluated right to left; returns every intermediate.

    Steps (Algorithm 1 and the Section 2 remark on inlining Q):
        W = S S^T + lambda I~          (Gram)
        L = Chol(W)                     (Cholesky)
        b = S v                         (rightmost product of S^T L^{-T} L^{-1} S v)
        a = L^{-1} b                    (forward triangular solve)
        y = L^{-T} a                    (backward triangular solve)
        z = S^T y                       (= Q^T Q v)
        x = (v - z) / lambda            (update of x)
    Keys: W, L, b, a, y, z, x.  V (and x) have shape (m,) or (m, k).
    """
    lam = float(lam)
    if not (lam > 0.0) or not np.isfinite(lam):
        raise ValueError("lambda must be a finite positive number (Appendix A)")
    S = _as_f64(S)
    m = S.shape[1]
    V2, vec = _as_columns(V, m)
    W = gram(S, lam)
    L = cholesky_lower(W)
    b = S @ V2
    a = forward_substitution(L, b)
    y = back_substitution_transposed(L, a)
    z = S.T @ y
    x = (V2 - z) / lam
    out = dict(W=W, L=L, b=b, a=a, y=y, z=z, x=x)
    if vec:
        for key in ("b", "a", "y", "z", "x"):
            out[key] = out[key][:, 0]
    return out


def solve(S, V, lam: float) -> np.ndarray:
    """x = (S^T S + lambda I)^{-1} v by Algorithm 1 (FP64).  See solve_steps."""
    return solve_steps(S, V, lam)["x"]


def apply_operator(S, X, lam: float) -> np.ndarray:
    """Matrix-free Eq. 1 operator: (S^T S + lambda I) x = S^T (S x) + lambda x, FP64."""
    S = _as_f64(S)
    X = _as_f64(X)
    return S.T @ (S @ X) + float(lam) * X


def residual_n_space(S, V, Y, lam: float) -> np.ndarray:
    """n-space residual r = S v - (S S^T + lambda I~) y = S (v - S^T y) - lambda y.

    Appendix A: the solution satisfies (S S^T + lambda I~) S x* = S v; the
    vector y of Algorithm 1 solves (S S^T + lambda I~) y = S v, so r is its
    residual.  Written as S (v - S^T y) - lambda y it is one pass over S.
    """
    S = _as_f64(S)
    m = S.shape[1]
    V2, vec = _as_columns(V, m)
    Y2 = _as_f64(Y)
    Y2 = Y2[:, None] if Y2.ndim == 1 else Y2
    r = S @ (V2 - S.T @ Y2) - float(lam) * Y2
    return r[:, 0] if vec else r


def sr_scores(O) -> np.ndarray:
    """Section 4, stochastic reconfiguration: S = (O - O_bar) / sqrt(n), with O the n x m matrix of
    log-derivatives of the wave function (one row per sample) and O_bar its average over the
    samples, i.e. the mean of each column over the n rows.  FP64."""
    O = _as_f64(O)
    n = O.shape[0]
    return (O - O.mean(axis=0, keepdims=True)) / np.sqrt(n)


def solve_batched(problems) -> list:
    """Independent solves: problems is an iterable of (S, V, lambda); one Algorithm 1 each."""
    return [solve(S, V, lam) for (S, V, lam) in problems]


def errors(S, V, lam: float, X, X_ref) -> dict:
    """Accuracy measures of a candidate solution X against the oracle's X_ref.

    e_rel   = ||x - x*|| / ||x*||            (per column, max over columns)
    e_range = ||S (x - x*)|| / ||S x*||       (error inside the row space of S)
    res     = ||(S^T S + lambda I) x - v|| / ||v||  (Eq. 1 residual, FP64)
    """
    S = _as_f64(S)
    m = S.shape[1]
    V2, _ = _as_columns(V, m)
    X2, _ = _as_columns(X, m)
    R2, _ = _as_columns(X_ref, m)
    D = X2 - R2
    e_rel = np.linalg.norm(D, axis=0) / np.maximum(np.linalg.norm(R2, axis=0), np.finfo(float).tiny)
    SR = S @ R2
    e_range = np.linalg.norm(S @ D, axis=0) / np.maximum(np.linalg.norm(SR, axis=0), np.finfo(float).tiny)
    res = np.linalg.norm(apply_operator(S, X2, lam) - V2, axis=0) / np.maximum(
        np.linalg.norm(V2, axis=0), np.finfo(float).tiny)
    return dict(e_rel=float(e_rel.max()), e_range=float(e_range.max()), res=float(res.max()))
