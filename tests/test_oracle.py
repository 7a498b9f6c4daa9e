"""Pins for the FP64 oracle, against facts that do not come from the oracle itself.

Each check is fixed by the paper (arXiv 2310.17556) or by mathematics:
a dense LAPACK solve of Eq. 1, exact rational Gauss-Jordan fixtures, the
orthonormal-row closed form of Algorithm 1, Appendix C's SVD closed form,
Appendix B's equivalence for v = S^T f, the n = 1 Sherman-Morrison form, the
S = 0 and large-lambda limits, Appendix A's intermediate identity, a textbook
Cholesky example and LAPACK/SciPy triangular routines.  The last test plants
plausible mistakes in the oracle and checks that a pin catches each one.
"""

import glob
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import alg1
from oracle.exact import solve_dense_exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dense_solve(S, V, lam):
    """Eq. 1 solved directly: the m x m system (S^T S + lam I) x = v via LAPACK."""
    S = np.asarray(S, np.float64)
    A = S.T @ S + lam * np.eye(S.shape[1])
    return np.linalg.solve(A, V)


@pytest.mark.parametrize("n,m,k,lam", [
    (1, 7, 1, 0.3), (3, 40, 2, 1e-2), (16, 300, 1, 1e-3), (64, 700, 3, 1e-1),
    (50, 30, 1, 0.5),   # m < n: still SPD, still solvable
    (8, 8, 2, 1e-4),
])
def test_matches_dense_lapack_solve(n, m, k, lam):
    rng = np.random.default_rng(1000 + n * 7 + m)
    S = rng.standard_normal((n, m)) / math.sqrt(n)
    V = rng.standard_normal((m, k))
    x = oracle.solve(S, V, lam)
    assert x.shape == (m, k)
    cond = (np.linalg.norm(S, 2) ** 2 + lam) / lam
    assert rel(x, dense_solve(S, V, lam)) <= 1e-13 * cond * 10


def test_vector_rhs_shape():
    rng = np.random.default_rng(2)
    S = rng.standard_normal((5, 20))
    v = rng.standard_normal(20)
    x = oracle.solve(S, v, 0.7)
    assert x.shape == (20,)
    assert rel(x, dense_solve(S, v, 0.7)) < 1e-12


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "eq1_exact_*.json"))))
def test_exact_rational_fixtures(path):
    with open(path) as f:
        doc = json.load(f)
    S = np.array(doc["S"], dtype=np.float64)
    v = np.array(doc["v"], dtype=np.float64)
    lam = float(Fraction(doc["lambda"]))
    x_exact = np.array([float(Fraction(e)) for e in doc["x"]])
    x = oracle.solve(S, v, lam)
    assert rel(x, x_exact) < 1e-12


def test_exact_rational_random_tiny():
    rng = np.random.default_rng(7)
    for trial in range(12):
        n = int(rng.integers(1, 4))
        m = int(rng.integers(1, 6))
        S = rng.integers(-3, 4, size=(n, m))
        v = rng.integers(-5, 6, size=m)
        lam = Fraction(int(rng.integers(1, 9)), int(rng.choice([1, 10, 100])))
        x_exact = solve_dense_exact(S.tolist(), v.tolist(), lam)
        x = oracle.solve(S.astype(float), v.astype(float), float(lam))
        assert rel(x, [float(e) for e in x_exact]) < 1e-11, (trial, n, m)


@pytest.mark.parametrize("lam", [1e-3, 0.25, 3.0])
def test_orthonormal_rows_closed_form(lam):
    # S S^T = I  =>  W = (1 + lam) I, L = sqrt(1 + lam) I, x = (v - S^T S v / (1 + lam)) / lam
    rng = np.random.default_rng(11)
    n, m = 24, 500
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    S = Q.T
    v = rng.standard_normal(m)
    st = oracle.solve_steps(S, v, lam)
    assert np.abs(st["W"] - (1 + lam) * np.eye(n)).max() < 1e-13
    assert np.abs(st["L"] - math.sqrt(1 + lam) * np.eye(n)).max() < 1e-13
    x_cf = (v - S.T @ (S @ v) / (1 + lam)) / lam
    assert rel(st["x"], x_cf) < 1e-13


@pytest.mark.parametrize("lam", [1e-2, 1e-4])
def test_svd_closed_form_appendix_c(lam):
    # Appendix C: x = V (Sigma^2 + lam)^-1 V^T v + (v - V V^T v) / lam
    rng = np.random.default_rng(13)
    n, m = 32, 900
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((m, n)))
    s = np.logspace(0, -3, n) / math.sqrt(n)
    S = (U * s) @ V.T
    v = rng.standard_normal(m)
    Vtv = V.T @ v
    x_cf = V @ (Vtv / (s ** 2 + lam)) + (v - V @ Vtv) / lam
    assert rel(oracle.solve(S, v, lam), x_cf) < 1e-12


def test_rende_equivalence_appendix_b():
    # Appendix B: for v = S^T f, x = S^T (S S^T + lam I~)^{-1} f
    rng = np.random.default_rng(17)
    n, m, lam = 20, 200, 3e-2
    S = rng.standard_normal((n, m)) / math.sqrt(n)
    f = rng.standard_normal(n)
    v = S.T @ f
    x_rvb = S.T @ np.linalg.solve(S @ S.T + lam * np.eye(n), f)
    assert rel(oracle.solve(S, v, lam), x_rvb) < 1e-12


def test_n1_sherman_morrison():
    # n = 1: (s s^T + lam I) x = v  =>  x = (v - s (s.v) / (|s|^2 + lam)) / lam
    rng = np.random.default_rng(19)
    s = rng.standard_normal(333)
    v = rng.standard_normal(333)
    lam = 0.05
    x_cf = (v - s * (s @ v) / (s @ s + lam)) / lam
    assert rel(oracle.solve(s[None, :], v, lam), x_cf) < 1e-13


def test_zero_score_matrix():
    v = np.linspace(-1, 1, 50)
    x = oracle.solve(np.zeros((4, 50)), v, 0.125)
    assert np.array_equal(x, v / 0.125)


def test_large_lambda_limit():
    rng = np.random.default_rng(23)
    S = rng.standard_normal((6, 80)) / math.sqrt(6)
    v = rng.standard_normal(80)
    lam = 1e8
    # lam x - v = -S^T S x, so |lam x - v| <= |S|^2 |v| / lam
    bound = np.linalg.norm(S, 2) ** 2 / lam
    assert rel(lam * oracle.solve(S, v, lam), v) <= bound * 1.01


def test_appendix_a_intermediate_identity():
    # Appendix A: S S^T S x* + lam S x* = S v
    rng = np.random.default_rng(29)
    S = rng.standard_normal((12, 150)) / math.sqrt(12)
    v = rng.standard_normal(150)
    lam = 1e-3
    x = oracle.solve(S, v, lam)
    lhs = S @ (S.T @ (S @ x)) + lam * (S @ x)
    assert rel(lhs, S @ v) < 1e-11


def test_cholesky_textbook_example():
    W = np.array([[4.0, 12, -16], [12, 37, -43], [-16, -43, 98]])
    L_exact = np.array([[2.0, 0, 0], [6, 1, 0], [-8, 5, 3]])
    assert np.array_equal(oracle.cholesky_lower(W), L_exact)


def test_cholesky_matches_lapack_and_reconstructs():
    rng = np.random.default_rng(31)
    A = rng.standard_normal((70, 200))
    W = A @ A.T + 0.1 * np.eye(70)
    L = oracle.cholesky_lower(W)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert (np.diag(L) > 0).all()
    assert np.abs(L @ L.T - W).max() < 1e-12 * np.abs(W).max()
    assert np.abs(L - np.linalg.cholesky(W)).max() < 1e-12 * np.abs(L).max()


def test_cholesky_reads_lower_triangle_only():
    rng = np.random.default_rng(37)
    A = rng.standard_normal((9, 30))
    W = A @ A.T + np.eye(9)
    Wg = np.tril(W) + np.triu(np.full_like(W, 1e30), 1)
    assert np.array_equal(oracle.cholesky_lower(W), oracle.cholesky_lower(Wg))


def test_cholesky_not_spd_reports_pivot():
    W = np.diag([2.0, 1.0, -1.0, 4.0])
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky_lower(W)
    assert e.value.pivot == 2


def test_substitutions_match_scipy():
    rng = np.random.default_rng(41)
    n = 40
    L = np.tril(rng.standard_normal((n, n))) + 5 * np.eye(n)
    B = rng.standard_normal((n, 3))
    A = oracle.forward_substitution(L, B)
    assert rel(A, scipy.linalg.solve_triangular(L, B, lower=True)) < 1e-13
    Y = oracle.back_substitution_transposed(L, B)
    assert rel(Y, scipy.linalg.solve_triangular(L, B, lower=True, trans="T")) < 1e-13


def test_residual_and_operator():
    rng = np.random.default_rng(43)
    n, m, lam = 10, 120, 2e-2
    S = rng.standard_normal((n, m))
    V = rng.standard_normal((m, 2))
    st = oracle.solve_steps(S, V, lam)
    # r(0) = S v, r(y) = 0 at the solution of (S S^T + lam I) y = S v
    assert rel(oracle.residual_n_space(S, V, np.zeros((n, 2)), lam), S @ V) < 1e-15
    r = oracle.residual_n_space(S, V, st["y"], lam)
    assert np.linalg.norm(r) < 1e-10 * np.linalg.norm(S @ V)
    A = S.T @ S + lam * np.eye(m)
    X = rng.standard_normal((m, 2))
    assert rel(oracle.apply_operator(S, X, lam), A @ X) < 1e-14


def test_error_metrics():
    rng = np.random.default_rng(47)
    S = rng.standard_normal((4, 60))
    v = rng.standard_normal(60)
    x = oracle.solve(S, v, 0.3)
    e = oracle.errors(S, v, 0.3, x, x)
    assert e["e_rel"] == 0.0 and e["e_range"] == 0.0 and e["res"] < 1e-12
    e2 = oracle.errors(S, v, 0.3, 1.01 * x, x)
    assert abs(e2["e_rel"] - 0.01) < 1e-12


@pytest.mark.parametrize("lam", [0.0, -1.0, float("nan"), float("inf")])
def test_invalid_lambda(lam):
    with pytest.raises(ValueError):
        oracle.solve(np.ones((2, 3)), np.ones(3), lam)


def test_batched_is_per_problem():
    rng = np.random.default_rng(53)
    probs = []
    for n, m in [(3, 20), (7, 50), (1, 9)]:
        probs.append((rng.standard_normal((n, m)), rng.standard_normal(m), 0.1))
    for (S, v, lam), x in zip(probs, oracle.solve_batched(probs)):
        assert rel(x, dense_solve(S, v, lam)) < 1e-12


# ---------------------------------------------------------------------------
# planted mistakes: each plausible slip in the oracle must fail a pin above


def _pin_dense(solve_fn):
    rng = np.random.default_rng(59)
    S = rng.standard_normal((6, 40)) / math.sqrt(6)
    v = rng.standard_normal(40)
    return rel(solve_fn(S, v, 0.05), dense_solve(S, v, 0.05)) < 1e-10


def test_sr_scores_section4_invariants():
    """Section 4's SR scores S = (O - O_bar) / sqrt(n): rows that all agree give S = 0 (so x = v /
    lambda); a common offset added to every row changes nothing; every column of S sums to zero;
    the 1 / sqrt(n) scale is the one of Section 2's S."""
    rng = np.random.default_rng(5)
    n, m = 7, 11
    mu = rng.standard_normal(m)
    # zero up to the rounding of the column mean (a sum of n equal values divided by n)
    assert np.abs(oracle.sr_scores(np.tile(mu, (n, 1)))).max() <= 4 * np.finfo(float).eps * np.abs(mu).max()
    v = rng.standard_normal(m)
    np.testing.assert_allclose(oracle.solve(oracle.sr_scores(np.tile(mu, (n, 1))), v, 0.3), v / 0.3, rtol=1e-14)
    O = rng.standard_normal((n, m))
    S = oracle.sr_scores(O)
    np.testing.assert_allclose(oracle.sr_scores(O + mu[None, :]), S, atol=1e-14)
    np.testing.assert_allclose(S.sum(axis=0), 0.0, atol=1e-14)
    # one sample away from the mean by e_j: S_ij = (1 - 1/n) / sqrt(n) there, -1/(n sqrt(n)) elsewhere
    E = np.zeros((n, m))
    E[2, 4] = 1.0
    Se = oracle.sr_scores(E)
    assert math.isclose(Se[2, 4], (1 - 1 / n) / math.sqrt(n), rel_tol=1e-14)
    assert math.isclose(Se[0, 4], -1 / (n * math.sqrt(n)), rel_tol=1e-14)


@pytest.mark.parametrize("lam", [1e-3, 0.5])
def test_sr_two_samples_closed_form(lam):
    """n = 2: S = [d; -d] / (2 sqrt 2) with d = o_1 - o_2, so S^T S = d d^T / 4 and Eq. 1 has the
    Sherman-Morrison solution x = v / lambda - d (d . v) / (lambda (4 lambda + ||d||^2))."""
    rng = np.random.default_rng(6)
    m = 9
    O = rng.standard_normal((2, m))
    v = rng.standard_normal(m)
    d = O[0] - O[1]
    x_cf = v / lam - d * (d @ v) / (lam * (4 * lam + d @ d))
    np.testing.assert_allclose(oracle.solve(oracle.sr_scores(O), v, lam), x_cf, rtol=1e-12, atol=1e-12)


def _complex_case(n, m, seed):
    rng = np.random.default_rng(seed)
    S = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / np.sqrt(2 * n)
    v = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    return S, v


@pytest.mark.parametrize("n,m,lam", [(5, 17, 0.3), (12, 9, 1e-2), (1, 6, 0.7)])
def test_complex_solve_matches_dense_hermitian_system(n, m, lam):
    """Section 4, complex SR: (S^dagger S + lambda I) x = v, checked against a dense complex
    LAPACK solve of that m x m system (a different algorithm from Algorithm 1)."""
    S, v = _complex_case(n, m, seed=11 + n)
    A = np.conj(S.T) @ S + lam * np.eye(m)
    np.testing.assert_allclose(oracle.solve_complex(S, v, lam), np.linalg.solve(A, v), rtol=1e-11, atol=1e-12)


def test_complex_solve_single_row_closed_form():
    """n = 1: S^dagger S = s^dagger s, so x = (v - s^dagger (s v) / (||s||^2 + lambda)) / lambda."""
    S, v = _complex_case(1, 8, seed=21)
    lam = 0.4
    s = S[0]
    x_cf = (v - np.conj(s) * (s @ v) / (np.vdot(s, s).real + lam)) / lam
    np.testing.assert_allclose(oracle.solve_complex(S, v, lam), x_cf, rtol=1e-12, atol=1e-12)


def test_complex_solve_with_real_scores_splits_into_two_real_solves():
    """Real S: the system does not mix Re x and Im x, so each is the real Algorithm 1's answer."""
    rng = np.random.default_rng(23)
    S = rng.standard_normal((6, 14))
    v = rng.standard_normal(14) + 1j * rng.standard_normal(14)
    x = oracle.solve_complex(S, v, 0.2)
    np.testing.assert_allclose(x.real, oracle.solve(S, v.real, 0.2), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(x.imag, oracle.solve(S, v.imag, 0.2), rtol=1e-12, atol=1e-12)


def test_real_part_scores_give_the_real_part_of_the_fisher_matrix():
    """Section 4, real-part SR: Concat[Re S, Im S] along n has S^T S = Re[S^dagger S]; the real
    solve on it matches a dense solve with Re[S^dagger S]."""
    S, _ = _complex_case(7, 11, seed=25)
    v = np.random.default_rng(26).standard_normal(11)
    Sr = oracle.real_part_scores(S)
    assert Sr.shape == (14, 11)
    np.testing.assert_allclose(Sr.T @ Sr, (np.conj(S.T) @ S).real, rtol=1e-12, atol=1e-13)
    A = (np.conj(S.T) @ S).real + 0.3 * np.eye(11)
    np.testing.assert_allclose(oracle.solve(Sr, v, 0.3), np.linalg.solve(A, v), rtol=1e-11, atol=1e-12)


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pin_dense(oracle.solve)

    def sign_flip(S, V, lam):
        st = alg1.solve_steps(S, V, lam)
        return (np.asarray(V) + st["z"]) / lam

    assert not _pin_dense(sign_flip)

    with monkeypatch.context() as mp:  # dropped damping term in W
        mp.setattr(alg1, "gram", lambda S, lam: np.asarray(S, np.float64) @ np.asarray(S, np.float64).T)
        assert not _pin_dense(alg1.solve)

    with monkeypatch.context() as mp:  # backward solve with L instead of L^T
        mp.setattr(alg1, "back_substitution_transposed",
                   lambda L, A: scipy.linalg.solve_triangular(L, A, lower=True))
        assert not _pin_dense(alg1.solve)

    with monkeypatch.context() as mp:  # wrong index in the Cholesky recurrence (uses W's row, not column)
        def bad_chol(W):
            W = np.asarray(W, np.float64)
            n = W.shape[0]
            L = np.zeros_like(W)
            for j in range(n):
                L[j, j] = math.sqrt(W[j, j] - L[j, :j] @ L[j, :j])
                L[j + 1:, j] = (W[j, j + 1:] * 0.5 + W[j + 1:, j] * 0.5 - L[j + 1:, :j] @ L[j, :j]) / L[j, j] * 1.001
            return L
        mp.setattr(alg1, "cholesky_lower", bad_chol)
        assert not _pin_dense(alg1.solve)
