"""The seeded input generators: shapes, determinism and the structure each recipe promises."""

import math

import torch

from paper_2310_17556_gb300 import workloads as wl


def test_gaussian_deterministic_and_scaled():
    a = wl.gaussian(64, 4096, seed=5)
    b = wl.gaussian(64, 4096, seed=5)
    assert a.shape == (64, 4096) and a.dtype == torch.float32
    assert torch.equal(a, b)
    assert not torch.equal(a, wl.gaussian(64, 4096, seed=6))
    # entries ~ N(0, 1/n)
    assert abs(a.double().var().item() * 64 - 1.0) < 0.05


def test_rhs_layout():
    v = wl.rhs(1000, 3, seed=1)
    assert v.shape == (3, 1000) and v.dtype == torch.float32
    assert torch.equal(v, wl.rhs(1000, 3, seed=1))


def test_orthonormal_rows():
    S = wl.orthonormal_rows(16, 300, seed=2)
    assert torch.allclose(S @ S.T, torch.eye(16, dtype=torch.float64), atol=1e-13)


def test_svd_structured_factors():
    S, U, s, V = wl.svd_structured(32, 500, seed=3, sigma_min=1e-3, dtype=torch.float64)
    assert torch.allclose(U.T @ U, torch.eye(32, dtype=torch.float64), atol=1e-12)
    assert torch.allclose(V.T @ V, torch.eye(32, dtype=torch.float64), atol=1e-12)
    assert abs(s[0].item() - 1 / math.sqrt(32)) < 1e-15
    assert abs(s[-1].item() - 1e-3 / math.sqrt(32)) < 1e-15
    sv = torch.linalg.svdvals(S)
    assert torch.allclose(sv, s, rtol=1e-9, atol=1e-15)


def test_heavy_tailed_bf16():
    S = wl.heavy_tailed(8, 5000, seed=4)
    assert S.dtype == torch.bfloat16 and S.shape == (8, 5000)
    assert torch.isfinite(S.float()).all()
    assert torch.equal(S, wl.heavy_tailed(8, 5000, seed=4))


def test_ragged_batch_shapes_ranges():
    shapes = wl.ragged_batch_shapes(64, seed=9)
    assert len(shapes) == 64
    for n, m, lam in shapes:
        assert 64 <= n <= 1024
        assert 10000 <= m <= 500000
        assert 1e-5 <= lam <= 1e-1
    assert shapes == wl.ragged_batch_shapes(64, seed=9)
