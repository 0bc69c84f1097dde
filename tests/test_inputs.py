"""The seeded input recipe (fe_inputs.py) against its stated definitions, CPU only.

kappa = exp(g) with g a random-Fourier-feature field: over draws of the features, g(x) has mean 0 and covariance
sigma^2 exp(-|x - y|^2 / (2 l^2)) (the squared-exponential kernel; E cos(omega . r) for omega ~ N(0, l^-2 I)).
The manufactured right-hand sides are -Laplace of their solutions; the batched table has the stated sizes and mix.
"""
import numpy as np
import pytest

import fe_inputs as I


def test_grf_covariance_is_the_squared_exponential_kernel():
    pts = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5], [0.7, 0.5, 0.5], [0.5, 0.9, 0.5], [0.3, 0.3, 0.3]])
    g = np.log(np.stack([I.grf_kappa(pts, seed=s) for s in range(1500)]))  # (draws, points)
    assert np.abs(g.mean(axis=0)).max() < 0.1
    C = np.cov(g, rowvar=False)
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    K = np.exp(-d2 / (2 * 0.2 ** 2))
    assert np.abs(C - K).max() < 0.12, np.round(C - K, 3)


def test_grf_is_deterministic_and_positive():
    pts = np.random.default_rng(0).uniform(0, 1, (1000, 3))
    a, b = I.grf_kappa(pts, seed=7), I.grf_kappa(pts, seed=7, chunk=97)
    assert np.array_equal(a, b) and (a > 0).all()
    assert not np.array_equal(a, I.grf_kappa(pts, seed=8))


def test_sin_product_rhs_is_minus_laplacian():
    x = np.random.default_rng(1).uniform(0.05, 0.95, (50, 3))
    h = 1e-4
    lap = sum((I.sin_product(x + h * e) - 2 * I.sin_product(x) + I.sin_product(x - h * e)) / h ** 2
              for e in np.eye(3))
    assert np.allclose(-lap, I.sin_product_rhs(x), rtol=1e-6, atol=1e-5)


def test_target_field_recipe():
    amp, freq = I.target_field_params()
    assert amp.shape == (8,) and freq.shape == (8, 3)
    assert set(np.unique(freq)) <= {1, 2, 3}
    x = np.random.default_rng(2).uniform(0, 1, (20, 3))
    ref = sum(a * np.prod(np.sin(np.pi * f * x), axis=1) for a, f in zip(amp, freq))
    assert np.allclose(I.target_field(x), ref, rtol=1e-14, atol=1e-14)
    # vanishes on the boundary (homogeneous Dirichlet data)
    xb = x.copy()
    xb[:, 1] = 1.0
    assert np.abs(I.target_field(xb)).max() < 1e-12


@pytest.mark.parametrize("n", [64, 7])
def test_batched_problem_table(n):
    t = I.batched_problem_table(n_problems=n)
    assert len(t) == n
    assert {N for N, _ in t} <= {16, 24, 32, 40, 48}
    degs = [k for _, k in t]
    assert degs.count(1) == n // 2 and degs.count(2) == n - n // 2
    assert t == I.batched_problem_table(n_problems=n)  # seeded
