"""Pins of the gPC oracle (Section 3 and Appendix A) against facts that do
not come from the oracle itself: a library Legendre evaluation, quadrature
exactness, known expansions, closed-form moments of uniform variables and an
exceedance count with a closed-form answer."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import gpc as G


def test_legendre_recurrence_matches_library():
    x = np.linspace(-1, 1, 41)
    L = G.legendre(8, x)
    for n in range(9):
        assert np.allclose(L[n], eval_legendre(n, x), rtol=0, atol=1e-14)


def test_legendre_printed_closed_forms():
    """Appendix A prints P_2, P_4 and P_5 in closed form; its P_3 reads
    5/2 x^2 - 3/2 x, which is not orthogonal to P_1 - the recurrence (and the
    reading 5/2 x^3 - 3/2 x) is used."""
    x = np.linspace(-1, 1, 17)
    L = G.legendre(5, x)
    assert np.allclose(L[2], 1.5 * x**2 - 0.5, atol=1e-15)
    assert np.allclose(L[3], 2.5 * x**3 - 1.5 * x, atol=1e-15)
    assert np.allclose(L[4], 35 / 8 * x**4 - 30 / 8 * x**2 + 3 / 8, atol=1e-14)
    assert np.allclose(L[5], 63 / 8 * x**5 - 70 / 8 * x**3 + 15 / 8 * x, atol=1e-14)
    xg, wg = G.gauss_legendre(8)
    printed_p3 = 2.5 * xg**2 - 1.5 * xg
    assert abs((wg * printed_p3 * xg).sum()) > 0.1  # the printed form is not orthogonal to P_1


def test_gauss_legendre_exactness_and_orthogonality():
    q = 5
    x, w = G.gauss_legendre(q)
    for k in range(2 * q):  # exact for degree <= 2q - 1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs((w * x**k).sum() - exact) < 1e-14
    # discrete orthogonality of the basis with the uniform density 1/2
    L = G.legendre(4, x)
    gram = 0.5 * (L * w) @ L.T
    assert np.allclose(gram, np.diag(1.0 / (2 * np.arange(5) + 1)), atol=1e-15)


def test_multi_index_counts():
    assert G.multi_indices(3, 4, "total").shape == (math.comb(7, 3), 3)
    assert G.multi_indices(3, 4, "tensor").shape == (125, 3)
    b = G.multi_indices(3, 4)
    assert not b[0].any() and (b.sum(1) <= 4).all()
    assert (np.diff(b.sum(1)) >= 0).all()
    h = G.multi_indices(3, 3, "hyperbolic")
    assert all(np.prod(r + 1) <= 4 for r in h)


def test_projection_recovers_known_coefficients():
    M, p, q = 3, 4, 5
    beta = G.multi_indices(M, p)
    rng = np.random.default_rng(3)
    true = rng.standard_normal((beta.shape[0], 7))
    th, w = G.tensor_grid(q, M)
    # values from an independently written product of scipy Legendre values
    vals = np.zeros((th.shape[0], 7))
    for t, b in enumerate(beta):
        P = np.ones(th.shape[0])
        for j in range(M):
            P *= eval_legendre(int(b[j]), th[:, j])
        vals += np.outer(P, true[t])
    coef = G.project(vals, th, w, beta)
    assert np.abs(coef - true).max() < 1e-12


def test_mean_variance_closed_forms():
    M, p, q = 3, 2, 3
    beta = G.multi_indices(M, p)
    th, w = G.tensor_grid(q, M)
    # f = theta_1 + theta_2 theta_3: mean 0, variance 1/3 + 1/9
    f = (th[:, 0] + th[:, 1] * th[:, 2])[:, None]
    m, v = G.mean_var(G.project(f, th, w, beta), beta)
    assert abs(m[0]) < 1e-15 and abs(v[0] - 4 / 9) < 1e-14
    # f = exp(a theta_1): mean sinh(a)/a, variance sinh(2a)/(2a) - (sinh(a)/a)^2
    a = 0.8
    beta8 = G.multi_indices(1, 10)
    th8, w8 = G.tensor_grid(12, 1)
    f = np.exp(a * th8)
    m, v = G.mean_var(G.project(f, th8, w8, beta8), beta8)
    mean = math.sinh(a) / a
    var = math.sinh(2 * a) / (2 * a) - mean**2
    assert abs(m[0] - mean) < 1e-14 and abs(v[0] - var) < 1e-12


def test_exceedance_on_midpoint_grid():
    """u = theta_1: P(theta_1 > 0.3) = 0.35; on a midpoint grid of 10^5
    points exactly 35000 exceed."""
    beta = G.multi_indices(2, 2)
    coef = np.zeros((beta.shape[0], 2))
    t1 = [t for t, b in enumerate(beta) if tuple(b) == (1, 0)][0]
    coef[t1, 0] = 1.0       # node 0: theta_1
    coef[0, 1] = 0.25       # node 1: constant 0.25, never above 0.3
    K = 100000
    g = -1 + (np.arange(K) + 0.5) * 2 / K
    theta = np.stack([g, np.zeros(K)], 1)
    pe = G.exceedance(coef, beta, theta, 0.3)
    assert pe[0] == 0.35 and pe[1] == 0.0


def test_evaluate_reproduces_quadrature_values_for_polynomials():
    beta = G.multi_indices(3, 3)
    th, w = G.tensor_grid(4, 3)
    f = (1 + th[:, 0] * th[:, 1] - 0.5 * th[:, 2] ** 3)[:, None]
    coef = G.project(f, th, w, beta)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (50, 3))
    assert np.allclose(G.evaluate(coef, beta, x)[:, 0], 1 + x[:, 0] * x[:, 1] - 0.5 * x[:, 2] ** 3,
                       atol=1e-13)
