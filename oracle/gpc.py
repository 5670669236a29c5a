"""Generalised polynomial chaos surrogate, plain numpy (arXiv:1906.01632).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may use this module; the product path never does.
It shares no code with the CUDA path.

What it computes, in the paper's order and notation (Section 3, "Generalized
Polynomial Chaos Expansion" and "Computing probability density functions";
Appendix A, "Legendre polynomials"):

* the 1D Legendre polynomials by the three-term recurrence of Appendix A;
* the multivariate basis P_beta(theta) = prod_j P_{beta_j}(theta_j) over a
  truncated multi-index set J_{M,p} (rule b, total degree <= p, is the
  default; rule c, every degree <= p, and a reading of rule a are offered);
* the coefficients by projection (eq. PCEcoef with the uniform density 1/2
  per dimension of Appendix A):
      u_beta(x) = 0.5^M / Q_beta * sum_i w_i P_beta(theta_i) u(x, theta_i),
      Q_beta = prod_j 1 / (2 beta_j + 1);
* the mean u_0 (eq. PCEcoef2) and the variance sum_{beta != 0} Q_beta u_beta^2
  (eq. var);
* the surrogate at sample points (eq. PCEpoint) and the exceedance estimate
  #{u_hat(theta_k) > c*} / N_s.

The quadrature nodes and weights are a library primitive
(numpy.polynomial.legendre.leggauss); everything else is written out.

Parity status: pinned in tests/test_oracle_gpc.py by a library Legendre
evaluation, Gauss-Legendre exactness and discrete orthogonality, exact
recovery of known polynomial coefficients, closed-form mean and variance of
smooth functions of uniform variables, and an exceedance count on a
midpoint grid with a closed-form answer.
"""
from __future__ import annotations

import itertools

import numpy as np


def legendre(n: int, x) -> np.ndarray:
    """[n+1, *x.shape]: P_0..P_n at x by (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
    (Appendix A)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((n + 1,) + x.shape)
    out[0] = 1.0
    if n >= 1:
        out[1] = x
    for k in range(1, n):
        out[k + 1] = ((2 * k + 1) * x * out[k] - k * out[k - 1]) / (k + 1)
    return out


def gauss_legendre(q: int):
    """q-point Gauss-Legendre rule on [-1, 1] (weights sum to 2)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


def tensor_grid(q: int, M: int):
    """Full tensor product of the q-point rule in M dimensions.  Point
    i = i_1 + q i_2 + q^2 i_3 + ... (first variable fastest); weights are the
    products of the 1D weights (they sum to 2^M)."""
    x, w = gauss_legendre(q)
    pts = np.empty((q ** M, M))
    wts = np.empty(q ** M)
    for i in range(q ** M):
        r = i
        wt = 1.0
        for j in range(M):
            k = r % q
            r //= q
            pts[i, j] = x[k]
            wt *= w[k]
        wts[i] = wt
    return pts, wts


def multi_indices(M: int, p: int, rule: str = "total") -> np.ndarray:
    """Truncated multi-index set J_{M,p} (Section 3), sorted by total degree,
    then lexicographically; beta = 0 comes first.

    rule "total": sum_j beta_j <= p (rule b);
    rule "tensor": beta_j <= p for every j (rule c);
    rule "hyperbolic": prod_j (beta_j + 1) <= p + 1 (the reading taken of
    rule a, whose printed form prod_j beta_j <= p admits every index with a
    zero component)."""
    out = []
    for beta in itertools.product(range(p + 1), repeat=M):
        if rule == "total":
            ok = sum(beta) <= p
        elif rule == "tensor":
            ok = True
        elif rule == "hyperbolic":
            ok = int(np.prod([b + 1 for b in beta])) <= p + 1
        else:
            raise ValueError(rule)
        if ok:
            out.append(beta)
    out.sort(key=lambda b: (sum(b), b))
    return np.array(out, dtype=np.int32).reshape(-1, M)


def norms(beta: np.ndarray) -> np.ndarray:
    """Q_beta = E[P_beta^2] = prod_j 1 / (2 beta_j + 1) (eq. spro)."""
    return np.prod(1.0 / (2.0 * beta + 1.0), axis=1)


def basis(beta: np.ndarray, theta) -> np.ndarray:
    """[Ns, T]: P_beta(theta_k) = prod_j P_{beta_j}(theta_kj)."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    Ns, M = theta.shape
    p = int(beta.max()) if beta.size else 0
    L = [legendre(p, theta[:, j]) for j in range(M)]  # each [p+1, Ns]
    out = np.ones((Ns, beta.shape[0]))
    for t in range(beta.shape[0]):
        for j in range(M):
            out[:, t] *= L[j][beta[t, j]]
    return out


def project(values, theta, w, beta) -> np.ndarray:
    """[T, N] coefficients of the truncated expansion by quadrature
    (eq. PCEcoef, Appendix A): values[i, n] = u(x_n, theta_i)."""
    values = np.asarray(values, dtype=np.float64)
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    w = np.asarray(w, dtype=np.float64)
    M = theta.shape[1]
    B = basis(beta, theta)  # [Nq, T]
    Q = norms(beta)
    coef = np.zeros((beta.shape[0], values.shape[1]))
    for t in range(beta.shape[0]):
        acc = np.zeros(values.shape[1])
        for i in range(values.shape[0]):
            acc += w[i] * B[i, t] * values[i]
        coef[t] = 0.5 ** M * acc / Q[t]
    return coef


def mean_var(coef, beta):
    """Mean u_0 (eq. PCEcoef2) and variance sum_{beta != 0} Q_beta u_beta^2
    (eq. var); beta[0] must be the zero index."""
    assert not beta[0].any()
    Q = norms(beta)
    var = np.zeros(coef.shape[1])
    for t in range(1, beta.shape[0]):
        var += Q[t] * coef[t] ** 2
    return coef[0].copy(), var


def evaluate(coef, beta, theta) -> np.ndarray:
    """[Ns, N]: the surrogate at the sample points (eq. PCEpoint)."""
    return basis(beta, theta) @ np.asarray(coef, dtype=np.float64)


def exceedance(coef, beta, theta, threshold: float, chunk: int = 4096) -> np.ndarray:
    """[N]: #{u_hat(theta_k) > threshold} / N_s (Section 3, exceedance
    estimate), evaluated in chunks of samples."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    count = np.zeros(np.asarray(coef).shape[1], dtype=np.int64)
    for k0 in range(0, theta.shape[0], chunk):
        count += (evaluate(coef, beta, theta[k0:k0 + chunk]) > threshold).sum(axis=0)
    return count / theta.shape[0]
