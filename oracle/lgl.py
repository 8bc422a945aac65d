"""Legendre-Gauss-Lobatto collocation (Sec. II, Eqs. field_expansion and lagrprod).

Oracle code (test infrastructure only). N points per dimension: the endpoints -1, +1 and the
N-2 roots of P'_{N-1}; quadrature weights w_k = 2 / (N (N-1) P_{N-1}(x_k)^2); Lagrange
polynomials l_j on those points, their derivatives and interpolation to arbitrary points.
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the three-term (Bonnet) recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n), valid away from +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    end = np.isclose(np.abs(x), 1.0, rtol=0, atol=0)
    dp = np.where(end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def lgl_nodes(N: int) -> np.ndarray:
    """The N LGL points in ascending order: -1, roots of P'_{N-1}, +1 (Newton iteration)."""
    if N < 2:
        raise ValueError("LGL needs N >= 2")
    p = N - 1
    x = -np.cos(np.pi * np.arange(N) / p)  # Chebyshev-Gauss-Lobatto start
    inner = x[1:-1].copy()
    for _ in range(100):
        P, dP = legendre(p, inner)
        # Legendre ODE: (1 - x^2) P'' = 2 x P' - p (p + 1) P
        d2P = (2 * inner * dP - p * (p + 1) * P) / (1.0 - inner**2)
        step = dP / d2P
        inner = inner - step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[1:-1] = inner
    x[0], x[-1] = -1.0, 1.0
    # enforce the exact symmetry of the point set
    return 0.5 * (x - x[::-1])


def lgl_weights(N: int) -> np.ndarray:
    x = lgl_nodes(N)
    P, _ = legendre(N - 1, x)
    return 2.0 / (N * (N - 1) * P * P)


def lagrange(xs: np.ndarray, j: int, t):
    """l_j(t) = prod_{k != j} (t - x_k) / (x_j - x_k)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    for k, xk in enumerate(xs):
        if k != j:
            out = out * (t - xk) / (xs[j] - xk)
    return out


def lagrange_deriv(xs: np.ndarray, j: int, t):
    """l_j'(t) by the product rule: sum_m [1/(x_j - x_m)] prod_{k != j, m} (t - x_k)/(x_j - x_k)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    for m, xm in enumerate(xs):
        if m == j:
            continue
        term = np.full_like(t, 1.0 / (xs[j] - xm))
        for k, xk in enumerate(xs):
            if k != j and k != m:
                term = term * (t - xk) / (xs[j] - xk)
        out = out + term
    return out


def diff_matrix(N: int) -> np.ndarray:
    """D_hat[k, l] = l_l'(x_k): logical-coordinate derivative of the nodal interpolant."""
    xs = lgl_nodes(N)
    return np.stack([lagrange_deriv(xs, l, xs) for l in range(N)], axis=1)


def interp_matrix(N_from: int, targets) -> np.ndarray:
    """I[t, j] = l_j(targets[t]) for the N_from LGL points."""
    xs = lgl_nodes(N_from)
    return np.stack([lagrange(xs, j, targets) for j in range(N_from)], axis=1)
