"""Gauss-Legendre (GL) and Gauss-Lobatto-Legendre (LGL) quadrature.

The paper integrates on GL nodes and builds metric terms on Lobatto nodes
(Sec. "Results", quadrature choices).  Nodes come from Newton's iteration on
the Legendre recurrence, the textbook construction.
"""
from __future__ import annotations

import math

import numpy as np


def legendre_and_derivative(N, x):
    """P_N(x) and P_N'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if N == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, N + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # P_N' = N (x P_N - P_{N-1}) / (x^2 - 1); only meaningful away from x = +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = N * (x * p1 - p0) / (x * x - 1.0)
    return p1, dp


def gauss_legendre(n):
    """n-point GL rule on [-1, 1]: roots of P_n, weights 2/((1-x^2) P_n'(x)^2)."""
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(n)
    x = -np.cos(math.pi * (i + 0.75) / (n + 0.5))  # ascending initial guesses
    for _ in range(100):
        P, dP = legendre_and_derivative(n, x)
        dx = P / dP
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    P, dP = legendre_and_derivative(n, x)
    w = 2.0 / ((1.0 - x * x) * dP * dP)
    return x, w


def gauss_lobatto(n):
    """n-point LGL rule (n >= 2): +-1 and the roots of P_{n-1}'.

    Weights 2/(N(N+1) P_N(x)^2) with N = n-1.  Interior roots by Newton on
    q(x) = P_N'(x), using q'(x) = (2x P_N' - N(N+1) P_N)/(1-x^2).
    """
    if n < 2:
        raise ValueError("n >= 2")
    N = n - 1
    x = -np.cos(math.pi * np.arange(n) / N)  # Chebyshev-Lobatto initial guesses
    xi = x[1:-1].copy()
    for _ in range(100):
        P, dP = legendre_and_derivative(N, xi)
        d2P = (2.0 * xi * dP - N * (N + 1) * P) / (1.0 - xi * xi)
        dx = dP / d2P
        xi = xi - dx
        if xi.size == 0 or np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], xi, [1.0]])
    P, _ = legendre_and_derivative(N, x)
    w = 2.0 / (N * (N + 1) * P * P)
    return x, w


def equispaced(n):
    """n equispaced points on [-1, 1] (mesh control-point positions)."""
    if n == 1:
        return np.zeros(1)
    return -1.0 + 2.0 * np.arange(n) / (n - 1)
