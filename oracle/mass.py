"""Weight-adjusted inverse of the FR modified mass matrix.

Eq. weight-adj ESFR mass:  (M_m + K_m)^{-1} ~ Pi~ (W J_m)^{-1} Pi~^T,
Pi~ = Pi~1 (x) Pi~1 (x) Pi~1 (Eq. Fr projection), applied by sum
factorisation: Pi~^T along each direction, the diagonal 1/(w J), then Pi~
along each direction (Sec. "Scalable Evaluations", 2 d n^{d+1} + n^d flops).

Also provided, for comparison only: the exact modified mass matrix M_m + K_m
of Eq. Km (dense, with J inside both M_m and K_m) and Chan and Wilcox's
weight-adjusted form, Eq. weight adj inv,
(M + K)^{-1} (M_{1/J} + K_{1/J}) (M + K)^{-1}.
"""
from __future__ import annotations

import itertools

import numpy as np

from .operators1d import tensor3


def w3(ops):
    w = ops.w
    return w[:, None, None] * w[None, :, None] * w[None, None, :]


def wa_inverse_apply(R, J, ops):
    """Pi~ (W J)^{-1} Pi~^T R for every element; R is (..., N_e, n, n, n)."""
    X = tensor3(ops.Pi1.T, R)
    X = X / (w3(ops) * J)
    return tensor3(ops.Pi1, X)


def dudt_from_residual(R, J, ops):
    """du/dt = -(M_m + K_m)^{-1} R with the weight-adjusted inverse."""
    return -wa_inverse_apply(R, J, ops)


def dense_wa_inverse(Je, ops):
    """Dense Pi~ (W J)^{-1} Pi~^T for one element (Je: n^3 Jacobians, xi fastest)."""
    Pi = np.kron(ops.Pi1, np.kron(ops.Pi1, ops.Pi1))
    Wv = w3(ops).ravel()
    return Pi @ np.diag(1.0 / (Wv * Je)) @ Pi.T


def _dense_deriv_powers(ops):
    n = ops.n
    I = np.eye(n)
    Dp = ops.Dp
    out = {}
    for s, v, w in itertools.product((0, ops.p), repeat=3):
        A = Dp if w == ops.p else I   # zeta slowest
        B = Dp if v == ops.p else I
        Cx = Dp if s == ops.p else I  # xi fastest
        out[(s, v, w)] = np.kron(A, np.kron(B, Cx))
    return out


def dense_fr_mass(Je, ops):
    """M_m + K_m of Eq. Km for one element: sum over (s,v,w) in {0,p}^3.

    c_(s,v,w) = c^{(s+v+w)/p}; the (0,0,0) term is M_m = W J itself.
    """
    Wv = w3(ops).ravel()
    MJ = np.diag(Wv * Je)
    total = np.zeros_like(MJ)
    for (s, v, w), Dsvw in _dense_deriv_powers(ops).items():
        k = (s + v + w) // ops.p
        coef = 1.0 if k == 0 else ops.c ** k
        total += coef * Dsvw.T @ MJ @ Dsvw
    return total


def dense_chan_wilcox(Je, ops):
    """(M + K)^{-1} (M_{1/J} + K_{1/J}) (M + K)^{-1}, Eq. weight adj inv."""
    one = np.ones_like(Je)
    MK = dense_fr_mass(one, ops)
    MK_invJ = dense_fr_mass(1.0 / Je, ops)
    MKi = np.linalg.inv(MK)
    return MKi @ MK_invJ @ MKi
