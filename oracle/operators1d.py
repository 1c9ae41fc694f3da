"""One-dimensional reference operators (collocated Lagrange basis).

* Lagrange basis and derivative on arbitrary node sets, by the product formula.
* The solution and volume quadrature nodes are one set: Gauss-Legendre (GL,
  the default) or Gauss-Lobatto-Legendre (LGL, the paper's kinetic-energy
  preserving case: the face nodes are then a subset of the volume nodes,
  Sec. "Nonlinear Stability", kinetic energy lemma).
* SBP pieces on those nodes: W = diag(w), D_ij = l_j'(xi_i), extrapolations
  t_-[j] = l_j(-1), t_+[j] = l_j(+1), skew operator S1 = W D - D^T W
  (Sec. "Computational Space", SBP property Eq. SBP).
* ESFR: K1 = c (D^p)^T W D^p is the 1D form of Eq. Km with J = 1
  (D^p = (M^{-1} S)^p, M = W for the collocated basis), and the 1D FR
  projection Pi~1 = (M1 + K1)^{-1} chi^T W = (W + K1)^{-1} W (Eq. Fr projection,
  chi = I when solution nodes = quadrature nodes).
"""
from __future__ import annotations

import math

import numpy as np

from . import quadrature


def lagrange_eval(nodes, x):
    """L[k, j] = l_j(x_k) for the Lagrange basis on ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    L = np.ones((x.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv(nodes, x):
    """Dm[k, j] = l_j'(x_k), from l_j' = sum_m 1/(x_j-x_m) prod_{l != j,m} (x-x_l)/(x_j-x_l)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    Dm = np.zeros((x.size, n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(x.size, 1.0 / (nodes[j] - nodes[m]))
            for l in range(n):
                if l != j and l != m:
                    term = term * (x - nodes[l]) / (nodes[j] - nodes[l])
            Dm[:, j] += term
    return Dm


def pth_derivative_coeffs(nodes):
    """g_j = d^p l_j / dxi^p = p! / prod_{k != j}(xi_j - xi_k), p = len(nodes)-1."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = nodes.size
    g = np.empty(n)
    for j in range(n):
        den = 1.0
        for k in range(n):
            if k != j:
                den *= nodes[j] - nodes[k]
        g[j] = math.factorial(n - 1) / den
    return g


class Ops1D:
    """All 1D operators for solution degree p, ESFR parameter c and node set
    ``nodes`` ("gl" or "lgl")."""

    def __init__(self, p, c=0.0, nodes="gl"):
        self.p = p
        self.n = n = p + 1
        self.c = float(c)
        self.nodes = nodes
        if nodes == "gl":
            self.xi, self.w = quadrature.gauss_legendre(n)
        elif nodes == "lgl":
            self.xi, self.w = quadrature.gauss_lobatto(n)
        else:
            raise ValueError(f"unknown node set {nodes!r}")
        self.W = np.diag(self.w)
        self.D = lagrange_deriv(self.xi, self.xi)
        self.t_minus = lagrange_eval(self.xi, -1.0)[0]
        self.t_plus = lagrange_eval(self.xi, 1.0)[0]
        self.S1 = self.W @ self.D - self.D.T @ self.W
        # ESFR correction operator, Eq. Km in 1D with J = 1
        Dp = np.linalg.matrix_power(self.D, p)
        self.Dp = Dp
        self.K1 = self.c * (Dp.T @ self.W @ Dp)
        self.M1 = self.W.copy()
        # ESFR projection, Eq. Fr projection with chi = I
        self.Pi1 = np.linalg.solve(self.M1 + self.K1, self.W)
        # Lobatto nodes of the same degree carry the metric construction
        self.xi_lgl, self.w_lgl = quadrature.gauss_lobatto(n)
        self.D_lgl = lagrange_deriv(self.xi_lgl, self.xi_lgl)
        self.I_lgl_to_gl = lagrange_eval(self.xi_lgl, self.xi)

    def t(self, side):
        """Extrapolation row to the face at xi = -1 (side 0) or +1 (side 1)."""
        return self.t_plus if side == 1 else self.t_minus


def apply_1d(A, X, d):
    """Apply the matrix A (m x n) along reference direction d of X[..., z, y, x].

    d = 0 acts on the last axis (xi), d = 1 on eta, d = 2 on zeta.
    """
    ax = X.ndim - 1 - d
    Y = np.tensordot(A, np.moveaxis(X, ax, 0), axes=(1, 0))
    return np.moveaxis(Y, 0, ax)


def tensor3(A, X):
    """Apply A along all three directions (sum factorisation, Eq. sum-factorization)."""
    return apply_1d(A, apply_1d(A, apply_1d(A, X, 0), 1), 2)


def c_hu(p):
    """ESFR parameter that turns the GL mass matrix into the Lobatto-lumped one.

    The paper describes c_HU by this property (Sec. "Maximum CFL"): on degree-p
    polynomials, M_GL + c K equals the mass matrix integrated with the
    (p+1)-point Lobatto rule.  Both sides are bilinear forms on P_p; their
    difference is rank one along the p-th derivative, so c follows from any
    pair of basis functions with nonzero p-th derivatives.  Evaluated here
    on the GL Lagrange basis.
    """
    n = p + 1
    xi, w = quadrature.gauss_legendre(n)
    xl, wl = quadrature.gauss_lobatto(n)
    L = lagrange_eval(xi, xl)  # GL Lagrange basis at the Lobatto nodes
    M_lob = L.T @ np.diag(wl) @ L
    M_gl = np.diag(w)
    D = lagrange_deriv(xi, xi)
    Dp = np.linalg.matrix_power(D, p)
    K_unit = Dp.T @ np.diag(w) @ Dp
    diff = M_lob - M_gl
    i = int(np.argmax(np.abs(np.diag(K_unit))))
    return float(diff[i, i] / K_unit[i, i])
