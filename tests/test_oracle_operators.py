"""Pins of the oracle's quadrature and 1D operators (closed forms, library routines, identities)."""
import math

import numpy as np
import pytest

from oracle import mass, quadrature
from oracle.operators1d import Ops1D, c_hu, lagrange_deriv, lagrange_eval, pth_derivative_coeffs


@pytest.mark.parametrize("n", range(1, 10))
def test_gl_matches_numpy_leggauss(n):
    x, w = quadrature.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=2e-15, rtol=0)
    assert np.allclose(w, wr, atol=2e-15, rtol=0)


def test_gl_lgl_closed_forms():
    x, w = quadrature.gauss_legendre(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-16)
    x, w = quadrature.gauss_legendre(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-16)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-16)
    x, w = quadrature.gauss_lobatto(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-16)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-16)
    x, w = quadrature.gauss_lobatto(4)
    assert np.allclose(x, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-16)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-16)


@pytest.mark.parametrize("n", range(2, 10))
def test_quadrature_exactness(n):
    x, w = quadrature.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 5e-15
    xl, wl = quadrature.gauss_lobatto(n)
    for k in range(2 * n - 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(wl, xl ** k) - exact) < 5e-15
    # one degree beyond: not exact (checks the rules are not over-claimed)
    assert abs(np.dot(w, x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6
    # LGL interior nodes are the roots of P'_{n-1}
    dP = np.polynomial.legendre.legder([0] * (n - 1) + [1])
    assert np.allclose(np.polynomial.legendre.legval(xl[1:-1], dP), 0, atol=1e-13)


@pytest.mark.parametrize("p", range(1, 8))
def test_lagrange_operators_exact_on_polynomials(p):
    ops = Ops1D(p)
    xi = ops.xi
    for k in range(p + 1):
        f = xi ** k
        df = k * xi ** (k - 1) if k else np.zeros_like(xi)
        assert np.allclose(ops.D @ f, df, atol=1e-12)
        assert abs(ops.t_plus @ f - 1.0) < 1e-13
        assert abs(ops.t_minus @ f - (-1.0) ** k) < 1e-13
    # an independent route to the same matrix: numpy polynomial fit derivative
    V = np.vander(xi, p + 1, increasing=True)
    dV = np.zeros_like(V)
    for k in range(1, p + 1):
        dV[:, k] = k * xi ** (k - 1)
    assert np.allclose(ops.D, dV @ np.linalg.inv(V), atol=1e-10)


@pytest.mark.parametrize("p", range(1, 8))
def test_sbp_property(p):
    """W D + D^T W = t+ t+^T - t- t-^T (SBP, Eq. SBP in 1D); S1 skew."""
    ops = Ops1D(p)
    lhs = ops.W @ ops.D + ops.D.T @ ops.W
    rhs = np.outer(ops.t_plus, ops.t_plus) - np.outer(ops.t_minus, ops.t_minus)
    assert np.allclose(lhs, rhs, atol=1e-13)
    assert np.allclose(ops.S1, -ops.S1.T, atol=0)


@pytest.mark.parametrize("p", range(1, 8))
def test_esfr_operator_and_projection(p):
    c = 0.37 * 10.0 ** (-p)
    ops = Ops1D(p, c)
    g = pth_derivative_coeffs(ops.xi)
    # D^p has identical rows g^T (p-th derivative of a degree-p interpolant)
    assert np.allclose(ops.Dp, np.tile(g, (ops.n, 1)), rtol=1e-9, atol=1e-9 * np.abs(g).max())
    # K1 = c (D^p)^T W D^p = 2 c g g^T
    assert np.allclose(ops.K1, 2 * c * np.outer(g, g), rtol=1e-8, atol=1e-12 * c * np.abs(g).max() ** 2)
    # Pi~1 = (W + K1)^{-1} W by Sherman-Morrison
    winv = 1.0 / ops.w
    sm = np.eye(ops.n) - 2 * c * np.outer(winv * g, g) / (1 + 2 * c * np.dot(g, winv * g))
    assert np.allclose(ops.Pi1, sm, atol=1e-12)
    assert np.allclose(ops.Pi1 @ np.ones(ops.n), 1.0, atol=1e-13)
    assert np.allclose(Ops1D(p, 0.0).Pi1, np.eye(ops.n), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_3d_fr_mass_is_tensor_product(p):
    """Eq. Km with J=1 and c_(s,v,w) = c^{#nonzero} equals (M1+K1)^{(x)3}."""
    ops = Ops1D(p, 0.05)
    dense = mass.dense_fr_mass(np.ones(ops.n ** 3), ops)
    A = ops.M1 + ops.K1
    assert np.allclose(dense, np.kron(A, np.kron(A, A)), atol=1e-12)


@pytest.mark.parametrize("p", range(1, 8))
def test_c_hu_lumps_the_mass_matrix(p):
    """M_GL + c_HU K equals the Lobatto-integrated mass matrix on P_p."""
    c = c_hu(p)
    assert c > 0
    n = p + 1
    xi, w = quadrature.gauss_legendre(n)
    xl, wl = quadrature.gauss_lobatto(n)
    L = lagrange_eval(xi, xl)
    ops = Ops1D(p, c)
    assert np.allclose(ops.M1 + ops.K1, L.T @ np.diag(wl) @ L, atol=1e-12)


def test_lagrange_deriv_offgrid():
    nodes = quadrature.gauss_lobatto(5)[0]
    x = np.linspace(-1, 1, 7)
    f = lambda t: 3 * t ** 4 - t ** 3 + 2 * t - 1
    df = lambda t: 12 * t ** 3 - 3 * t ** 2 + 2
    assert np.allclose(lagrange_deriv(nodes, x) @ f(nodes), df(x), atol=1e-12)
    assert np.allclose(lagrange_eval(nodes, x) @ f(nodes), f(x), atol=1e-13)
