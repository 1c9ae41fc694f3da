"""Metric terms of curvilinear hexahedra in conservative-curl form.

Paper: mapping x = sum_i Theta_i(xi) x_i (Sec. "Computational Space"),
J = a_1 . (a_2 x a_3), C^T = J (J^Omega)^{-1} with rows J a^i, built in
Kopriva's conservative-curl form so that the discrete GCL (Eq. GCL)
sum_i d/dxi^i (C)_{ni} = 0 holds; face normals n^ = C . n^r / J^Gamma
(Eq. normals def) must be watertight for free-stream preservation.

Construction (the readings listed in the design notes):
  1. the degree-p_geo map, given by control points at equispaced reference
     nodes, is evaluated at the degree-q = p Lobatto (LGL) nodes;
  2. d_k X_m there is the exact derivative of the map (LGL differentiation is
     exact for degree <= q);
  3. (J a^i)_n = -[curl_xi (X_l grad_xi X_m)]_i, (n, m, l) cyclic, where the
     products X_l d_k X_m are interpolated on the LGL nodes and the curl is
     the exact derivative of that interpolant; X_l is taken relative to the
     element's first control point: curl(c grad X_m) = 0 for a constant c
     (the discrete derivatives along different directions commute), so the
     shift changes only rounding, which would otherwise grow like |X|/h;
  4. the resulting degree-<=q polynomials are interpolated to the GL volume
     nodes; face values are the LGL face layer interpolated tangentially to
     the face GL nodes;
  5. J at GL nodes is a_1 . (a_2 x a_3) of the map's exact derivative.
One normal per face is shared by both neighbours: the one computed in the
element on the face's minus side (the face is that element's xi_d = +1 face).
"""
from __future__ import annotations

import numpy as np

from . import quadrature
from .operators1d import apply_1d, lagrange_eval


class StructuredMesh:
    """Periodic nx x ny x nz block of elements, e = ex + nx*(ey + ny*ez)."""

    def __init__(self, nx, ny, nz):
        self.shape = (nx, ny, nz)
        self.n_el = nx * ny * nz
        e = np.arange(self.n_el)
        self.ex = e % nx
        self.ey = (e // nx) % ny
        self.ez = e // (nx * ny)

    def neighbor(self, d, side):
        """Index array of the neighbour across face (d, side): side 0 is xi_d=-1."""
        nx, ny, nz = self.shape
        step = 1 if side == 1 else -1
        ex, ey, ez = self.ex.copy(), self.ey.copy(), self.ez.copy()
        if d == 0:
            ex = (ex + step) % nx
        elif d == 1:
            ey = (ey + step) % ny
        else:
            ez = (ez + step) % nz
        return ex + nx * (ey + ny * ez)


def _to_nodal(ctrl, q):
    """[N_e][q^3][3] -> (3, N_e, q, q, q) with axes (zeta, eta, xi)."""
    ne = ctrl.shape[0]
    X = ctrl.reshape(ne, q, q, q, 3)
    return np.moveaxis(X, -1, 0)


def metric_terms(ctrl, p_geo, ops, dtype=None):
    """Metric data of every element.

    ``ctrl``: control points [N_e][(p_geo+1)^3][3] (real or complex).
    Returns a dict with
      C     (3, 3, N_e, n, n, n)  C[d, c] = (J a^d)_c at GL volume nodes
      J     (N_e, n, n, n)        Jacobian determinant at GL nodes
      Cf    (3, 3, N_e, n, n)     own xi_d=+1 face row (J a^d) at face GL nodes
      Cf_m  (3, 3, N_e, n, n)     own xi_d=-1 face row (J a^d), before sharing
      xyz   (3, N_e, n, n, n)     physical coordinates of the GL nodes
      C_lgl (3, 3, N_e, n, n, n)  the metric on the LGL construction nodes
    """
    n = ops.n
    q = p_geo + 1
    if p_geo > ops.p:
        raise ValueError("p_geo must not exceed p")
    X_eq = _to_nodal(np.asarray(ctrl), q)
    # 1. the map at the LGL nodes of degree p (exact: p_geo <= p)
    E = lagrange_eval(quadrature.equispaced(q), ops.xi_lgl)
    X = X_eq
    for d in range(3):
        X = apply_1d(E, X, d)
    # 2. exact derivatives on LGL nodes: dX[k][m] = d X_m / d xi^k
    Dl = ops.D_lgl
    dX = [[apply_1d(Dl, X[m], k) for m in range(3)] for k in range(3)]
    # 3. conservative curl, coordinates relative to the first control point
    Xr = X - X_eq[(slice(None), slice(None), 0, 0, 0)][..., None, None, None]
    Cl = [[None] * 3 for _ in range(3)]
    for nn in range(3):
        m = (nn + 1) % 3
        l = (nn + 2) % 3
        V = [Xr[l] * dX[k][m] for k in range(3)]  # V_k = (X_l - c_l) d_k X_m
        curl = [
            apply_1d(Dl, V[2], 1) - apply_1d(Dl, V[1], 2),  # d_eta V_3 - d_zeta V_2
            apply_1d(Dl, V[0], 2) - apply_1d(Dl, V[2], 0),  # d_zeta V_1 - d_xi V_3
            apply_1d(Dl, V[1], 0) - apply_1d(Dl, V[0], 1),  # d_xi V_2 - d_eta V_1
        ]
        for i in range(3):
            Cl[i][nn] = -curl[i]
    C_lgl = np.stack([np.stack(row) for row in Cl])
    # 4. to GL volume nodes
    I = ops.I_lgl_to_gl
    C = C_lgl
    for d in range(3):
        C = apply_1d(I, C, d)
    # face rows: LGL layer xi_d = +-1 of (J a^d), interpolated tangentially
    Cf = []
    Cf_m = []
    for d in range(3):
        ax = C_lgl[d].ndim - 1 - d
        plus = np.take(C_lgl[d], n - 1, axis=ax)   # (3, N_e, n, n)
        minus = np.take(C_lgl[d], 0, axis=ax)
        for dd in range(2):  # the two remaining directions, as last two axes
            plus = apply_1d(I, plus, dd)
            minus = apply_1d(I, minus, dd)
        Cf.append(plus)
        Cf_m.append(minus)
    Cf = np.stack(Cf)
    Cf_m = np.stack(Cf_m)
    # 5. Jacobian from the map's exact derivative at GL nodes
    a = [np.stack([dX[k][m] for m in range(3)]) for k in range(3)]  # a_k on LGL
    a_gl = []
    for k in range(3):
        ak = a[k]
        for d in range(3):
            ak = apply_1d(I, ak, d)
        a_gl.append(ak)
    J = (a_gl[0][0] * (a_gl[1][1] * a_gl[2][2] - a_gl[1][2] * a_gl[2][1])
         - a_gl[0][1] * (a_gl[1][0] * a_gl[2][2] - a_gl[1][2] * a_gl[2][0])
         + a_gl[0][2] * (a_gl[1][0] * a_gl[2][1] - a_gl[1][1] * a_gl[2][0]))
    # physical coordinates of GL nodes
    Eg = lagrange_eval(quadrature.equispaced(q), ops.xi)
    xyz = X_eq
    for d in range(3):
        xyz = apply_1d(Eg, xyz, d)
    return {"C": C, "J": J, "Cf": Cf, "Cf_m": Cf_m, "xyz": xyz, "C_lgl": C_lgl,
            "a_gl": a_gl}


def node_coordinates(ctrl, p_geo, ops):
    """Physical coordinates of the GL nodes only, (3, N_e, n, n, n): the map
    evaluated at the GL nodes (step 1 of ``metric_terms`` without the metric)."""
    q = p_geo + 1
    X = _to_nodal(np.asarray(ctrl), q)
    Eg = lagrange_eval(quadrature.equispaced(q), ops.xi)
    for d in range(3):
        X = apply_1d(Eg, X, d)
    return X


def shared_face_normals(geo, mesh):
    """Face rows used by both sides of every face (the minus-side element's).

    Returns nf with shape (3 [d], 2 [side], 3 [comp], N_e, n, n): for element e
    the row on its xi_d=+1 face is its own, the row on its xi_d=-1 face is the
    +1 face row of its minus-side neighbour.
    """
    Cf = geo["Cf"]
    out = []
    for d in range(3):
        nb = mesh.neighbor(d, 0)
        minus = Cf[d][:, nb]
        plus = Cf[d]
        out.append(np.stack([minus, plus]))
    return np.stack(out)


def node_coordinates_abi(geo):
    """Physical GL node coordinates in the ABI layout [N_e][3][n^3]."""
    xyz = geo["xyz"]
    ne = xyz.shape[1]
    n = xyz.shape[-1]
    return np.ascontiguousarray(np.moveaxis(xyz, 0, 1).reshape(ne, 3, n ** 3))
