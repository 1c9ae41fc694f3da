"""Pins of the oracle's metric terms: affine exactness, exact cofactors, GCL, watertightness."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import geometry
from oracle.operators1d import Ops1D, apply_1d


def _geo(ctrl, shape, p, p_geo=None):
    ops = Ops1D(p)
    mesh = geometry.StructuredMesh(*shape)
    geo = geometry.metric_terms(ctrl, p if p_geo is None else p_geo, ops)
    return ops, mesh, geo


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_affine_mesh_exact(p):
    shape = (3, 2, 4)
    ctrl = wl.control_points(*shape, p, [0, -1, 2], [3, 1, 6])
    ops, mesh, geo = _geo(ctrl, shape, p)
    hx, hy, hz = 1.0, 1.0, 1.0
    Cexp = np.diag([hy * hz / 4, hx * hz / 4, hx * hy / 4])
    # round-off scale: |X| (up to 6) times the LGL differentiation norm (~n^2)
    tol = 1e-15 * 6 * (p + 1) ** 2
    for d in range(3):
        for c in range(3):
            assert np.allclose(geo["C"][d, c], Cexp[d, c], atol=tol)
            assert np.allclose(geo["Cf"][d, c], Cexp[d, c], atol=tol)
    assert np.allclose(geo["J"], hx * hy * hz / 8, atol=1e-14)
    # GL node coordinates of element (1, 1, 2)
    e = 1 + 3 * (1 + 2 * 2)
    xi = ops.xi
    x = geo["xyz"][0, e]
    assert np.allclose(x[0, 0, :], 0 + 1 + (xi + 1) / 2, atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_trilinear_map_gives_exact_cofactors(p):
    """For a trilinear map the products X_l d_k X_m have degree <= 2, so for p >= 2
    the conservative-curl metric equals the exact cofactor a_j x a_k at every node."""
    rng = np.random.default_rng(3)
    verts = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], float)
    verts = verts * [1.5, 1.0, 0.8] + 0.15 * rng.standard_normal((8, 3))
    ctrl = verts[None]  # one element, p_geo = 1, xi fastest
    ops, mesh, geo = _geo(ctrl, (1, 1, 1), p, p_geo=1)
    xi = ops.xi
    Z, Y, X = np.meshgrid(xi, xi, xi, indexing="ij")
    s = [(1 - X) / 2, (1 + X) / 2]
    t = [(1 - Y) / 2, (1 + Y) / 2]
    r = [(1 - Z) / 2, (1 + Z) / 2]
    ds = [-0.5 * np.ones_like(X), 0.5 * np.ones_like(X)]
    a = [np.zeros((3,) + X.shape) for _ in range(3)]
    for k in (0, 1):
        for j in (0, 1):
            for i in (0, 1):
                v = verts[i + 2 * j + 4 * k][:, None, None, None]
                a[0] += v * ds[i] * t[j] * r[k]
                a[1] += v * s[i] * ds[j] * r[k]
                a[2] += v * s[i] * t[j] * ds[k]
    exact = [np.cross(a[1], a[2], axis=0), np.cross(a[2], a[0], axis=0), np.cross(a[0], a[1], axis=0)]
    for d in range(3):
        assert np.allclose(geo["C"][d, :, 0], exact[d], atol=1e-14)
    J = np.sum(a[0] * exact[0], axis=0)
    assert np.allclose(geo["J"][0], J, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("warp", ["tgv", "paper"])
def test_gcl_watertight_consistent(p, warp):
    shape = (3, 2, 2)
    if warp == "paper":
        ctrl = wl.control_points(*shape, p, 0.0, 2 * math.pi, wl.make_warp_paper(0.2, 0.0, 2 * math.pi))
    else:
        ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    ops, mesh, geo = _geo(ctrl, shape, p)
    C, Cf, Cfm = geo["C"], geo["Cf"], geo["Cf_m"]
    scale = np.abs(C).max()
    # discrete GCL at GL nodes: sum_i D_i (J a^i)_n = 0
    for c in range(3):
        gcl = sum(apply_1d(ops.D, C[i, c], i) for i in range(3))
        assert np.abs(gcl).max() < 2e-13 * scale
    # the volume metric extrapolated along lines gives the face rows
    for d in range(3):
        for s, face in ((1, Cf), (0, Cfm)):
            ext = np.take(apply_1d(ops.t(s)[None, :], C[d], d), 0, axis=C[d].ndim - 1 - d)
            assert np.abs(ext - face[d]).max() < 2e-13 * scale
    # watertight: own +face row equals the +neighbour's own -face row (periodic seam included)
    for d in range(3):
        nb = mesh.neighbor(d, 1)
        assert np.abs(Cf[d] - Cfm[d][:, nb]).max() < 1e-13 * scale
    # closed surface: sum over faces of s w_f (J a^d) = 0 per element
    wf = np.outer(ops.w, ops.w)
    tot = sum(np.sum(wf * (Cf[d] - Cfm[d]), axis=(-1, -2)) for d in range(3))
    assert np.abs(tot).max() < 1e-13 * scale
    assert geo["J"].min() > 0


def test_node_coordinates_reproduce_a_polynomial_map():
    """A map of degree <= p_geo per direction is reproduced exactly at the GL nodes."""
    p, pg = 4, 3

    def warp(X, Y, Z):
        return (X + 0.05 * X ** 2 * Y - 0.02 * Z ** 3, Y + 0.03 * X * Y * Z, Z + 0.04 * Y ** 3 - 0.01 * X * Z)

    ctrl = wl.control_points(2, 1, 1, pg, [-1, 0, 0], [1, 1, 1], warp)
    ops, mesh, geo = _geo(ctrl, (2, 1, 1), p, p_geo=pg)
    xyz = geometry.node_coordinates_abi(geo)
    xi = ops.xi
    Z, Y, Xg = np.meshgrid(xi, xi, xi, indexing="ij")
    for e, x0 in ((0, -1.0), (1, 0.0)):
        X = x0 + (Xg.ravel() + 1) / 2
        Yv = (Y.ravel() + 1) / 2
        Zv = (Z.ravel() + 1) / 2
        expect = np.stack(warp(X, Yv, Zv))
        assert np.abs(xyz[e] - expect).max() < 1e-14
