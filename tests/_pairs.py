"""Helpers that set up the same seeded problem for the CUDA library and the oracle."""
import math

import numpy as np

import workloads as wl
from oracle.operators1d import c_hu
from oracle.problem import Problem


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over all entries (all five variables together)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_ctrl(shape, p, kind="tgv", p_geo=None):
    pg = p if p_geo is None else p_geo
    if kind == "tgv":
        return wl.control_points(*shape, pg, -math.pi, math.pi, wl.warp_tgv)
    if kind == "unit":
        return wl.control_points(*shape, pg, 0.0, 1.0, wl.warp_unit)
    if kind == "paper":
        return wl.control_points(*shape, pg, 0.0, 2 * math.pi, wl.make_warp_paper(0.2, 0.0, 2 * math.pi))
    if kind == "affine":
        return wl.control_points(*shape, pg, -math.pi, math.pi)
    raise ValueError(kind)


def c_value(p, c_kind):
    return 0.0 if c_kind == "dg" else c_hu(p)


def oracle_problem(shape, p, c_kind="dg", face_flux="ec", kind="tgv", p_geo=None, nodes="gl"):
    ctrl = make_ctrl(shape, p, kind, p_geo)
    P = Problem(ctrl, shape, p, p_geo=p_geo, c=c_value(p, c_kind), face_flux=face_flux, nodes=nodes)
    return ctrl, P


def state_for(P, kind="tgv", seed=wl.PARITY_SEED):
    xyz = P.node_coords()
    if kind in ("tgv", "paper", "affine"):
        return np.ascontiguousarray(wl.perturbed_tgv_state(xyz, seed))
    return np.ascontiguousarray(wl.perturbed_density_wave_state(xyz, seed))


def oracle_metrics_abi(P):
    """The oracle's metric terms in the library's layouts (C, J, Cf)."""
    ne, n = P.mesh.n_el, P.n
    C = np.ascontiguousarray(np.moveaxis(P.C.reshape(3, 3, ne, n ** 3), 2, 0).reshape(ne, 9, n ** 3))
    J = np.ascontiguousarray(P.J.reshape(ne, n ** 3))
    Cf = np.ascontiguousarray(np.moveaxis(P.geo["Cf"].reshape(3, 3, ne, n * n), 2, 0))
    return C, J, Cf
