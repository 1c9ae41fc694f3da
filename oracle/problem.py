"""Oracle driver: one structured periodic mesh, its operators and metrics.

Inputs use the library's ABI layouts (control points [N_e][(p_geo+1)^3][3],
state [N_e][5][n^3]); internally the oracle works on (5, N_e, n, n, n).
"""
from __future__ import annotations

import numpy as np

from . import diagnostics, geometry, mass, residual, timestep
from .operators1d import Ops1D


class Problem:
    def __init__(self, ctrl, shape, p, p_geo=None, c=0.0, gamma=1.4, face_flux="ec", nodes="gl",
                 vol_flux="chandrashekar"):
        self.p = p
        self.n = p + 1
        self.p_geo = p if p_geo is None else p_geo
        self.gamma = gamma
        self.face_flux = face_flux
        self.vol_flux = vol_flux
        self.ops = Ops1D(p, c, nodes)
        self.mesh = geometry.StructuredMesh(*shape)
        self.geo = geometry.metric_terms(ctrl, self.p_geo, self.ops)
        self.nf = geometry.shared_face_normals(self.geo, self.mesh)
        self.C = self.geo["C"]
        self.J = self.geo["J"]

    # layouts ---------------------------------------------------------------
    def to_internal(self, u):
        n = self.n
        u = np.asarray(u)
        ne = u.shape[0]
        return np.ascontiguousarray(np.moveaxis(u.reshape(ne, 5, n, n, n), 1, 0))

    def to_abi(self, U):
        ne = U.shape[1]
        return np.ascontiguousarray(np.moveaxis(U, 0, 1).reshape(ne, 5, self.n ** 3))

    def node_coords(self):
        return geometry.node_coordinates_abi(self.geo)

    # the scheme --------------------------------------------------------------
    def residual(self, U):
        return residual.residual(U, self.C, self.nf, self.mesh, self.ops, self.gamma, self.face_flux,
                                 self.vol_flux)

    def dense_residual(self, U):
        return residual.dense_residual(U, self.C, self.nf, self.mesh, self.ops, self.gamma,
                                       self.face_flux, self.vol_flux)

    def dudt(self, U):
        return mass.dudt_from_residual(self.residual(U), self.J, self.ops)

    def rk4_step(self, U, dt):
        return timestep.rk4_step(U, dt, self.dudt)

    def cfl_dt(self, U, cfl, dx):
        return timestep.cfl_dt(U, cfl, dx, self.gamma)

    # ABI-layout conveniences --------------------------------------------------
    def dudt_abi(self, u):
        return self.to_abi(self.dudt(self.to_internal(u)))

    def residual_abi(self, u):
        return self.to_abi(self.residual(self.to_internal(u)))

    def rk4_step_abi(self, u, dt):
        return self.to_abi(self.rk4_step(self.to_internal(u), dt))

    def diagnostics(self, U):
        R = self.residual(U)
        rate, scale = diagnostics.entropy_rate(U, R, self.gamma)
        Q, Qabs = diagnostics.conserved_totals(U, self.J, self.ops)
        return {
            "entropy": diagnostics.entropy_total(U, self.J, self.ops, self.gamma),
            "entropy_rate": rate,
            "entropy_rate_scale": scale,
            "Q": Q,
            "Q_abs": Qabs,
            "kinetic_energy": diagnostics.kinetic_energy(U, self.J, self.ops),
        }


def dx_of(lengths, shape, p):
    """Average node spacing min_d L_d/(N_d (p+1))."""
    return min(L / (N * (p + 1)) for L, N in zip(lengths, shape))
