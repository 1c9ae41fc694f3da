"""Uncollocated NSFR: solution on LGL nodes, volume and face quadrature on GL nodes.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): the plain FP64 statement
of the paper's own setting, in which the solution's coefficients live on the
p+1 Lobatto (LGL) nodes and the volume and face integrals use N_q >= p+1
Gauss-Legendre (GL) points per direction, N_q > p+1 being the paper's
"overintegration" (Sec. "Results": integration on GL nodes, overintegration
N_q = (p+1) + k).  With n = p+1:

  chi  (N_q x n)  the LGL Lagrange basis at the GL points; W their weights;
  M1 = chi^T W chi (the exact 1D mass), Pi = M1^{-1} chi^T W (the L2
  projection onto the solution space, Pi chi = I);
  entropy projection (Sec. "Nonlinearly Stable Flux Reconstruction", entropy
  projected variables): v~^ = Pi v(chi u^), then u~ = u(chi v~^) at the GL
  volume points and u~_f = u(l_f v~^) at the GL face points;
  flux differencing on the GL points with the hybridised SBP operator of
  D_q = chi D Pi: S_q = W D_q - D_q^T W, face extrapolations
  E_-+ = l(-+1)^T Pi (W D_q + D_q^T W = E+^T E+ - E-^T E- because the
  quadrature integrates degree 2p exactly), i.e. the same line-wise form as
  the collocated scheme on the GL points, applied to u~;
  residual on the solution space R^ = chi^T R_q (chi^T E^T = l^T since
  Pi chi = I, so the face rows are tested with the solution's face values);
  mass: (M_m + K_m)^{-1} ~ Pi~ (W J)^{-1} Pi~^T, Pi~1 = (M1 + K1)^{-1} chi^T W,
  K1 = c (D^p)^T M1 D^p (Eq. Km in 1D, Eq. Fr projection, Eq. weight-adj ESFR
  mass).
With N_q = p+1, chi is square and the scheme is the GL-collocated one written
in the LGL basis (pinned in the tests).
"""
from __future__ import annotations

import types

import numpy as np

from . import diagnostics, geometry, physics, quadrature, residual, timestep
from .operators1d import apply_1d, lagrange_deriv, lagrange_eval


def tensor3(A, X):
    """A along all three directions (A may be rectangular)."""
    return apply_1d(A, apply_1d(A, apply_1d(A, X, 0), 1), 2)


class UncollocatedProblem:
    """One structured periodic mesh; solution degree p on LGL nodes, N_q GL points."""

    def __init__(self, ctrl, shape, p, nq=None, p_geo=None, c=0.0, gamma=1.4, face_flux="ec",
                 vol_flux="chandrashekar"):
        n = p + 1
        nq = n if nq is None else nq
        if nq < n:
            raise ValueError("N_q >= p + 1 (the quadrature must integrate degree 2p)")
        self.p, self.n, self.nq = p, n, nq
        self.p_geo = p if p_geo is None else p_geo
        self.gamma, self.face_flux, self.c = gamma, face_flux, float(c)
        self.vol_flux = vol_flux
        xs, _ = quadrature.gauss_lobatto(n)
        xq, wq = quadrature.gauss_legendre(nq)
        self.xs, self.xq, self.wq = xs, xq, wq
        self.chi = lagrange_eval(xs, xq)                       # N_q x n
        W = np.diag(wq)
        self.M1 = self.chi.T @ W @ self.chi
        self.Pi = np.linalg.solve(self.M1, self.chi.T @ W)     # n x N_q
        self.D = lagrange_deriv(xs, xs)
        Dq = self.chi @ self.D @ self.Pi
        lm = lagrange_eval(xs, -1.0)[0]
        lp = lagrange_eval(xs, 1.0)[0]
        Dp = np.linalg.matrix_power(self.D, p)
        self.K1 = self.c * (Dp.T @ self.M1 @ Dp)
        self.Pit = np.linalg.solve(self.M1 + self.K1, self.chi.T @ W)  # Pi~1, n x N_q
        # operators of the GL points, in the form the line-wise residual uses
        q = types.SimpleNamespace()
        q.n, q.p, q.w, q.W = nq, p, wq, W
        q.D = Dq
        q.S1 = W @ Dq - Dq.T @ W
        q.t_minus, q.t_plus = lm @ self.Pi, lp @ self.Pi
        q.t = lambda side: q.t_plus if side == 1 else q.t_minus
        self.qops = q
        # the metric construction: Lobatto layer of degree p, evaluated at the GL points
        g = types.SimpleNamespace()
        g.n, g.p, g.xi = n, p, xq
        g.xi_lgl, _ = quadrature.gauss_lobatto(n)
        g.D_lgl = lagrange_deriv(g.xi_lgl, g.xi_lgl)
        g.I_lgl_to_gl = lagrange_eval(g.xi_lgl, xq)
        self.mesh = geometry.StructuredMesh(*shape)
        self.geo = geometry.metric_terms(ctrl, self.p_geo, g)
        self.nf = geometry.shared_face_normals(self.geo, self.mesh)
        self.C, self.J = self.geo["C"], self.geo["J"]       # at the GL points
        self.solution_coords_ops = types.SimpleNamespace(xi=xs)

    # layouts: the state is [N_e][5][n^3] coefficients at the LGL nodes (xi fastest)
    def to_internal(self, u):
        n, ne = self.n, np.asarray(u).shape[0]
        return np.ascontiguousarray(np.moveaxis(np.asarray(u).reshape(ne, 5, n, n, n), 1, 0))

    def to_abi(self, U):
        ne = U.shape[1]
        return np.ascontiguousarray(np.moveaxis(U, 0, 1).reshape(ne, 5, self.n ** 3))

    def node_coords(self, ctrl):
        """Physical coordinates of the LGL solution nodes [N_e][3][n^3] (for initial states)."""
        X = geometry.node_coordinates(ctrl, self.p_geo, self.solution_coords_ops)
        ne = X.shape[1]
        return np.ascontiguousarray(np.moveaxis(X, 0, 1).reshape(ne, 3, self.n ** 3))

    # the scheme -----------------------------------------------------------------
    def projected(self, U):
        """v~^ = Pi v(chi u^) and the projected state u~ = u(chi v~^) at the GL points."""
        Vh = tensor3(self.Pi, physics.entropy_variables(tensor3(self.chi, U), self.gamma))
        Uq = physics.conserved_from_entropy(tensor3(self.chi, Vh), self.gamma)
        return Vh, Uq

    def residual(self, U):
        """R^ = chi^T R_q; R_q the collocated line-wise residual of u~ on the GL points
        (its face states t . v(u~) equal l_f v~^ because Pi chi = I)."""
        _, Uq = self.projected(U)
        Rq = residual.residual(Uq, self.C, self.nf, self.mesh, self.qops, self.gamma, self.face_flux,
                               self.vol_flux)
        return tensor3(self.chi.T, Rq)

    def dudt(self, U):
        X = tensor3(self.Pit.T, self.residual(U))
        wq = self.wq
        X = X / (wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * self.J)
        return -tensor3(self.Pit, X)

    def rk4_step(self, U, dt):
        return timestep.rk4_step(U, dt, self.dudt)

    def entropy_rate(self, U):
        """-v~^ . R^ over the mesh and the scale sum |v~^ R^| (the projected entropy
        variables make the volume terms telescope, Sec. "Nonlinear Stability")."""
        Vh, _ = self.projected(U)
        R = self.residual(U)
        prod = Vh * R
        return -diagnostics.fsum(prod), diagnostics.fsum(np.abs(prod))

    def diagnostics(self, U):
        """The scheme's scalars with the solution at the GL points, u_q = chi u^, and the point
        weights W J: S = sum W J U(u_q), Q_k = sum W J (u_q)_k, KE = sum W J rho|u|^2/2 (the
        GL quadrature of the solution); the entropy rate -sum_i v~^_i . R^_i and its scale
        sum_i |v~^_i . R^_i| (per solution node); sum R^."""
        Uq = tensor3(self.chi, U)
        wq = self.wq
        wj = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * self.J
        rho, vel, _ = physics.primitive(Uq, self.gamma)
        Vh, _ = self.projected(U)
        R = self.residual(U)
        vr = np.sum(Vh * R, axis=0)  # v~^_i . R^_i per solution node, as the collocated diagnostics
        rate, scale = -diagnostics.fsum(vr), diagnostics.fsum(np.abs(vr))
        return {"entropy": diagnostics.fsum(wj * physics.entropy_function(Uq, self.gamma)),
                "entropy_rate": rate, "entropy_rate_scale": scale,
                "Q": [diagnostics.fsum(wj * Uq[k]) for k in range(5)],
                "kinetic_energy": diagnostics.fsum(wj * 0.5 * rho * np.sum(vel * vel, axis=0)),
                "sum_R": [diagnostics.fsum(R[k]) for k in range(5)]}

    # ABI conveniences
    def dudt_abi(self, u):
        return self.to_abi(self.dudt(self.to_internal(u)))

    def residual_abi(self, u):
        return self.to_abi(self.residual(self.to_internal(u)))

    def rk4_step_abi(self, u, dt):
        return self.to_abi(self.rk4_step(self.to_internal(u), dt))
