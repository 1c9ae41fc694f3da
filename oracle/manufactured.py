"""The manufactured solution of Sec. "Manufactured Solution Convergence" and its source term.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``).  The paper takes
Gassner et al.'s manufactured solution of the Euler equations,

    rho = 2 + sin(theta) / 10,   u = v = w = 1,   rho e = rho^2,
    theta = pi (x + y + z - 2 t),

periodic with period 2 in x, y and z, and drives it with the source
q = du/dt + div F(u) of that solution.  The source is written out here from the
definition (no constant is taken from the printed table, whose c_3 is garbled):
with rho_t = -(pi/5) cos(theta), rho_x = rho_y = rho_z = (pi/10) cos(theta),
p = (gamma-1)(rho^2 - 3 rho / 2) and p_x = (gamma-1)(2 rho - 3/2) rho_x,

    q_rho  = rho_t + 3 rho_x                              = c1 cos(theta)
    q_mom  = rho_t + 3 rho_x + p_x                        = c2 cos(theta) + c3 sin(2 theta)
    q_E    = 2 rho (rho_t + 3 rho_x) + 3 p_x              = c4 cos(theta) + c5 sin(2 theta)

    c1 = pi/10,  c2 = pi (5 gamma - 3)/20,  c3 = pi (gamma - 1)/100,
    c4 = pi (15 gamma - 7)/20,  c5 = pi (3 gamma - 2)/100

(the same three momentum components, since u = v = w).  The tests pin these
against a numerical divergence of the exact flux and against the four
constants the paper prints legibly; c3 is read as pi (gamma - 1) / 100.

The source enters the semi-discrete system as a volume integral beside the
residual, (M_m + K_m) du/dt = -R + chi^T W J q, so with the weight-adjusted
inverse du/dt = -Pi~ (W J)^{-1} Pi~^T (R - W J q) (Eq. weight-adj ESFR mass);
the paper does not spell out how its source is discretised, this is the
standard DG/FR form.  The L2 error is the paper's
sqrt(sum_m (u_m - u_exact)^T W J_m (u_m - u_exact)) at the volume nodes.
"""
from __future__ import annotations

import math

import numpy as np

from . import mass, physics, timestep
from .problem import Problem


def source_constants(gamma):
    pi = math.pi
    return {"c1": pi / 10.0, "c2": pi * (5.0 * gamma - 3.0) / 20.0, "c3": pi * (gamma - 1.0) / 100.0,
            "c4": pi * (15.0 * gamma - 7.0) / 20.0, "c5": pi * (3.0 * gamma - 2.0) / 100.0}


def exact_state(X, t):
    """Conserved state (5, ...) of the manufactured solution at coordinates X (3, ...)."""
    th = math.pi * (X[0] + X[1] + X[2] - 2.0 * t)
    rho = 2.0 + 0.1 * np.sin(th)
    return np.stack([rho, rho, rho, rho, rho * rho])


def exact_primitive(X, t, gamma):
    """(rho, p) of the manufactured solution."""
    U = exact_state(X, t)
    rho = U[0]
    return rho, (gamma - 1.0) * (U[4] - 1.5 * rho)


def source(X, t, gamma):
    """q (5, ...) at coordinates X (3, ...), time t."""
    k = source_constants(gamma)
    th = math.pi * (X[0] + X[1] + X[2] - 2.0 * t)
    c, s2 = np.cos(th), np.sin(2.0 * th)
    qm = k["c2"] * c + k["c3"] * s2
    return np.stack([k["c1"] * c, qm, qm, qm, k["c4"] * c + k["c5"] * s2])


class ManufacturedProblem(Problem):
    """The collocated NSFR problem with the manufactured source; the mesh is any
    periodic mesh of [-1, 1]^3 (the solution's period is 2)."""

    def __init__(self, ctrl, shape, p, **kw):
        super().__init__(ctrl, shape, p, **kw)
        self.X = self.geo["xyz"]                      # (3, N_e, n, n, n) volume nodes
        self.WJ = mass.w3(self.ops) * self.J

    def dudt_t(self, U, t):
        """du/dt = -Pi~ (W J)^{-1} Pi~^T (R - W J q(t))."""
        q = source(self.X, t, self.gamma)
        return mass.dudt_from_residual(self.residual(U) - self.WJ * q, self.J, self.ops)

    def rk4_step_t(self, U, t, dt):
        """Classic RK4 with the stage times t, t + dt/2, t + dt/2, t + dt."""
        k1 = self.dudt_t(U, t)
        k2 = self.dudt_t(U + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = self.dudt_t(U + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = self.dudt_t(U + dt * k3, t + dt)
        return U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def initial(self, t=0.0):
        return exact_state(self.X, t)

    def l2_errors(self, U, t):
        """(density, pressure) L2 errors against the exact solution at time t."""
        rho_e, p_e = exact_primitive(self.X, t, self.gamma)
        rho, _, p = physics.primitive(U, self.gamma)
        return (math.sqrt(float(np.sum(self.WJ * (rho - rho_e) ** 2))),
                math.sqrt(float(np.sum(self.WJ * (p - p_e) ** 2))))

    def run(self, t_end, dt_of):
        """Integrate from the exact state at t = 0 to t_end; dt_of(U) gives the step
        (shortened to land on t_end)."""
        U, t = self.initial(0.0), 0.0
        while t < t_end - 1e-14:
            dt = min(dt_of(U), t_end - t)
            U = self.rk4_step_t(U, t, dt)
            t += dt
        return U, t

    def cfl_dt(self, U, cfl, dx):
        return timestep.cfl_dt(U, cfl, dx, self.gamma)
