"""Time integration: classic four-stage, fourth-order Runge-Kutta.

The paper advances every test with a 4-stage 4th-order RK scheme and an
adaptive step from the maximum wave speed at CFL 0.1 (Sec. "Results").  The
step is dt = CFL dx / max_i(|u_i| + a_i), dx = L/(N (p+1)), the average node
spacing (the paper's dx for its manufactured-solution test).
"""
from __future__ import annotations

import numpy as np

from . import physics


def rk4_step(U, dt, rhs):
    k1 = rhs(U)
    k2 = rhs(U + 0.5 * dt * k1)
    k3 = rhs(U + 0.5 * dt * k2)
    k4 = rhs(U + dt * k3)
    return U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def cfl_dt(U, cfl, dx, gamma):
    lam = physics.max_wavespeed(U, gamma)
    return cfl * dx / float(np.max(np.real(lam)))
