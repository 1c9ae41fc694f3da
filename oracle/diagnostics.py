"""Scalar diagnostics of the semi-discrete and fully discrete scheme.

* entropy rate: v^ (M_m + K_m) du/dt = -sum_m sum_i v(u_i) . R_i
  (Sec. "Nonlinear Stability"; collocation makes v^ the nodal v(u)); the
  paper checks it to O(1e-13) on the Taylor-Green vortex.
* conservation: 1^ (M_m + K_m) du/dt = -sum of face fluxes, which cancel on a
  periodic mesh (Sec. "Global Conservation"), so sum_m sum_i R_i = 0 per
  variable; with the weight-adjusted inverse the conserved functional is
  Q = sum_m (W J)^T Pi~^{-1} u, Pi~1^{-1} = I + W^{-1} K1.
* entropy S = sum W J U(u), kinetic energy KE = sum W J rho|u|^2/2.
All sums use math.fsum (exactly rounded).
"""
from __future__ import annotations

import math

import numpy as np

from . import physics
from .mass import w3
from .operators1d import tensor3


def fsum(x):
    return math.fsum(np.ravel(np.real(x)))


def entropy_rate(U, R, gamma):
    """(-sum v.R, sum |v_i . R_i|): the semi-discrete entropy rate and its scale."""
    V = physics.entropy_variables(U, gamma)
    vr = np.sum(V * R, axis=0)
    return -fsum(vr), fsum(np.abs(vr))


def residual_totals(R):
    """Per-variable sum of R and sum of |R|."""
    return [fsum(R[k]) for k in range(5)], [fsum(np.abs(R[k])) for k in range(5)]


def conserved_totals(U, J, ops):
    """Q_var = sum_m (W J)^T (Pi~^{-1} u)_var."""
    Pinv1 = np.eye(ops.n) + np.diag(1.0 / ops.w) @ ops.K1
    X = tensor3(Pinv1, U)
    wj = w3(ops) * J
    return [fsum(wj * X[k]) for k in range(5)], [fsum(np.abs(wj * X[k])) for k in range(5)]


def entropy_total(U, J, ops, gamma):
    return fsum(w3(ops) * J * physics.entropy_function(U, gamma))


def kinetic_energy(U, J, ops):
    rho = U[0]
    ke = 0.5 * np.sum(U[1:4] * U[1:4], axis=0) / rho
    return fsum(w3(ops) * J * ke)


def kinetic_energy_c(U, J, ops):
    """Kinetic energy without rounding to float (complex-step safe)."""
    rho = U[0]
    ke = 0.5 * np.sum(U[1:4] * U[1:4], axis=0) / rho
    return np.sum(w3(ops) * J * ke)


def l2_error(U, U_exact, J, ops, var=0):
    """sqrt(sum_m (u - u_ex)^T W J (u - u_ex)) for one variable (Eq. L2-error)."""
    e = U[var] - U_exact[var]
    return math.sqrt(fsum(w3(ops) * J * e * e))
