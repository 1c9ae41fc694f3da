"""Pins of the oracle's manufactured solution (Sec. "Manufactured Solution Convergence").

* The closed-form source equals du/dt + div F(u) of the exact solution,
  differentiated numerically (complex step in x, y, z and t through the
  oracle's own Euler flux): a dropped term, a wrong sign or a wrong constant
  fails it.
* The constants the paper prints legibly (c1, c2, c4, c5 at gamma = 1.4,
  tests/golden) and the reading of the garbled c3.
* The semi-discrete operator with the source, at the exact solution, tends to
  the exact du/dt at order >= p on the warped mesh (the source's
  discretisation and sign).
* A run converges at about p + 1 (the paper's orders).
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle import manufactured as mm
from oracle import physics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mms_source_constants.json")


def _complex_step_divergence(X, t, gamma, h=1e-30):
    """du/dt + sum_d dF_d/dx_d of the exact solution by complex steps."""
    dU_dt = np.imag(mm.exact_state(X, t + 1j * h)) / h
    div = np.zeros_like(dU_dt)
    for d in range(3):
        Xc = X.astype(complex)
        Xc[d] = Xc[d] + 1j * h
        nvec = np.zeros((3,) + X.shape[1:])
        nvec[d] = 1.0
        F = physics.euler_flux(mm.exact_state(Xc, t), nvec, gamma)
        div += np.imag(F) / h
    return dU_dt + div


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0, 1.3])
def test_source_is_the_divergence_of_the_exact_flux(gamma):
    rng = np.random.default_rng(7)
    X = rng.uniform(-1.0, 1.0, (3, 200))
    for t in (0.0, 0.37, 1.9):
        q_num = _complex_step_divergence(X, t, gamma)
        q = mm.source(X, t, gamma)
        assert np.abs(q - q_num).max() < 1e-13 * np.abs(q_num).max()


def test_source_constants_match_the_printed_ones():
    g = json.load(open(GOLDEN))
    k = mm.source_constants(g["gamma"])
    for name in ("c1", "c2", "c4", "c5"):
        assert abs(k[name] - g[name]) < 1e-15 * abs(g[name])
    assert abs(k["c3"] - g["c3_reading"]) < 1e-15 * g["c3_reading"]


def test_exact_solution_is_periodic_and_pressure_positive():
    X = np.random.default_rng(3).uniform(-1.0, 1.0, (3, 50))
    for d in range(3):
        Y = X.copy()
        Y[d] += 2.0
        assert np.allclose(mm.exact_state(X, 0.3), mm.exact_state(Y, 0.3), atol=1e-14)
    rho, p = mm.exact_primitive(X, 0.3, 1.4)
    assert rho.min() >= 1.9 and p.min() > 0.3


def _truncation(n_el, p, c=0.0, face_flux="ec_roe", t=0.3, with_source=True):
    ctrl = wl.mms_mesh(n_el, p)
    P = mm.ManufacturedProblem(ctrl, (n_el,) * 3, p, c=c, face_flux=face_flux)
    Ue = mm.exact_state(P.X, t)
    h = 1e-30
    dUe = np.imag(mm.exact_state(P.X, t + 1j * h)) / h
    E = (P.dudt_t(Ue, t) if with_source else P.dudt(Ue)) - dUe
    return math.sqrt(float(np.sum(P.WJ * E * E)))


@pytest.mark.parametrize("p,c,face_flux,m", [(2, 0.0, "ec_roe", 4), (3, 1e-3, "ec", 2)])
def test_semi_discrete_operator_with_source_is_consistent(p, c, face_flux, m):
    """||du/dt(u_exact) - d u_exact/dt|| falls with h (observed rates 1.6-2.0 on these
    coarse warped meshes, p - 1 asserted); without the source it stays O(1) (about 5)."""
    e1 = _truncation(m, p, c, face_flux)
    e2 = _truncation(2 * m, p, c, face_flux)
    assert e2 < e1 / 2 ** (p - 1)
    assert _truncation(2 * m, p, c, face_flux, with_source=False) > 5 * e2


def test_run_converges_at_about_p_plus_one():
    """p = 2 to t = 0.5 on the affine periodic mesh: L2 errors of density and pressure
    fall at about p + 1 between 4^3 and 8^3 elements (observed 2.86 and 2.84; 2.5
    asserted).  On the paper's warped mesh (beta = 1/50, the warp's sin(5 pi y) has
    a wavelength of 0.4) these meshes are pre-asymptotic; its orders are measured on
    finer meshes with the library."""
    p, t_end = 2, 0.5
    errs = []
    for n_el in (4, 8):
        P = mm.ManufacturedProblem(wl.mms_mesh(n_el, p, warp="none"), (n_el,) * 3, p, face_flux="ec_roe")
        dx = 2.0 / (n_el * (p + 1))
        U, t = P.run(t_end, lambda U: 0.1 * dx)
        assert abs(t - t_end) < 1e-14
        errs.append(P.l2_errors(U, t_end))
    assert math.log2(errs[0][0] / errs[1][0]) > p + 0.5
    assert math.log2(errs[0][1] / errs[1][1]) > p + 0.5
