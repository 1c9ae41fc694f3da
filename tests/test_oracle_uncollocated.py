"""Pins of the oracle's uncollocated NSFR (solution on LGL nodes, GL quadrature with
N_q >= p+1 points per direction, N_q > p+1 being the paper's overintegration).

* With N_q = p+1 the scheme is the GL-collocated one written in the LGL basis: du^/dt equals
  chi^{-1} applied to the collocated du/dt of the interpolated state (two independent
  code paths: dense chi/Pi operators against the collocated operators).
* The hybridised SBP property of the GL-point operators for any N_q.
* Free-stream preservation, global conservation, entropy conservation of the EC scheme at
  the paper's 1e-13 with overintegration (its NSFR-EC rows with overintegration 3), entropy
  dissipation with Roe, and order p+1 on the density wave.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle import diagnostics, physics
from oracle.operators1d import c_hu
from oracle.problem import Problem
from oracle.uncollocated import UncollocatedProblem, tensor3

CLAIMS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))
G = 1.4


def _tgv(shape, p, nq, c=0.0, face_flux="ec", seed=wl.PARITY_SEED, kind="tgv"):
    if kind == "tgv":
        ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    else:  # the density wave on the warped unit cube
        ctrl = wl.control_points(*shape, p, 0.0, 1.0, wl.warp_unit)
    P = UncollocatedProblem(ctrl, shape, p, nq=nq, c=c, face_flux=face_flux)
    xs = P.node_coords(ctrl)
    u = wl.perturbed_tgv_state(xs, seed) if kind == "tgv" else wl.perturbed_density_wave_state(xs, seed)
    return ctrl, P, P.to_internal(u)


# Roe is checked on the density wave: on the low-Mach vortex its acoustic terms amplify
# rounding (the residual moves by ~3e-12 per ulp of the state)
@pytest.mark.parametrize("p,c_kind,face_flux,kind", [(2, "dg", "ec", "tgv"), (3, "hu", "ec_roe", "unit"),
                                                     (4, "hu", "ec", "tgv")])
def test_square_chi_is_the_gl_collocated_scheme_in_the_lgl_basis(p, c_kind, face_flux, kind):
    shape = (2, 2, 1)
    c = 0.0 if c_kind == "dg" else c_hu(p)
    ctrl, P, U = _tgv(shape, p, p + 1, c, face_flux, kind=kind)
    Pg = Problem(ctrl, shape, p, c=c, face_flux=face_flux)
    Ug = tensor3(P.chi, U)                      # the same polynomials, at the GL nodes
    dg = Pg.dudt(Ug)
    du = P.dudt(U)
    ref = tensor3(np.linalg.inv(P.chi), dg)
    assert np.abs(du - ref).max() < 1e-11 * np.abs(ref).max()
    # and the residuals: R^ = chi^T R_GL
    assert np.abs(P.residual(U) - tensor3(P.chi.T, Pg.residual(Ug))).max() < 1e-12 * np.abs(Pg.residual(Ug)).max()


@pytest.mark.parametrize("p,extra", [(1, 0), (2, 1), (3, 3), (5, 2)])
def test_gl_point_operators_are_hybrid_sbp(p, extra):
    ctrl = wl.control_points(1, 1, 1, p, -1.0, 1.0)
    P = UncollocatedProblem(ctrl, (1, 1, 1), p, nq=p + 1 + extra)
    q = P.qops
    B = q.W @ q.D + q.D.T @ q.W
    assert np.abs(B - (np.outer(q.t_plus, q.t_plus) - np.outer(q.t_minus, q.t_minus))).max() < 1e-13
    assert np.abs(P.Pi @ P.chi - np.eye(p + 1)).max() < 1e-13
    assert np.abs(P.chi.T @ q.t_plus - np.eye(p + 1)[-1]).max() < 1e-13  # chi^T E^T = l(+1) = e_N (LGL)


@pytest.mark.parametrize("p,extra", [(2, 2), (3, 1)])
def test_overintegrated_free_stream_and_conservation(p, extra):
    ctrl, P, U = _tgv((3, 2, 2), p, p + 1 + extra, c=c_hu(p), face_flux="ec_roe", kind="unit")
    fs = P.to_internal(wl.free_stream_state(P.node_coords(ctrl)))
    scale = np.abs(physics.euler_flux(fs, np.ones((3,) + fs.shape[1:]), G)).max()
    assert np.abs(P.residual(fs)).max() < 1e-13 * scale * np.abs(P.C).max()
    R = P.residual(U)
    for k in range(5):
        tot = diagnostics.fsum(R[k])
        assert abs(tot) < 1e-14 * diagnostics.fsum(np.abs(R[k])) * 50


@pytest.mark.parametrize("p,extra,c_kind", [(2, 3, "dg"), (3, 3, "hu"), (4, 1, "dg")])
def test_overintegrated_entropy_conservation_ec(p, extra, c_kind):
    """The paper's NSFR-EC rows with overintegration: -v~^ . R^ = 0 at 1e-13."""
    _, P, U = _tgv((2, 2, 2), p, p + 1 + extra, c=0.0 if c_kind == "dg" else c_hu(p))
    rate, scale = P.entropy_rate(U)
    assert abs(rate) < CLAIMS["entropy_rate_order"]["value"] * scale


def test_overintegrated_roe_dissipates_entropy():
    _, P, U = _tgv((2, 2, 2), 3, 6, face_flux="ec_roe")
    rate, scale = P.entropy_rate(U)
    assert rate < -1e-10 * scale


def test_overintegration_changes_the_scheme():
    _, P4, U = _tgv((2, 1, 1), 3, 4)
    _, P6, _ = _tgv((2, 1, 1), 3, 6)
    d4, d6 = P4.dudt(U), P6.dudt(U)
    assert np.abs(d4 - d6).max() > 1e-6 * np.abs(d4).max()


def _wave_error(p, nq, N, tf=0.2, cfl=0.2):
    ctrl = wl.control_points(N, 1, 1, p, 0.0, 1.0, wl.warp_x_only)
    P = UncollocatedProblem(ctrl, (N, 1, 1), p, nq=nq, face_flux="ec_roe")
    xs = P.node_coords(ctrl)
    U = P.to_internal(wl.density_wave_x_state(xs, 0.0))
    dx = 1.0 / (N * (p + 1))
    dt0 = cfl * dx / (1.0 + math.sqrt(1.4 / 2.0))
    nsteps = int(math.ceil(tf / dt0))
    for _ in range(nsteps):
        U = P.rk4_step(U, tf / nsteps)
    err = U - P.to_internal(wl.density_wave_x_state(xs, tf))
    # L2 norm of the rho error with the GL quadrature of the solution polynomial
    Eq = tensor3(P.chi, err[0:1])[0]
    wq = P.wq
    w3 = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]
    return math.sqrt(diagnostics.fsum(w3 * P.J * Eq * Eq))


def test_overintegrated_order_of_accuracy():
    p = 2
    errs = [_wave_error(p, p + 3, N) for N in (4, 8, 16)]
    order = math.log(errs[-2] / errs[-1]) / math.log(2.0)
    assert order > (p + 1) - 0.25, (errs, order)


@pytest.mark.parametrize("nq", [4, 6])
def test_uncollocated_diagnostics_of_a_constant_state(nq):
    """A constant state is a polynomial of every degree, so chi reproduces it at the GL
    points: S = -rho s/(gamma-1) V, Q = u V and KE = rho|u|^2/2 V with V = (2 pi)^3; its
    residual and entropy rate vanish."""
    p = 3
    ctrl = wl.control_points(2, 2, 1, p, -math.pi, math.pi, wl.warp_tgv)
    P = UncollocatedProblem(ctrl, (2, 2, 1), p, nq=nq)
    rho, vel, pr = 1.3, (0.7, -0.4, 0.25), 2.1
    U = P.to_internal(wl.free_stream_state(P.node_coords(ctrl), rho, vel, pr))
    d = P.diagnostics(U)
    V = (2 * math.pi) ** 3
    s = math.log(pr) - 1.4 * math.log(rho)
    assert abs(d["entropy"] - (-rho * s / 0.4 * V)) < 1e-12 * abs(rho * s / 0.4 * V)
    E = pr / 0.4 + 0.5 * rho * sum(v * v for v in vel)
    for k, q in enumerate([rho, rho * vel[0], rho * vel[1], rho * vel[2], E]):
        assert abs(d["Q"][k] - q * V) < 1e-12 * abs(q * V)
    ke = 0.5 * rho * sum(v * v for v in vel) * V
    assert abs(d["kinetic_energy"] - ke) < 1e-12 * ke
    assert abs(d["entropy_rate"]) < 1e-12 * abs(ke)


def test_uncollocated_taylor_green_kinetic_energy_is_pi_cubed():
    """(1/2) int rho |u|^2 = pi^3 at t = 0 on the warped [-pi, pi]^3; the GL quadrature of the
    Lobatto interpolant converges to it as p grows (over-integration does not change the
    interpolant, only its quadrature)."""
    errs = []
    for p in (3, 4, 5):
        ctrl = wl.control_points(4, 4, 4, p, -math.pi, math.pi, wl.warp_tgv)
        P = UncollocatedProblem(ctrl, (4, 4, 4), p, nq=p + 2)
        U = P.to_internal(wl.tgv_state(P.node_coords(ctrl)))
        errs.append(abs(P.diagnostics(U)["kinetic_energy"] - math.pi ** 3) / math.pi ** 3)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5, errs
