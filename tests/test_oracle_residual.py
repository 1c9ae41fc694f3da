"""Pins of the oracle's NSFR residual, WA mass inverse and RK4 against the paper's theorems
and a dense brute-force assembly of Eq. NSFR."""
import json
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle import diagnostics, mass, physics, residual
from oracle.operators1d import Ops1D, c_hu
from oracle.problem import Problem

CLAIMS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))
G = 1.4


def flux_scale(P, U):
    """Largest reference-direction flux |f(u) . (J a^d)|: the round-off scale of R."""
    return max(np.abs(physics.euler_flux(U, P.C[d], G)).max() for d in range(3))


def tgv_problem(N, p, c=0.0, face_flux="ec", shape=None):
    shape = shape or (N, N, N)
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    P = Problem(ctrl, shape, p, c=c, face_flux=face_flux)
    U = P.to_internal(wl.perturbed_tgv_state(P.node_coords()))
    return P, U


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hybrid_sbp(p):
    """Q~ + Q~^T = diag(0, W_f diag(n^r_f)) for each direction (Eq. SBP Qtilde)."""
    ops = Ops1D(p)
    n = ops.n
    nv, nfp = n ** 3, n ** 2
    _, _, _, Wf = residual.dense_operators(ops)
    for d in range(3):
        Q = residual.hybrid_qtilde(ops, d)
        S = Q + Q.T
        expect = np.zeros_like(S)
        for s in (0, 1):
            f = 2 * d + s
            sl = slice(nv + f * nfp, nv + (f + 1) * nfp)
            expect[sl, sl] = Wf * (1.0 if s else -1.0)
        assert np.abs(S - expect).max() < 1e-13


@pytest.mark.parametrize("p,shape,face_flux", [(1, (1, 1, 1), "ec"), (2, (2, 1, 1), "ec"),
                                               (2, (1, 2, 2), "ec_roe"), (3, (2, 2, 1), "ec"),
                                               (3, (1, 1, 2), "ec_roe")])
def test_linewise_matches_dense_assembly(p, shape, face_flux):
    """The sum-factorised residual equals the literal dense Eq. NSFR."""
    P, U = tgv_problem(None, p, face_flux=face_flux, shape=shape)
    R = P.residual(U)
    Rd = P.dense_residual(U)
    assert np.abs(R - Rd).max() < 1e-13 * flux_scale(P, U)


def test_dense_check_catches_a_planted_sign_error(monkeypatch):
    """Planted mistake in the line-wise form (hybrid sign flipped): the dense pin must fail."""
    P, U = tgv_problem(None, 2, shape=(2, 1, 1))
    Rd = P.dense_residual(U)
    orig = residual.face_terms

    def wrong(*a, **k):
        return -orig(*a, **k)

    monkeypatch.setattr(residual, "face_terms", wrong)
    R = P.residual(U)
    assert np.abs(R - Rd).max() > 1e-3 * np.abs(Rd).max()


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("face_flux", ["ec", "ec_roe"])
def test_free_stream_preservation(p, face_flux):
    ctrl = wl.control_points(3, 2, 2, p, -math.pi, math.pi, wl.warp_tgv)
    P = Problem(ctrl, (3, 2, 2), p, c=c_hu(p), face_flux=face_flux)
    u = wl.free_stream_state(P.node_coords())
    U = P.to_internal(u)
    R = P.residual(U)
    fscale = np.abs(physics.euler_flux(U, P.C[0], G)).max()
    assert np.abs(R).max() < 1e-13 * fscale
    assert np.abs(P.dudt(U)).max() < 1e-12 * fscale / P.J.min()


@pytest.mark.parametrize("p,N", [(2, 3), (3, 2), (4, 2), (5, 2)])
def test_global_conservation(p, N):
    P, U = tgv_problem(N, p, c=c_hu(p), face_flux="ec_roe")
    R = P.residual(U)
    tot, _ = diagnostics.residual_totals(R)
    # round-off scale: total magnitude of the flux terms that cancel in the sum
    fabs = sum(np.abs(physics.euler_flux(U, P.C[d], G)) for d in range(3))
    for k in range(5):
        assert abs(tot[k]) < 1e-14 * diagnostics.fsum(fabs[k])


@pytest.mark.parametrize("p,N", [(3, 3), (4, 2), (5, 2)])
def test_entropy_conservation_ec(p, N):
    """-sum v.R = 0 with the EC face flux (Sec. Nonlinear Stability), at the paper's 1e-13."""
    P, U = tgv_problem(N, p, c=c_hu(p))
    R = P.residual(U)
    rate, scale = diagnostics.entropy_rate(U, R, G)
    assert abs(rate) < CLAIMS["entropy_rate_order"]["value"] * scale


def test_roe_dissipates_entropy():
    P, U = tgv_problem(2, 3, face_flux="ec_roe")
    rate, scale = diagnostics.entropy_rate(U, P.residual(U), G)
    assert rate < -1e-10 * scale   # dissipative: entropy (= -rho s/(gamma-1)) decreases


@pytest.mark.parametrize("p", [1, 2, 3])
def test_wa_inverse_matches_dense(p):
    ops = Ops1D(p, 0.3 * c_hu(p))
    P, U = tgv_problem(2, p, c=ops.c)
    R = P.residual(U)
    D = mass.wa_inverse_apply(R, P.J, P.ops)
    n = ops.n
    for e in range(3):
        A = mass.dense_wa_inverse(P.J[e].ravel(), P.ops)
        for k in range(5):
            assert np.allclose(D[k, e].ravel(), A @ R[k, e].ravel(), rtol=1e-12, atol=1e-13 * np.abs(D).max())


def test_wa_inverse_dg_is_exact():
    """c = 0: the collocated mass matrix W J is diagonal and the WA inverse is exact."""
    P, U = tgv_problem(2, 3)
    R = P.residual(U)
    assert np.allclose(mass.wa_inverse_apply(R, P.J, P.ops), R / (mass.w3(P.ops) * P.J), rtol=1e-14, atol=0)
    Je = P.J[1].ravel()
    exact = np.linalg.inv(mass.dense_fr_mass(Je, P.ops))
    assert np.allclose(mass.dense_wa_inverse(Je, P.ops), exact, rtol=1e-12)


def test_wa_inverse_affine_reading():
    """On an affine element Pi~ (WJ)^{-1} Pi~^T = (M+K)^{-1} M (M+K)^{-1} / J (the printed
    formula, which differs from the exact (M_m+K_m)^{-1} for c != 0)."""
    ops = Ops1D(3, c_hu(3))
    J = 0.37
    A = mass.dense_wa_inverse(np.full(64, J), ops)
    MK = mass.dense_fr_mass(np.ones(64), ops)
    M = mass.dense_fr_mass(np.ones(64), Ops1D(3, 0.0))
    MKi = np.linalg.inv(MK)
    assert np.allclose(A, MKi @ M @ MKi / J, rtol=1e-11)
    assert not np.allclose(A, np.linalg.inv(J * MK), rtol=1e-3)
    # Chan-Wilcox form is exact on an affine element
    assert np.allclose(mass.dense_chan_wilcox(np.full(64, J), ops), np.linalg.inv(J * MK), rtol=1e-11)


@pytest.mark.parametrize("c_kind", ["dg", "hu"])
def test_rk4_conserves_the_fr_functional(c_kind):
    p = 3
    c = 0.0 if c_kind == "dg" else c_hu(p)
    P, U = tgv_problem(2, p, c=c, face_flux="ec_roe")
    Q0, Qa = diagnostics.conserved_totals(U, P.J, P.ops)
    dt = P.cfl_dt(U, 0.1, 2 * math.pi / (2 * (p + 1)))
    U1 = P.rk4_step(U, dt)
    Q1, _ = diagnostics.conserved_totals(U1, P.J, P.ops)
    for k in range(5):
        assert abs(Q1[k] - Q0[k]) < 1e-13 * Qa[k]


def test_complex_step_matches_central_differences():
    """The oracle's reference derivative (complex step) agrees with central FD."""
    P, U = tgv_problem(2, 2)
    dU = wl.random_cotangent(U.shape, seed=3) * np.abs(U).max(axis=(1, 2, 3, 4), keepdims=True)
    h = 1e-30
    Jd = np.imag(P.dudt(U + 1j * h * dU)) / h
    eps = 1e-6
    fd = (P.dudt(U + eps * dU) - P.dudt(U - eps * dU)) / (2 * eps)
    assert np.abs(Jd - fd).max() < 1e-6 * np.abs(Jd).max()
