"""Pins of the oracle's LGL-collocated variant (solution and volume quadrature on
Gauss-Lobatto-Legendre nodes, the paper's kinetic-energy preserving setting).

The same theorems as for GL hold: SBP (exact: LGL integrates degree 2p-1),
the hybridised SBP property, the dense Eq. NSFR, free-stream preservation,
global conservation and entropy conservation with the EC flux (the paper's
NSFR-EC-LGL rows conserve entropy).  What is particular to LGL is pinned too:
the face extrapolations are unit vectors, so the entropy-projected face state
is the boundary node's own state and the hybrid terms reduce to the classical
collocated SBP surface term.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle import diagnostics, physics, residual
from oracle.operators1d import Ops1D, c_hu
from oracle.problem import Problem

CLAIMS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))
G = 1.4


def lgl_problem(shape, p, c=0.0, face_flux="ec", warp=wl.warp_tgv):
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, warp)
    P = Problem(ctrl, shape, p, c=c, face_flux=face_flux, nodes="lgl")
    U = P.to_internal(wl.perturbed_tgv_state(P.node_coords()))
    return P, U


def flux_scale(P, U):
    return max(np.abs(physics.euler_flux(U, P.C[d], G)).max() for d in range(3))


@pytest.mark.parametrize("p", range(1, 8))
def test_lgl_sbp_and_unit_extrapolations(p):
    ops = Ops1D(p, nodes="lgl")
    n = ops.n
    assert ops.xi[0] == -1.0 and ops.xi[-1] == 1.0
    e0, en = np.eye(n)[0], np.eye(n)[-1]
    assert np.abs(ops.t_minus - e0).max() < 1e-15 and np.abs(ops.t_plus - en).max() < 1e-15
    B = ops.W @ ops.D + ops.D.T @ ops.W
    assert np.abs(B - (np.outer(en, en) - np.outer(e0, e0))).max() < 1e-13
    # the derivative is exact on degree-p polynomials
    for k in range(p + 1):
        assert np.abs(ops.D @ ops.xi ** k - k * ops.xi ** max(k - 1, 0) * (k > 0)).max() < 1e-12


def test_lgl_mass_is_not_the_exact_mass():
    """LGL quadrature integrates degree 2p-1 only: W differs from the exact Lagrange mass
    (this is why c_HU on GL reproduces the LGL-lumped mass, Sec. "Maximum CFL")."""
    p = 3
    ops = Ops1D(p, nodes="lgl")
    xg, wg = np.polynomial.legendre.leggauss(p + 2)
    from oracle.operators1d import lagrange_eval
    L = lagrange_eval(ops.xi, xg)
    M_exact = L.T @ np.diag(wg) @ L
    assert np.abs(M_exact - ops.W).max() > 1e-3


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lgl_hybrid_sbp(p):
    ops = Ops1D(p, nodes="lgl")
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


@pytest.mark.parametrize("p,shape,face_flux", [(1, (1, 1, 1), "ec"), (2, (2, 1, 1), "ec_roe"),
                                               (3, (1, 2, 1), "ec")])
def test_lgl_linewise_matches_dense_assembly(p, shape, face_flux):
    P, U = lgl_problem(shape, p, c=0.4 * c_hu(p), face_flux=face_flux)
    R = P.residual(U)
    Rd = P.dense_residual(U)
    assert np.abs(R - Rd).max() < 1e-13 * flux_scale(P, U)


def test_lgl_face_state_is_the_boundary_node():
    """chi_f v(u) at an LGL face is v at the boundary node, so u~_f = u there (to rounding)."""
    P, U = lgl_problem((2, 1, 1), 3)
    Uf = residual.face_states(U, P.ops, G)
    n = P.n
    for d in range(3):
        ax = U.ndim - 1 - d
        for s in (0, 1):
            ub = np.take(U, n - 1 if s else 0, axis=ax)
            assert np.abs(Uf[d][s] - ub).max() < 1e-12 * np.abs(ub).max()


@pytest.mark.parametrize("p", [2, 4])
@pytest.mark.parametrize("face_flux", ["ec", "ec_roe"])
def test_lgl_free_stream_preservation(p, face_flux):
    ctrl = wl.control_points(3, 2, 2, p, -math.pi, math.pi, wl.warp_tgv)
    P = Problem(ctrl, (3, 2, 2), p, c=c_hu(p), face_flux=face_flux, nodes="lgl")
    U = P.to_internal(wl.free_stream_state(P.node_coords()))
    fscale = np.abs(physics.euler_flux(U, P.C[0], G)).max()
    assert np.abs(P.residual(U)).max() < 1e-13 * fscale


@pytest.mark.parametrize("p,N", [(2, 3), (4, 2)])
def test_lgl_global_conservation(p, N):
    P, U = lgl_problem((N, N, N), p, c=c_hu(p), face_flux="ec_roe")
    tot, _ = diagnostics.residual_totals(P.residual(U))
    fabs = sum(np.abs(physics.euler_flux(U, P.C[d], G)) for d in range(3))
    for k in range(5):
        assert abs(tot[k]) < 1e-14 * diagnostics.fsum(fabs[k])


@pytest.mark.parametrize("p,N,c_kind", [(3, 3, "dg"), (4, 2, "hu"), (5, 2, "dg")])
def test_lgl_entropy_conservation_ec(p, N, c_kind):
    """The paper's NSFR-EC-LGL rows: -sum v.R = 0 at 1e-13 with the EC face flux."""
    P, U = lgl_problem((N, N, N), p, c=0.0 if c_kind == "dg" else c_hu(p))
    rate, scale = diagnostics.entropy_rate(U, P.residual(U), G)
    assert abs(rate) < CLAIMS["entropy_rate_order"]["value"] * scale


def test_lgl_roe_dissipates_entropy():
    """Roe dissipation acts on face jumps; an LGL state sampled from a continuous field has
    none (neighbouring boundary nodes coincide), so the elements get independent offsets."""
    P, U = lgl_problem((2, 2, 2), 3, face_flux="ec_roe")
    rate0, scale = diagnostics.entropy_rate(U, P.residual(U), G)
    assert abs(rate0) < CLAIMS["entropy_rate_order"]["value"] * scale
    rng = np.random.default_rng(4)
    U = U * (1.0 + 1e-3 * rng.standard_normal((1, U.shape[1], 1, 1, 1)))
    rate, scale = diagnostics.entropy_rate(U, P.residual(U), G)
    assert rate < -1e-10 * scale


def _wave_error(p, N, tf=0.2, cfl=0.2):
    ctrl = wl.control_points(N, 1, 1, p, 0.0, 1.0, wl.warp_x_only)
    P = Problem(ctrl, (N, 1, 1), p, c=0.0, face_flux="ec_roe", nodes="lgl")
    xyz = P.node_coords()
    U = P.to_internal(wl.density_wave_x_state(xyz, 0.0))
    dx = 1.0 / (N * (p + 1))
    dt0 = cfl * dx / (1.0 + math.sqrt(1.4 / 2.0))
    nsteps = int(math.ceil(tf / dt0))
    for _ in range(nsteps):
        U = P.rk4_step(U, tf / nsteps)
    return diagnostics.l2_error(U, P.to_internal(wl.density_wave_x_state(xyz, tf)), P.J, P.ops, 0)


@pytest.mark.parametrize("p,Ns", [(2, (4, 8, 16)), (3, (4, 8))])
def test_lgl_order_of_accuracy(p, Ns):
    """Order p+1 on the exact density wave (curved mesh, Roe face flux) on LGL nodes too."""
    errs = [_wave_error(p, N) for N in Ns]
    order = math.log(errs[-2] / errs[-1]) / math.log(2.0)
    assert order > (p + 1) - 0.25, (errs, order)


def pressure_part(UL, UR, nvec, gamma):
    """The pressure part of Chandrashekar's flux: p_hat n in the momentum (p_hat =
    rho_bar / (2 beta_bar)); zero mass flux.  Its energy component is irrelevant to the
    kinetic-energy variables, whose energy component is zero, and is left zero."""
    rL, _, pL = physics.primitive(UL, gamma)
    rR, _, pR = physics.primitive(UR, gamma)
    p_hat = 0.5 * (rL + rR) / (rL / (2.0 * pL) + rR / (2.0 * pR))
    F = np.zeros((5,) + np.shape(p_hat), dtype=np.result_type(UL, nvec))
    F[1:4] = p_hat * nvec
    return F


def ke_change_without_pressure(P, U, monkeypatch):
    """sum_i v_KE,i . R_i with the pressure part removed from every two-point flux (volume,
    hybrid and face), v_KE = (-|u|^2/2, u, 0): the kinetic-energy change net of the
    pressure work (the paper's kinetic-energy lemma).  Returns (value, scale)."""
    full = physics.chandrashekar

    def no_pressure(UL, UR, nvec, gamma):
        return full(UL, UR, nvec, gamma) - pressure_part(UL, UR, nvec, gamma)

    monkeypatch.setattr(physics, "chandrashekar", no_pressure)
    R = P.residual(U)
    monkeypatch.setattr(physics, "chandrashekar", full)
    _, vel, _ = physics.primitive(U, G)
    terms = -0.5 * np.sum(vel * vel, axis=0) * R[0] + np.sum(vel * R[1:4], axis=0)
    return diagnostics.fsum(terms), diagnostics.fsum(np.abs(terms))


@pytest.mark.parametrize("p", [2, 4])
def test_kinetic_energy_lemma_lgl_conserves_gl_does_not(p, monkeypatch):
    """Kinetic-energy lemma (Sec. "Nonlinear Stability"): with a kinetic-energy preserving
    two-point flux, the kinetic-energy change net of pressure work vanishes discretely only
    when the face nodes are volume nodes (LGL); on GL it does not (the paper's TGV
    kinetic-energy figures: 1e-12 on LGL, not conserved on GL)."""
    shape = (2, 2, 2)
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    out = {}
    for nodes in ("lgl", "gl"):
        P = Problem(ctrl, shape, p, c=c_hu(p), nodes=nodes)
        U = P.to_internal(wl.perturbed_tgv_state(P.node_coords()))
        out[nodes] = ke_change_without_pressure(P, U, monkeypatch)
    ke, scale = out["lgl"]
    assert abs(ke) < 1e-13 * scale
    ke, scale = out["gl"]
    assert abs(ke) > 1e-8 * scale


def test_lgl_differs_from_gl():
    """The two node sets give different schemes (guards against the option being ignored)."""
    ctrl = wl.control_points(2, 2, 2, 3, -math.pi, math.pi, wl.warp_tgv)
    Pl = Problem(ctrl, (2, 2, 2), 3, nodes="lgl")
    Pg = Problem(ctrl, (2, 2, 2), 3, nodes="gl")
    assert np.abs(Pl.node_coords() - Pg.node_coords()).max() > 1e-2
