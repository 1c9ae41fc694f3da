"""Pins of the oracle's second two-point flux, Chandrashekar's flux with Ranocha's pressure
terms (Sec. "Results": the EC runs use Chandrashekar's flux "with Ranocha's pressure fix"),
and of the residual built on it.

* flux: consistency with the Euler flux, symmetry, the Tadmor shuffle on 10^5 random pairs
  (Eq. tadmor shuffle), kinetic-energy preservation (F_m = F_rho u_bar + p_bar n with the
  arithmetic pressure mean), the pressure-equilibrium values for equal velocity and
  pressure, and two planted mistakes that the shuffle pin catches;
* residual: the sum-factorised form against the literal dense Eq. NSFR, global
  conservation, free-stream preservation and entropy conservation at the paper's 1e-13;
* on the Lobatto-collocated scheme (face states are nodal values) a density wave with
  constant velocity and pressure keeps its pressure: dp/dt = 0 at round-off.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import diagnostics, physics
from oracle.operators1d import c_hu
from oracle.problem import Problem
from tests.test_oracle_physics import random_states

G = 1.4


def _pairs(n, spread, seed):
    UL = random_states(n, seed, 0.5)
    rng = np.random.default_rng(seed + 1)
    rhoR = UL[0] * np.exp(rng.uniform(-spread, spread, n))
    _, uL, pL = physics.primitive(UL, G)
    uR = uL + rng.uniform(-spread, spread, (3, n))
    pR = pL * np.exp(rng.uniform(-spread, spread, n))
    UR = np.concatenate([rhoR[None], rhoR * uR, (pR / (G - 1) + 0.5 * rhoR * np.sum(uR * uR, axis=0))[None]])
    return UL, UR, rng.standard_normal((3, n))


def _shuffle_residual(F, UL, UR, nvec):
    dv = physics.entropy_variables(UL, G) - physics.entropy_variables(UR, G)
    lhs = np.sum(dv * F, axis=0)
    rhs = physics.entropy_potential(UL, nvec) - physics.entropy_potential(UR, nvec)
    vabs = np.abs(physics.entropy_variables(UL, G)) + np.abs(physics.entropy_variables(UR, G))
    scale = np.sum(vabs * np.abs(F), axis=0) + np.abs(physics.entropy_potential(UL, nvec)) \
        + np.abs(physics.entropy_potential(UR, nvec))
    return np.abs(lhs - rhs) / scale


def test_ranocha_consistency_and_symmetry():
    U = random_states(2000, 21)
    nvec = np.random.default_rng(22).standard_normal((3, 2000))
    F = physics.ranocha(U, U, nvec, G)
    f = physics.euler_flux(U, nvec, G)
    assert np.allclose(F, f, rtol=1e-14, atol=1e-14 * np.abs(f).max())
    U2 = random_states(2000, 23)
    assert np.allclose(physics.ranocha(U, U2, nvec, G), physics.ranocha(U2, U, nvec, G), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("spread", [1e-3, 0.05, 0.8])
def test_ranocha_tadmor_shuffle(spread):
    UL, UR, nvec = _pairs(100000, spread, 30)
    assert np.max(_shuffle_residual(physics.ranocha(UL, UR, nvec, G), UL, UR, nvec)) < 2e-15


def test_ranocha_kinetic_energy_preservation_and_pressure_mean():
    """F_m - F_rho u_bar = p_bar n with p_bar = (p_L + p_R)/2 (Jameson's KEP form)."""
    UL, UR, nvec = _pairs(5000, 0.5, 40)
    F = physics.ranocha(UL, UR, nvec, G)
    _, uL, pL = physics.primitive(UL, G)
    _, uR, pR = physics.primitive(UR, G)
    rest = F[1:4] - F[0] * 0.5 * (uL + uR)
    assert np.allclose(rest, 0.5 * (pL + pR) * nvec, rtol=1e-12, atol=1e-12 * np.abs(F[1:4]).max())


def test_ranocha_pressure_equilibrium_values():
    """Equal velocity and pressure on both sides, any densities: F_m = F_rho u + p n and
    F_E = F_rho |u|^2/2 + gamma/(gamma-1) p u . n (the density jump carries no pressure work)."""
    n = 3000
    rng = np.random.default_rng(50)
    rL, rR = np.exp(rng.uniform(-1, 1, n)), np.exp(rng.uniform(-1, 1, n))
    u = rng.uniform(-1, 1, (3, n))
    p = np.exp(rng.uniform(-1, 1, n))
    q2 = np.sum(u * u, axis=0)

    def cons(r):
        return np.concatenate([r[None], r * u, (p / (G - 1) + 0.5 * r * q2)[None]])

    nvec = rng.standard_normal((3, n))
    F = physics.ranocha(cons(rL), cons(rR), nvec, G)
    un = np.sum(u * nvec, axis=0)
    assert np.allclose(F[1:4], F[0] * u + p * nvec, rtol=1e-13, atol=1e-13 * np.abs(F[1:4]).max())
    assert np.allclose(F[4], 0.5 * q2 * F[0] + G / (G - 1) * p * un, rtol=1e-13, atol=1e-13 * np.abs(F[4]).max())


def test_shuffle_catches_planted_pressure_mistakes():
    """Planted mistakes in the pressure terms: the product mean (p_L u_L + p_R u_R)/2 in place
    of the cross mean, or Chandrashekar's momentum pressure p_hat with Ranocha's energy term.
    Each breaks the shuffle by far more than the pin's 2e-15."""
    UL, UR, nvec = _pairs(2000, 0.3, 60)
    _, uL, pL = physics.primitive(UL, G)
    _, uR, pR = physics.primitive(UR, G)
    F = physics.ranocha(UL, UR, nvec, G)
    cross = 0.5 * (pL * np.sum(uR * nvec, 0) + pR * np.sum(uL * nvec, 0))
    same = 0.5 * (pL * np.sum(uL * nvec, 0) + pR * np.sum(uR * nvec, 0))
    wrong1 = F.copy()
    wrong1[4] += same - cross
    assert np.max(_shuffle_residual(wrong1, UL, UR, nvec)) > 1e-6
    bL, bR = UL[0] / (2 * pL), UR[0] / (2 * pR)
    p_hat = 0.5 * (UL[0] + UR[0]) / (bL + bR)
    wrong2 = F.copy()
    wrong2[1:4] += (p_hat - 0.5 * (pL + pR)) * nvec
    assert np.max(_shuffle_residual(wrong2, UL, UR, nvec)) > 1e-6


def _tgv(shape, p, c=0.0, face_flux="ec", nodes="gl"):
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    P = Problem(ctrl, shape, p, c=c, face_flux=face_flux, nodes=nodes, vol_flux="ranocha")
    return P, P.to_internal(wl.perturbed_tgv_state(P.node_coords()))


@pytest.mark.parametrize("p,shape,face_flux", [(1, (1, 1, 1), "ec"), (2, (2, 1, 1), "ec_roe"),
                                               (3, (1, 2, 1), "ec"), (2, (1, 1, 2), "ec_es")])
def test_ranocha_linewise_matches_dense_assembly(p, shape, face_flux):
    P, U = _tgv(shape, p, face_flux=face_flux)
    fscale = max(np.abs(physics.euler_flux(U, P.C[d], G)).max() for d in range(3))
    assert np.abs(P.residual(U) - P.dense_residual(U)).max() < 1e-13 * fscale


@pytest.mark.parametrize("p,N", [(3, 3), (4, 2), (5, 2)])
def test_ranocha_entropy_conservation_and_conservation(p, N):
    P, U = _tgv((N, N, N), p, c=c_hu(p))
    R = P.residual(U)
    rate, scale = diagnostics.entropy_rate(U, R, G)
    assert abs(rate) < 1e-13 * scale
    tot, _ = diagnostics.residual_totals(R)
    fabs = sum(np.abs(physics.euler_flux(U, P.C[d], G)) for d in range(3))
    for k in range(5):
        assert abs(tot[k]) < 1e-14 * diagnostics.fsum(fabs[k])


@pytest.mark.parametrize("face_flux", ["ec", "ec_roe"])
def test_ranocha_free_stream(face_flux):
    p = 3
    ctrl = wl.control_points(3, 2, 2, p, -math.pi, math.pi, wl.warp_tgv)
    P = Problem(ctrl, (3, 2, 2), p, c=c_hu(p), face_flux=face_flux, vol_flux="ranocha")
    U = P.to_internal(wl.free_stream_state(P.node_coords()))
    fscale = np.abs(physics.euler_flux(U, P.C[0], G)).max()
    assert np.abs(P.residual(U)).max() < 1e-13 * fscale


def test_ranocha_differs_from_chandrashekar():
    """The two fluxes share the mass flux but not the pressure terms."""
    UL, UR, nvec = _pairs(1000, 0.3, 70)
    Fr = physics.ranocha(UL, UR, nvec, G)
    Fc = physics.chandrashekar(UL, UR, nvec, G)
    assert np.allclose(Fr[0], Fc[0], rtol=1e-14)
    assert np.abs(Fr[1:] - Fc[1:]).max() > 1e-4 * np.abs(Fc[1:]).max()


@pytest.mark.parametrize("vol_flux", ["ranocha", "chandrashekar"])
def test_pressure_equilibrium_of_the_lobatto_scheme(vol_flux):
    """A density wave with constant velocity and pressure on the Lobatto-collocated scheme
    (face states are the nodal end values): dp/dt = (gamma-1)(dE/dt - u . dm/dt + |u|^2/2
    drho/dt) = 0 at round-off, for a curved mesh (free-stream preservation supplies the
    metric identities)."""
    p, shape = 3, (2, 2, 2)
    ctrl = wl.control_points(*shape, p, 0.0, 1.0, wl.warp_unit)
    P = Problem(ctrl, shape, p, nodes="lgl", vol_flux=vol_flux)
    xyz = P.node_coords()
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rho = 2.0 + 0.3 * np.sin(2 * math.pi * (x + y + z))
    vel, pr = (0.7, -0.3, 0.4), 1.5
    one = np.ones_like(x)
    U = P.to_internal(wl.conserved_from_primitive(rho, vel[0] * one, vel[1] * one, vel[2] * one, pr * one, G))
    D = P.dudt(U)
    v = np.array(vel)[:, None, None, None, None]
    dp = (G - 1) * (D[4] - np.sum(v * D[1:4], axis=0) + 0.5 * float(np.dot(vel, vel)) * D[0])
    assert np.abs(D[0]).max() > 1e-2
    assert np.abs(dp).max() < 1e-12 * np.abs(D[4]).max()
