"""Pins of the entropy-variable matrix dissipation (face flux "ec_es"):
f* = f_EC - (1/2) R |Lambda| T R^T [[v]].

* Linearised at a state, R |Lambda| T R^T [[v]] is Roe's |A_n| [[u]] (Barth's scaling
  gives R T R^T = du/dv): checked by complex-step derivatives to 1e-12, which fixes the
  eigenvectors, the speeds and the scaling all at once.
* The linearised matrix is symmetric positive semi-definite, and for finite jumps every
  face dissipates entropy: [[v]] . D >= 0 on 10^4 random pairs.
* A zero jump gives no dissipation; the scheme stays free-stream preserving,
  conservative, equal to its dense assembly, and strictly entropy dissipative.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import diagnostics, physics
from oracle.operators1d import c_hu
from oracle.problem import Problem

G = 1.4
H = 1e-30


def _state(r, u, p):
    u = np.asarray(u, dtype=float)
    return np.array([r, r * u[0], r * u[1], r * u[2], p / (G - 1) + 0.5 * r * u @ u])


def _linearised(fn, U, nvec):
    """Columns: d fn(U, u(v + h e_k)) / dh at h = 0, by the complex step."""
    V = physics.entropy_variables(U[:, None], G)[:, 0]
    M = np.zeros((5, 5))
    for k in range(5):
        Vc = V.astype(complex)
        Vc[k] += 1j * H
        UR = physics.conserved_from_entropy(Vc[:, None], G)
        M[:, k] = np.imag(fn(U[:, None].astype(complex), UR, nvec[:, None], G)[:, 0]) / H
    return M


STATES = [(_state(1.3, [0.4, -0.2, 0.7], 2.0), np.array([0.3, -0.8, 0.5])),
          (_state(0.7, [-1.5, 0.1, 0.2], 0.4), np.array([1.7, 0.2, -0.1])),  # supersonic along n
          (_state(1.0, [0.0, 0.0, 0.0], 71.4), np.array([0.0, 0.0, 2.5]))]   # at rest, low Mach


@pytest.mark.parametrize("U,nvec", STATES)
def test_linearisation_is_roe_in_entropy_variables(U, nvec):
    D = _linearised(physics.es_matrix_dissipation, U, nvec)
    A = _linearised(lambda a, b, n, g: physics.roe_matrix_apply(a, b, n, g, absolute=True), U, nvec)
    assert np.abs(D - A).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("U,nvec", STATES)
def test_linearised_matrix_is_symmetric_positive_semidefinite(U, nvec):
    D = _linearised(physics.es_matrix_dissipation, U, nvec)
    assert np.abs(D - D.T).max() < 1e-12 * np.abs(D).max()
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > -1e-12 * np.abs(D).max()


def test_every_face_dissipates_entropy_for_finite_jumps():
    rng = np.random.default_rng(7)
    m = 10000
    r = rng.uniform(0.2, 3.0, (2, m))
    vel = rng.normal(0.0, 1.0, (2, 3, m))
    p = rng.uniform(0.1, 5.0, (2, m))
    UL = np.concatenate([r[0][None], r[0] * vel[0], (p[0] / (G - 1) + 0.5 * r[0] * (vel[0] ** 2).sum(0))[None]])
    UR = np.concatenate([r[1][None], r[1] * vel[1], (p[1] / (G - 1) + 0.5 * r[1] * (vel[1] ** 2).sum(0))[None]])
    nvec = rng.normal(0.0, 1.0, (3, m))
    D = physics.es_matrix_dissipation(UL, UR, nvec, G)
    dv = physics.entropy_variables(UR, G) - physics.entropy_variables(UL, G)
    prod = (dv * D).sum(0)
    assert prod.min() >= -1e-12 * np.abs(dv * D).sum(0).max()
    # no jump, no dissipation
    assert np.abs(physics.es_matrix_dissipation(UL, UL, nvec, G)).max() == 0.0


def _problem(shape, p, face_flux, nodes="gl"):
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    P = Problem(ctrl, shape, p, c=c_hu(p), face_flux=face_flux, nodes=nodes)
    return P, P.to_internal(wl.perturbed_tgv_state(P.node_coords()))


def test_es_scheme_matches_dense_assembly_and_preserves_free_stream():
    P, U = _problem((2, 1, 1), 2, "ec_es")
    scale = max(np.abs(physics.euler_flux(U, P.C[d], G)).max() for d in range(3))
    assert np.abs(P.residual(U) - P.dense_residual(U)).max() < 1e-13 * scale
    Uf = P.to_internal(wl.free_stream_state(P.node_coords()))
    assert np.abs(P.residual(Uf)).max() < 1e-13 * np.abs(physics.euler_flux(Uf, P.C[0], G)).max()


def test_es_scheme_conserves_and_dissipates_entropy():
    P, U = _problem((3, 2, 2), 3, "ec_es")
    R = P.residual(U)
    tot, _ = diagnostics.residual_totals(R)
    fabs = sum(np.abs(physics.euler_flux(U, P.C[d], G)) for d in range(3))
    for k in range(5):
        assert abs(tot[k]) < 1e-14 * diagnostics.fsum(fabs[k])
    rate, scale = diagnostics.entropy_rate(U, R, G)
    assert rate < -1e-10 * scale
