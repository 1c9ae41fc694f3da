"""Pins of the oracle's time step, wave speed, RK4 weights, kinetic energy and entropy
total against closed forms (no value here comes from the oracle itself).

* |u| + a with a = sqrt(gamma p / rho) on states whose speeds are chosen integers;
* dt = CFL dx / max(|u| + a) (Sec. "Results": RK4 at CFL 0.1 from the maximum wave speed);
* classic RK4 (Sec. "Results": four-stage, fourth-order): one step of y' = lambda y is the
  degree-4 Taylor polynomial of exp(lambda dt), which fixes the weights (1, 2, 2, 1)/6 and
  the stage nodes (0, 1/2, 1/2, 1); the observed order on nonlinear problems is 4;
* kinetic energy of the Taylor-Green vortex at t = 0 (Sec. "Inviscid Taylor Green Vortex"):
  (1/2) int |u|^2 over [-pi, pi]^3 = pi^3 exactly; the warp is a change of variables, so the
  warped mesh has the same integral;
* the entropy total of a constant state is -rho s/(gamma-1) times the volume (2 pi)^3.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import diagnostics, physics, timestep
from oracle.problem import Problem

G = 1.4


def conserved(rho, vel, p):
    vel = np.asarray(vel, dtype=np.float64)
    E = p / (G - 1.0) + 0.5 * rho * float(vel @ vel)
    return np.array([rho, rho * vel[0], rho * vel[1], rho * vel[2], E])


# two states with |u| = 5 and a = 4 (|u| + a = 9), |u| = 3 and a = 5 (|u| + a = 8)
STATE_9 = conserved(1.2, (3.0, 4.0, 0.0), 16.0 * 1.2 / G)
STATE_8 = conserved(2.0, (1.0, 2.0, -2.0), 25.0 * 2.0 / G)


def test_wavespeed_closed_form():
    U = np.stack([STATE_9, STATE_8], axis=1)
    lam = physics.max_wavespeed(U, G)
    assert abs(lam[0] - 9.0) < 4e-15 * 9.0
    assert abs(lam[1] - 8.0) < 4e-15 * 8.0


def test_cfl_dt_closed_form():
    U = np.stack([STATE_8, STATE_9, STATE_8], axis=1)
    dt = timestep.cfl_dt(U, 0.1, 0.5, G)
    assert abs(dt - 0.1 * 0.5 / 9.0) < 1e-16


def test_wavespeed_of_a_free_stream_grid():
    """Every node of a free stream on a mesh has the same |u| + a."""
    P = Problem(wl.control_points(2, 2, 1, 3, -math.pi, math.pi, wl.warp_tgv), (2, 2, 1), 3)
    rho, vel, p = 1.3, (0.7, -0.4, 0.25), 2.1
    U = P.to_internal(wl.free_stream_state(P.node_coords(), rho, vel, p))
    expect = math.sqrt(sum(v * v for v in vel)) + math.sqrt(G * p / rho)
    lam = physics.max_wavespeed(U, G)
    assert np.abs(lam - expect).max() < 4e-15 * expect


def test_rk4_one_step_is_the_taylor_polynomial():
    """y' = lambda y: one RK4 step multiplies y by 1 + z + z^2/2 + z^3/6 + z^4/24, z = lambda dt."""
    y0 = np.array([1.0, -0.5, 2.0])
    for lam, dt in ((-1.0, 0.3), (2.0, 0.05), (-7.5, 0.1)):
        z = lam * dt
        stab = 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0
        y1 = timestep.rk4_step(y0, dt, lambda y: lam * y)
        assert np.abs(y1 - stab * y0).max() < 4e-16 * np.abs(y0).max() * max(1.0, abs(stab))


def test_rk4_stage_nodes_on_a_quadrature_problem():
    """A right-hand side that depends on an extra clock variable: y' = (1, 3 t^2, 4 t^3), t the
    first component.  RK4 integrates t^2 and t^3 exactly (Simpson's rule, nodes 0, 1/2, 1)."""
    def rhs(y):
        t = y[0]
        return np.array([1.0, 3.0 * t * t, 4.0 * t ** 3])

    y0 = np.array([0.2, 0.2 ** 3, 0.2 ** 4])
    dt = 0.7
    y1 = timestep.rk4_step(y0, dt, rhs)
    t1 = 0.2 + dt
    assert abs(y1[0] - t1) < 1e-15
    assert abs(y1[1] - t1 ** 3) < 1e-14
    assert abs(y1[2] - t1 ** 4) < 1e-14


def _order(rhs, y0, exact, T, n_steps):
    errs = []
    for m in n_steps:
        dt = T / m
        y = y0.copy()
        for _ in range(m):
            y = timestep.rk4_step(y, dt, rhs)
        errs.append(np.abs(y - exact).max())
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_rk4_observed_order_is_four():
    # y' = -y^2, y(0) = 1: y(t) = 1/(1 + t); and a rotation with a nonlinear rate
    orders = _order(lambda y: -y * y, np.array([1.0]), np.array([1.0 / 3.0]), 2.0, [10, 20, 40])
    assert all(3.85 < o < 4.2 for o in orders), orders
    # y = (cos phi, sin phi) with phi' = 1 + |y|^2 = 2: exact phi(T) = 2 T
    def rot(y):
        w = 1.0 + y[0] * y[0] + y[1] * y[1]
        return np.array([-w * y[1], w * y[0]])
    T = 1.0
    orders = _order(rot, np.array([1.0, 0.0]), np.array([math.cos(2 * T), math.sin(2 * T)]), T, [16, 32, 64])
    assert all(3.85 < o < 4.2 for o in orders), orders


def _tgv_ke_errors(warp, ps=(3, 4, 5)):
    errs = []
    for p in ps:
        ctrl = wl.control_points(4, 4, 4, p, -math.pi, math.pi, wl.WARPS[warp])
        P = Problem(ctrl, (4, 4, 4), p)
        U = P.to_internal(wl.tgv_state(P.node_coords()))
        errs.append(abs(diagnostics.kinetic_energy(U, P.J, P.ops) - math.pi ** 3) / math.pi ** 3)
    return errs


def test_kinetic_energy_of_the_taylor_green_vortex_is_pi_cubed():
    """(1/2) int_{[-pi,pi]^3} rho |u|^2 = pi^3 at t = 0 (rho = 1).  On the undeformed mesh of
    4^3 elements the Gauss sums of the trigonometric integrand cancel between elements shifted
    by pi/2, so the quadrature is exact to rounding; on the warped mesh the quadrature error
    falls with p."""
    assert max(_tgv_ke_errors("none")) < 1e-14
    errs = _tgv_ke_errors("tgv")
    assert errs[-1] < 1e-6, errs
    assert errs[0] > errs[1] > errs[2], errs


def test_entropy_total_of_a_constant_state():
    rho, vel, p = 1.3, (0.7, -0.4, 0.25), 2.1
    P = Problem(wl.control_points(2, 3, 2, 3, -math.pi, math.pi, wl.warp_tgv), (2, 3, 2), 3)
    U = P.to_internal(wl.free_stream_state(P.node_coords(), rho, vel, p))
    s = math.log(p) - G * math.log(rho)
    expect = -rho * s / (G - 1.0) * (2 * math.pi) ** 3
    got = diagnostics.entropy_total(U, P.J, P.ops, G)
    assert abs(got - expect) < 1e-12 * abs(expect)
    # the kinetic energy of the same free stream: rho |u|^2 / 2 times the volume
    ke = 0.5 * rho * sum(v * v for v in vel) * (2 * math.pi) ** 3
    assert abs(diagnostics.kinetic_energy(U, P.J, P.ops) - ke) < 1e-12 * ke


def test_wavespeed_pin_catches_a_planted_sound_speed(monkeypatch):
    """Planted mistake (sound speed sqrt(p/rho) without gamma): the closed form fails."""
    def wrong(U, gamma):
        rho, vel, p = physics.primitive(U, gamma)
        return np.sqrt(np.sum(vel * vel, axis=0)) + np.sqrt(p / rho)

    monkeypatch.setattr(physics, "max_wavespeed", wrong)
    lam = physics.max_wavespeed(np.stack([STATE_9], axis=1), G)
    assert abs(lam[0] - 9.0) > 0.1
