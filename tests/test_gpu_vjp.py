"""The hand-written adjoint (nsfr_vjp) and the RK4 discrete adjoint.

Reference derivatives come from the oracle by the complex-step method (exact to
round-off); the adjoint is compared through dot products <rbar, J d> = <J^T rbar, d>
for seeded random directions d, at relative 1e-10.  The RK4 adjoint with
checkpointing is also compared with central finite differences of the library's
own trajectories (step 1e-6, relative 1e-6).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import diagnostics  # noqa: E402
from oracle.operators1d import c_hu  # noqa: E402
from oracle.problem import Problem  # noqa: E402
from tests._pairs import oracle_metrics_abi  # noqa: E402

pytestmark = pytest.mark.gpu
H = 1e-30  # complex step


def _setup(shape, p, c, amp=1.0):
    from paper_2312_07725_gb300 import Solver
    warp = wl.make_warp_scaled(wl.warp_tgv, amp)
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, warp)
    P = Problem(ctrl, shape, p, c=c)
    S = Solver(ctrl, shape, p, c=c)
    return ctrl, P, S


def _dot_scale(a, b):
    return float(np.sum(np.abs(a * b)))


@pytest.mark.parametrize("p,shape,c_kind", [(2, (2, 2, 1), "dg"), (3, (2, 1, 2), "hu"), (4, (1, 2, 2), "hu")])
def test_state_vjp_matches_complex_step(p, shape, c_kind):
    c = 0.0 if c_kind == "dg" else c_hu(p)
    ctrl, P, S = _setup(shape, p, c)
    S.set_metrics(*oracle_metrics_abi(P))
    u = np.ascontiguousarray(wl.perturbed_tgv_state(P.node_coords()))
    rng = np.random.default_rng(5)
    rbar = rng.standard_normal(u.shape)
    ub = torch.zeros(u.shape, dtype=torch.float64, device="cuda")
    S.vjp(torch.from_numpy(u).cuda(), torch.from_numpy(rbar).cuda(), ub)
    ub = ub.cpu().numpy()
    U = P.to_internal(u)
    scale_u = np.abs(u).max(axis=(0, 2), keepdims=True)
    for trial in range(3):
        du = rng.standard_normal(u.shape) * scale_u
        jd = P.to_abi(np.imag(P.dudt(U + 1j * H * P.to_internal(du))) / H)
        lhs = float(np.sum(rbar * jd))
        rhs = float(np.sum(ub * du))
        assert abs(lhs - rhs) < 1e-10 * _dot_scale(rbar, jd), (lhs, rhs)


@pytest.mark.parametrize("p,shape,c_kind", [(2, (2, 2, 1), "dg"), (3, (1, 2, 2), "hu"), (4, (2, 1, 1), "hu"),
                                            (5, (1, 1, 2), "dg"), (6, (1, 2, 1), "hu"), (7, (2, 1, 1), "hu")])
def test_control_point_vjp_matches_complex_step(p, shape, c_kind):
    c = 0.0 if c_kind == "dg" else c_hu(p)
    ctrl, P, S = _setup(shape, p, c)
    u = np.ascontiguousarray(wl.perturbed_tgv_state(P.node_coords()))
    rng = np.random.default_rng(6)
    rbar = rng.standard_normal(u.shape)
    ub = torch.zeros(u.shape, dtype=torch.float64, device="cuda")
    xb = torch.zeros(ctrl.shape, dtype=torch.float64, device="cuda")
    S.vjp(torch.from_numpy(u).cuda(), torch.from_numpy(rbar).cuda(), ub, xb)
    xb = xb.cpu().numpy()
    U = P.to_internal(u)
    for trial in range(3):
        dx = rng.standard_normal(ctrl.shape)
        Pc = Problem(ctrl + 1j * H * dx, shape, p, c=c)
        jd = P.to_abi(np.imag(Pc.dudt(U.astype(complex))) / H)
        lhs = float(np.sum(rbar * jd))
        rhs = float(np.sum(xb * dx))
        assert abs(lhs - rhs) < 1e-10 * _dot_scale(rbar, jd), (lhs, rhs)


def _strong_state(xyz):
    """Taylor-Green state with 30% density and pressure perturbations: most node
    pairs of a line then take the log branch of the log means, not the series."""
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    drho, du, dv, dw, dp = wl.smooth_perturbation(xyz, amp_rel=0.3, amp_vel=0.3)
    p = (100.0 / wl.GAMMA + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0) * (1.0 + dp)
    return wl.conserved_from_primitive(1.0 + drho, np.sin(x) * np.cos(y) * np.cos(z) + du,
                                       -np.cos(x) * np.sin(y) * np.cos(z) + dv, dw, p)


@pytest.mark.parametrize("p,shape", [(3, (2, 1, 2)), (4, (1, 2, 1))])
def test_vjp_log_branch_matches_complex_step(p, shape):
    """State and control-point VJP where the log means take their log branch
    ((a-b)/(a+b) above 1% for most pairs)."""
    c = c_hu(p)
    ctrl, P, S = _setup(shape, p, c)
    u = np.ascontiguousarray(_strong_state(P.node_coords()))
    rho = u[:, 0].reshape(-1, p + 1, p + 1, p + 1)
    f = (rho[..., :, None] - rho[..., None, :]) / (rho[..., :, None] + rho[..., None, :])
    assert np.mean(f * f >= 1e-4) > 0.5
    rng = np.random.default_rng(11)
    rbar = rng.standard_normal(u.shape)
    ub = torch.zeros(u.shape, dtype=torch.float64, device="cuda")
    xb = torch.zeros(ctrl.shape, dtype=torch.float64, device="cuda")
    S.vjp(torch.from_numpy(u).cuda(), torch.from_numpy(rbar).cuda(), ub, xb)
    ub, xb = ub.cpu().numpy(), xb.cpu().numpy()
    U = P.to_internal(u)
    du = rng.standard_normal(u.shape) * np.abs(u).max(axis=(0, 2), keepdims=True)
    jd = P.to_abi(np.imag(P.dudt(U + 1j * H * P.to_internal(du))) / H)
    assert abs(float(np.sum(rbar * jd)) - float(np.sum(ub * du))) < 1e-10 * _dot_scale(rbar, jd)
    dx = rng.standard_normal(ctrl.shape)
    Pc = Problem(ctrl + 1j * H * dx, shape, p, c=c)
    jd = P.to_abi(np.imag(Pc.dudt(U.astype(complex))) / H)
    assert abs(float(np.sum(rbar * jd)) - float(np.sum(xb * dx))) < 1e-10 * _dot_scale(rbar, jd)


def _ke_grad(u, wj):
    rho = u[:, 0]
    m = u[:, 1:4]
    g = torch.zeros_like(u)
    g[:, 0] = -0.5 * wj * (m * m).sum(dim=1) / rho ** 2
    g[:, 1:4] = wj[:, None] * m / rho[:, None]
    return g


def _ke(u, wj):
    return float((0.5 * wj * (u[:, 1:4] ** 2).sum(dim=1) / u[:, 0]).sum())


def test_rk4_adjoint_against_fd_and_oracle():
    """dKE(u_N)/du_0 and dKE(u_N)/d(mesh amplitude) on the 2^3, p=2 warped TGV mesh,
    6 frozen-dt RK4 steps, checkpoints every 4 steps."""
    from paper_2312_07725_gb300 import Solver
    from paper_2312_07725_gb300.autograd import rk4_adjoint
    shape, p, c, nsteps = (2, 2, 2), 2, c_hu(2), 6
    ctrl, P, S = _setup(shape, p, c)
    u0 = np.ascontiguousarray(wl.tgv_state(P.node_coords()))
    dx = 2 * math.pi / (2 * (p + 1))
    dt = P.cfl_dt(P.to_internal(u0), 0.1, dx)
    wj = torch.from_numpy(S.quadrature()).cuda()
    u0d = torch.from_numpy(u0).cuda()
    lam, xbar, uN = rk4_adjoint(S, u0d, dt, nsteps, lambda v: _ke_grad(v, wj), checkpoint_every=4)
    lam, xbar = lam.cpu().numpy(), xbar.cpu().numpy()
    rng = np.random.default_rng(8)
    d = rng.standard_normal(u0.shape) * np.abs(u0).max(axis=(0, 2), keepdims=True) * 1e-2

    def traj_ke(solver, v0, wjt):
        v = torch.from_numpy(np.ascontiguousarray(v0)).cuda()
        for _ in range(nsteps):
            solver.rk_step(v, dt=dt)
        return _ke(v, wjt)

    # (a) central finite differences of the library's trajectory
    eps = 1e-6
    fd = (traj_ke(S, u0 + eps * d, wj) - traj_ke(S, u0 - eps * d, wj)) / (2 * eps)
    adj = float(np.sum(lam * d))
    assert abs(fd - adj) < 1e-6 * abs(adj)
    # (b) the oracle's complex-step derivative of its own RK4 trajectory (same frozen dt)
    U = P.to_internal(u0).astype(complex) + 1j * H * P.to_internal(d)
    for _ in range(nsteps):
        U = P.rk4_step(U, dt)
    ref = np.imag(diagnostics.kinetic_energy_c(U, P.J, P.ops)) / H
    assert abs(ref - adj) < 1e-10 * abs(ref)

    # mesh amplitude a: ctrl(a) = ctrl + a D(X), D a smooth 2 pi-periodic displacement
    # (the Taylor-Green warp itself vanishes at every p = 2 control point of a 2^3 mesh;
    # the field is O(1) so that dKE/da stands well above the rounding noise of the FD)
    X0 = wl.control_points(*shape, p, -math.pi, math.pi)
    Xs, Ys, Zs = X0[..., 0], X0[..., 1], X0[..., 2]
    dctrl = 1.0 * np.stack([np.sin(Xs + 0.3) * np.cos(Ys - 0.2) * np.sin(Zs + 0.7),
                             np.cos(Xs - 0.5) * np.sin(Ys + 0.4) * np.cos(Zs),
                             np.sin(Xs) * np.sin(Ys + 0.9) * np.cos(Zs - 0.1)], axis=-1)
    adj_a = float(np.sum(xbar * dctrl))

    def ke_at_amp(a):
        S2 = Solver(np.ascontiguousarray(ctrl + a * dctrl), shape, p, c=c)
        return traj_ke(S2, u0, torch.from_numpy(S2.quadrature()).cuda())

    fd_a = (ke_at_amp(eps) - ke_at_amp(-eps)) / (2 * eps)
    assert abs(fd_a - adj_a) < 1e-6 * abs(adj_a)
    Pc = Problem(ctrl + 1j * H * dctrl, shape, p, c=c)
    U = P.to_internal(u0).astype(complex)
    for _ in range(nsteps):
        U = Pc.rk4_step(U, dt)
    ref_a = np.imag(diagnostics.kinetic_energy_c(U, Pc.J, Pc.ops)) / H
    assert abs(ref_a - adj_a) < 1e-10 * abs(ref_a)


def test_autograd_function_backward():
    """torch.autograd through dudt() gives the VJP: sum(w * dudt(u)) gradient."""
    from paper_2312_07725_gb300.autograd import dudt
    shape, p = (2, 2, 1), 3
    ctrl, P, S = _setup(shape, p, 0.0)
    S.set_metrics(*oracle_metrics_abi(P))
    u0 = np.ascontiguousarray(wl.perturbed_tgv_state(P.node_coords()))
    u = torch.from_numpy(u0).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(9).standard_normal(u0.shape)).cuda()
    (dudt(u, S) * w).sum().backward()
    g = u.grad.cpu().numpy()
    d = np.random.default_rng(10).standard_normal(u0.shape) * np.abs(u0).max(axis=(0, 2), keepdims=True)
    jd = P.to_abi(np.imag(P.dudt(P.to_internal(u0) + 1j * H * P.to_internal(d))) / H)
    lhs = float(np.sum(w.cpu().numpy() * jd))
    assert abs(lhs - float(np.sum(g * d))) < 1e-10 * _dot_scale(w.cpu().numpy(), jd)
