"""GPU parity of the uncollocated scheme (nsfr_setup_uncollocated: solution on the
p+1 Lobatto nodes, nq >= p+1 Gauss-Legendre quadrature points, nq > p+1 the paper's
overintegration) against the oracle's UncollocatedProblem.

Bars as for the collocated path: the library's metric terms at the GL points and its
node coordinates at 1e-12, R^ = chi^T R_q, du^/dt and one RK4 step at 1e-12 with the
oracle's metric terms injected (the residual is ill-conditioned, see test_gpu_parity), per
variable and element-wise as ``tests._pairs.check_parity`` states.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle.operators1d import c_hu  # noqa: E402
from oracle.uncollocated import UncollocatedProblem  # noqa: E402
from tests._pairs import check_parity, difference_floor, rel_l2, ulp_sensitivity  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _metrics_abi(P):
    ne, m = P.mesh.n_el, P.nq
    C = np.ascontiguousarray(np.moveaxis(P.C.reshape(3, 3, ne, m ** 3), 2, 0).reshape(ne, 9, m ** 3))
    J = np.ascontiguousarray(P.J.reshape(ne, m ** 3))
    Cf = np.ascontiguousarray(np.moveaxis(P.geo["Cf"].reshape(3, 3, ne, m * m), 2, 0))
    return C, J, Cf


def _case(shape, p, nq, c_kind="dg", face_flux="ec", kind="tgv"):
    from paper_2312_07725_gb300 import Solver
    c = 0.0 if c_kind == "dg" else c_hu(p)
    if kind == "tgv":
        ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    else:
        ctrl = wl.control_points(*shape, p, 0.0, 1.0, wl.warp_unit)
    P = UncollocatedProblem(ctrl, shape, p, nq=nq, c=c, face_flux=face_flux)
    S = Solver(np.ascontiguousarray(ctrl), shape, p, c=c, face_flux=face_flux, nq=nq)
    xs = P.node_coords(ctrl)
    u = wl.perturbed_tgv_state(xs) if kind == "tgv" else wl.perturbed_density_wave_state(xs)
    return ctrl, P, S, np.ascontiguousarray(u)


@pytest.mark.parametrize("p,nq", [(2, 3), (2, 5), (4, 6), (7, 8)])
def test_uncollocated_metrics_and_nodes_match_oracle(p, nq):
    ctrl, P, S, _ = _case((3, 2, 2), p, nq)
    C, J, Cf = S.metrics()
    Co, Jo, Cfo = _metrics_abi(P)
    assert rel_l2(C, Co) < TOL and rel_l2(J, Jo) < TOL and rel_l2(Cf, Cfo) < TOL
    assert np.abs(S.node_coords() - P.node_coords(ctrl)).max() < 1e-13 * np.pi


CASES = [
    (1, 2, (2, 3, 2), "dg", "ec", "tgv"),
    (2, 3, (3, 2, 2), "hu", "ec", "tgv"),       # nq = p+1: the collocated scheme in the LGL basis
    (2, 5, (3, 2, 1), "dg", "ec", "tgv"),       # overintegration by 2
    (3, 5, (2, 2, 2), "hu", "ec_roe", "unit"),
    (3, 7, (2, 1, 2), "dg", "ec_es", "unit"),
    (4, 6, (3, 3, 1), "hu", "ec", "tgv"),       # 9 elements: ragged last CTA
    (5, 7, (2, 1, 1), "dg", "ec", "tgv"),
]


@pytest.mark.parametrize("p,nq,shape,c_kind,face_flux,kind", CASES)
def test_uncollocated_residual_and_dudt_match_oracle(p, nq, shape, c_kind, face_flux, kind):
    _, P, S, u = _case(shape, p, nq, c_kind, face_flux, kind)
    S.set_metrics(*_metrics_abi(P))
    ud = torch.from_numpy(u).cuda()
    R = torch.empty_like(ud)
    D = torch.empty_like(ud)
    S.residual_raw(ud, R)
    S.residual(ud, D)
    torch.cuda.synchronize()
    def res(x):
        return P.to_abi(P.residual(P.to_internal(x)))

    def dudt(x):
        return P.to_abi(P.dudt(P.to_internal(x)))

    check_parity(R.cpu().numpy(), res(u), TOL, ulp_sensitivity(res, u), what="R^")
    check_parity(D.cpu().numpy(), dudt(u), TOL, ulp_sensitivity(dudt, u), what="du^/dt")


def test_uncollocated_rk4_step_matches_oracle():
    _, P, S, u = _case((3, 2, 2), 3, 5, "hu", "ec")
    S.set_metrics(*_metrics_abi(P))
    dt = 2e-3
    u1 = P.rk4_step_abi(u, dt)
    ud = torch.from_numpy(u).cuda()
    S.rk_step(ud, dt=dt)
    torch.cuda.synchronize()
    du = u1 - u
    sens = ulp_sensitivity(lambda x: P.rk4_step_abi(x, dt) - x, u)
    check_parity(ud.cpu().numpy() - u, du, TOL, sens, difference_floor(u1, du), what="RK4 step")


def test_uncollocated_context_rejects_what_it_does_not_support():
    from paper_2312_07725_gb300 import NSFRError, Solver
    ctrl, P, S, u = _case((2, 2, 2), 2, 4)
    ud = torch.from_numpy(u).cuda()
    with pytest.raises(NSFRError):  # the grid cotangent is not offered for this scheme
        S.vjp(ud, torch.ones_like(ud), torch.zeros_like(ud),
              torch.zeros((S.n_el, (S.p_geo + 1) ** 3, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        Solver(np.ascontiguousarray(ctrl), (2, 2, 2), 2, nq=4, precision="fp32_bulk_ff")
    with pytest.raises(NSFRError):
        Solver(np.ascontiguousarray(ctrl), (2, 2, 2), 2, nq=2)  # nq < p+1


@pytest.mark.parametrize("p,nq", [(3, 4), (3, 6), (4, 7)])
def test_uncollocated_entropy_conservation_of_the_library_residual(p, nq):
    """The paper's overintegrated NSFR-EC rows: -v~^ . R^ = 0, with R^ the library's residual
    and v~^ = Pi v(chi u^) the projected entropy variables (from the oracle)."""
    _, P, S, u = _case((2, 2, 2), p, nq, "hu", "ec")
    S.set_metrics(*_metrics_abi(P))
    ud = torch.from_numpy(u).cuda()
    R = torch.empty_like(ud)
    S.residual_raw(ud, R)
    torch.cuda.synchronize()
    Vh, _ = P.projected(P.to_internal(u))
    prod = P.to_abi(Vh) * R.cpu().numpy()
    assert abs(prod.sum()) < 1e-13 * np.abs(prod).sum()


@pytest.mark.parametrize("p,nq,face_flux", [(3, 4, "ec"), (3, 6, "ec"), (4, 7, "ec"), (2, 5, "ec_roe")])
def test_uncollocated_diagnostics_match_oracle(p, nq, face_flux):
    """nsfr_entropy on the uncollocated scheme against the oracle's diagnostics: the entropy,
    kinetic energy and GL quadrature of the solution at 1e-13 relative, the entropy rate
    -v~^ . R^ at the paper's 1e-13 of its scale for EC faces (negative with Roe), the scale
    and sum R^ against the oracle's."""
    _, P, S, u = _case((2, 2, 2), p, nq, "hu", face_flux)
    S.set_metrics(*_metrics_abi(P))
    g = S.entropy(torch.from_numpy(u).cuda())
    o = P.diagnostics(P.to_internal(u))
    assert abs(g["entropy"] - o["entropy"]) < 1e-13 * abs(o["entropy"])
    assert abs(g["kinetic_energy"] - o["kinetic_energy"]) < 1e-13 * abs(o["kinetic_energy"])
    qabs = sum(abs(q) for q in o["Q"])
    for k in range(5):
        assert abs(g["Q"][k] - o["Q"][k]) < 1e-13 * qabs
    assert abs(g["entropy_rate_scale"] - o["entropy_rate_scale"]) < 1e-10 * o["entropy_rate_scale"]
    if face_flux == "ec":
        assert abs(g["entropy_rate"]) < 1e-13 * g["entropy_rate_scale"]
    else:
        assert g["entropy_rate"] < -1e-8 * g["entropy_rate_scale"]
        assert abs(g["entropy_rate"] - o["entropy_rate"]) < 1e-10 * o["entropy_rate_scale"]


@pytest.mark.parametrize("p,nq,shape,c_kind,face_flux", [(2, 3, (3, 2, 2), "hu", "ec"), (3, 5, (2, 2, 2), "hu", "ec"),
                                                         (4, 6, (3, 3, 1), "dg", "ec_roe"), (3, 6, (2, 1, 2), "hu", "ec_es"),
                                                         (6, 7, (2, 1, 1), "hu", "ec"), (7, 8, (1, 2, 1), "hu", "ec")])
def test_uncollocated_fp32_bulk_within_1e5(p, nq, shape, c_kind, face_flux):
    """The FP32-bulk form of the uncollocated scheme (FP32 flux differencing and return to
    the solution nodes, FP64 entropy projection and face fluxes): du^/dt within 1e-5 of the
    oracle over all variables, per variable within max(1e-5, 4x the oracle's change under a
    2^-24 relative change of the state); the raw residual likewise, and one RK4 step."""
    from paper_2312_07725_gb300 import Solver
    ctrl, P, _, u = _case(shape, p, nq, c_kind, face_flux)
    c = 0.0 if c_kind == "dg" else c_hu(p)
    B = Solver(np.ascontiguousarray(ctrl), shape, p, c=c, face_flux=face_flux, nq=nq, precision="fp32_bulk")
    B.set_metrics(*_metrics_abi(P))
    ud = torch.from_numpy(u).cuda()
    D, R = torch.empty_like(ud), torch.empty_like(ud)
    B.residual(ud, D)
    B.residual_raw(ud, R)
    torch.cuda.synchronize()

    def dudt(x):
        return P.to_abi(P.dudt(P.to_internal(x)))

    def res(x):
        return P.to_abi(P.residual(P.to_internal(x)))

    check_parity(D.cpu().numpy(), dudt(u), 1e-5, ulp_sensitivity(dudt, u, rel=2.0 ** -24), what="bulk du^/dt")
    check_parity(R.cpu().numpy(), res(u), 1e-5, ulp_sensitivity(res, u, rel=2.0 ** -24), what="bulk R^")
    dt = 2e-3
    u1 = P.rk4_step_abi(u, dt)
    B.rk_step(ud, dt=dt)
    torch.cuda.synchronize()
    assert rel_l2(ud.cpu().numpy() - u, u1 - u) < 1e-5


@pytest.mark.parametrize("p,nq,shape,c_kind", [(2, 3, (2, 2, 1), "dg"), (2, 4, (2, 1, 2), "hu"),
                                               (3, 5, (1, 2, 2), "hu"), (4, 6, (2, 1, 1), "dg")])
def test_uncollocated_state_vjp_matches_complex_step(p, nq, shape, c_kind):
    """The adjoint of du^/dt for the uncollocated scheme (the reverse of the flux differencing
    on the GL points and of the entropy projection chi, v(u), Pi, u(v)) against the oracle's
    complex-step derivatives, through dot products <rbar, J d> = <J^T rbar, d> at 1e-10;
    nq = p+1 (square chi) and overintegration."""
    _, P, S, u = _case(shape, p, nq, c_kind, "ec")
    S.set_metrics(*_metrics_abi(P))
    rng = np.random.default_rng(7)
    rbar = rng.standard_normal(u.shape)
    ub = torch.zeros(u.shape, dtype=torch.float64, device="cuda")
    S.vjp(torch.from_numpy(u).cuda(), torch.from_numpy(rbar).cuda(), ub)
    ub = ub.cpu().numpy()
    U = P.to_internal(u)
    scale_u = np.abs(u).max(axis=(0, 2), keepdims=True)
    h = 1e-30
    for _ in range(3):
        du = rng.standard_normal(u.shape) * scale_u
        jd = P.to_abi(np.imag(P.dudt(U + 1j * h * P.to_internal(du))) / h)
        lhs, rhs = float(np.sum(rbar * jd)), float(np.sum(ub * du))
        assert abs(lhs - rhs) < 1e-10 * float(np.sum(np.abs(rbar * jd))), (lhs, rhs)
