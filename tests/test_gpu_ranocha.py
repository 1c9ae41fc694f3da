"""GPU parity of the second volume flux, Chandrashekar's flux with Ranocha's pressure terms
(NSFR_FLUX_RANOCHA; Sec. "Results": the paper's EC runs), against the oracle's
``vol_flux="ranocha"`` scheme.

Bars as for the Chandrashekar path (tests._pairs.check_parity): R, du/dt and one RK4 step
at 1e-12 with the oracle's metric terms injected, per variable and element-wise within
max(1e-12, 4x the oracle's 1-ulp sensitivity); GL and LGL collocated, the uncollocated
(overintegrated) scheme, EC, Roe and entropy-variable face fluxes, ragged CTAs; the
semi-discrete entropy rate of the EC scheme at the paper's 1e-13.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle.operators1d import c_hu  # noqa: E402
from oracle.problem import Problem  # noqa: E402
from oracle.uncollocated import UncollocatedProblem  # noqa: E402
from tests._pairs import (check_parity, difference_floor, make_ctrl, oracle_metrics_abi, state_for,  # noqa: E402
                          ulp_sensitivity)

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _case(shape, p, c_kind, face_flux, kind, nodes="gl"):
    from paper_2312_07725_gb300 import Solver
    c = 0.0 if c_kind == "dg" else c_hu(p)
    ctrl = make_ctrl(shape, p, kind)
    P = Problem(ctrl, shape, p, c=c, face_flux=face_flux, nodes=nodes, vol_flux="ranocha")
    S = Solver(np.ascontiguousarray(ctrl), shape, p, c=c, face_flux=face_flux, nodes=nodes, vol_flux="ranocha")
    S.set_metrics(*oracle_metrics_abi(P))
    return P, S, state_for(P, kind)


CASES = [
    # p, shape, c, face flux, mesh, nodes
    (1, (2, 3, 2), "dg", "ec", "tgv", "gl"),
    (2, (3, 2, 5), "hu", "ec", "tgv", "gl"),       # 30 elements: ragged last CTA
    (3, (4, 4, 4), "dg", "ec", "tgv", "gl"),
    (3, (3, 3, 2), "hu", "ec_roe", "unit", "gl"),
    (4, (3, 3, 1), "hu", "ec", "tgv", "gl"),       # ragged at 2 elements per CTA
    (4, (2, 3, 2), "dg", "ec_es", "paper", "gl"),
    (5, (2, 2, 3), "hu", "ec", "tgv", "gl"),
    (6, (3, 1, 1), "dg", "ec_roe", "unit", "gl"),
    (7, (2, 1, 2), "hu", "ec", "tgv", "gl"),
    (3, (3, 2, 2), "hu", "ec", "tgv", "lgl"),
    (5, (2, 2, 2), "dg", "ec_roe", "unit", "lgl"),
]


@pytest.mark.parametrize("p,shape,c_kind,face_flux,kind,nodes", CASES)
def test_ranocha_residual_and_dudt_match_oracle(p, shape, c_kind, face_flux, kind, nodes):
    P, S, u = _case(shape, p, c_kind, face_flux, kind, nodes)
    ud = torch.from_numpy(u).cuda()
    R, D = torch.empty_like(ud), torch.empty_like(ud)
    S.residual_raw(ud, R)
    S.residual(ud, D)
    torch.cuda.synchronize()
    check_parity(R.cpu().numpy(), P.residual_abi(u), TOL, ulp_sensitivity(P.residual_abi, u), what="R")
    check_parity(D.cpu().numpy(), P.dudt_abi(u), TOL, ulp_sensitivity(P.dudt_abi, u), what="du/dt")


def test_ranocha_rk4_step_matches_oracle():
    P, S, u = _case((3, 2, 2), 4, "hu", "ec_roe", "tgv")
    dt = 2e-3
    u1 = P.rk4_step_abi(u, dt)
    ud = torch.from_numpy(u).cuda()
    S.rk_step(ud, dt=dt)
    torch.cuda.synchronize()
    du = u1 - u
    sens = ulp_sensitivity(lambda x: P.rk4_step_abi(x, dt) - x, u)
    check_parity(ud.cpu().numpy() - u, du, TOL, sens, difference_floor(u1, du), what="RK4 step")


@pytest.mark.parametrize("p,N", [(3, 3), (4, 2), (5, 2)])
def test_ranocha_entropy_rate_is_round_off(p, N):
    """EC volume and face fluxes: the semi-discrete entropy rate of the library's residual
    vanishes to the paper's 1e-13 and the conserved totals of R cancel."""
    P, S, u = _case((N, N, N), p, "hu", "ec", "tgv")
    d = S.entropy(torch.from_numpy(u).cuda())
    assert abs(d["entropy_rate"]) < 1e-13 * d["entropy_rate_scale"]
    o = P.diagnostics(P.to_internal(u))
    assert abs(d["entropy_rate_scale"] - o["entropy_rate_scale"]) < 1e-10 * o["entropy_rate_scale"]


def test_ranocha_differs_from_chandrashekar_on_the_gpu():
    """The context's flux choice reaches the kernels: the two fluxes give different du/dt."""
    from paper_2312_07725_gb300 import Solver
    P, S, u = _case((2, 2, 2), 3, "dg", "ec", "tgv")
    C = Solver(np.ascontiguousarray(make_ctrl((2, 2, 2), 3, "tgv")), (2, 2, 2), 3)
    C.set_metrics(*oracle_metrics_abi(P))
    ud = torch.from_numpy(u).cuda()
    a, b = torch.empty_like(ud), torch.empty_like(ud)
    S.residual(ud, a)
    C.residual(ud, b)
    torch.cuda.synchronize()
    assert float((a - b).abs().max()) > 1e-6 * float(b.abs().max())


@pytest.mark.parametrize("p,nq,shape,face_flux", [(2, 4, (2, 2, 2), "ec"), (3, 5, (3, 1, 2), "ec_roe")])
def test_ranocha_uncollocated_matches_oracle(p, nq, shape, face_flux):
    from paper_2312_07725_gb300 import Solver
    ctrl = wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv)
    P = UncollocatedProblem(ctrl, shape, p, nq=nq, c=c_hu(p), face_flux=face_flux, vol_flux="ranocha")
    S = Solver(np.ascontiguousarray(ctrl), shape, p, c=c_hu(p), face_flux=face_flux, nq=nq, vol_flux="ranocha")
    ne = P.mesh.n_el
    C = np.ascontiguousarray(np.moveaxis(P.C.reshape(3, 3, ne, nq ** 3), 2, 0).reshape(ne, 9, nq ** 3))
    J = np.ascontiguousarray(P.J.reshape(ne, nq ** 3))
    Cf = np.ascontiguousarray(np.moveaxis(P.geo["Cf"].reshape(3, 3, ne, nq * nq), 2, 0))
    S.set_metrics(C, J, Cf)
    u = np.ascontiguousarray(wl.perturbed_tgv_state(P.node_coords(ctrl)))
    ud = torch.from_numpy(u).cuda()
    D = torch.empty_like(ud)
    S.residual(ud, D)
    torch.cuda.synchronize()
    check_parity(D.cpu().numpy(), P.dudt_abi(u), TOL, ulp_sensitivity(P.dudt_abi, u), what="du^/dt")


def test_ranocha_context_rejects_what_it_does_not_support():
    from paper_2312_07725_gb300 import NSFRError, Solver
    ctrl = np.ascontiguousarray(make_ctrl((2, 2, 2), 2, "tgv"))
    with pytest.raises(NSFRError):
        Solver(ctrl, (2, 2, 2), 2, precision="fp32_bulk", vol_flux="ranocha")
    S = Solver(ctrl, (2, 2, 2), 2, vol_flux="ranocha")
    u = torch.from_numpy(np.ascontiguousarray(wl.perturbed_tgv_state(S.node_coords()))).cuda()
    with pytest.raises(NSFRError):
        S.vjp(u, torch.ones_like(u), torch.zeros_like(u))
