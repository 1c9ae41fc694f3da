"""GPU parity of the LGL-collocated variant (nsfr_setup with NSFR_NODES_LGL: the
solution and volume quadrature on Gauss-Lobatto-Legendre nodes) against the
oracle's LGL variant, with the same bars as the GL path: the library's metric
terms at 1e-12, R, du/dt and one RK4 step at 1e-12 with the oracle's metric
terms injected (per variable and element-wise as ``tests._pairs.check_parity`` states), the FP32-bulk du/dt within 1e-5, and the semi-discrete entropy
rate of the EC scheme at the paper's 1e-13.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._pairs import (check_parity, difference_floor, oracle_metrics_abi, oracle_problem, rel_l2,  # noqa: E402
                          state_for, ulp_sensitivity)

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _solver(ctrl, shape, P, precision="fp64"):
    from paper_2312_07725_gb300 import Solver
    return Solver(np.ascontiguousarray(ctrl), shape, P.p, p_geo=P.p_geo, c=P.ops.c, face_flux=P.face_flux,
                  gamma=P.gamma, precision=precision, nodes="lgl")


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("p", [1, 3, 4, 7])
def test_lgl_metrics_match_oracle(p):
    shape = (3, 2, 2)
    ctrl, P = oracle_problem(shape, p, nodes="lgl")
    S = _solver(ctrl, shape, P)
    C, J, Cf = S.metrics()
    Co, Jo, Cfo = oracle_metrics_abi(P)
    assert rel_l2(C, Co) < TOL and rel_l2(J, Jo) < TOL and rel_l2(Cf, Cfo) < TOL
    assert np.abs(S.node_coords() - P.node_coords()).max() < 1e-13 * np.pi


CASES = [
    (1, (2, 3, 2), "dg", "ec", "tgv"),
    (2, (3, 2, 5), "hu", "ec_roe", "unit"),
    (3, (3, 3, 2), "dg", "ec", "tgv"),
    (4, (3, 3, 1), "hu", "ec", "tgv"),       # 9 elements: ragged last CTA
    (5, (2, 2, 2), "dg", "ec_roe", "paper"),
    (7, (2, 1, 2), "hu", "ec", "tgv"),
]


@pytest.mark.parametrize("p,shape,c_kind,face_flux,kind", CASES)
def test_lgl_residual_and_dudt_match_oracle(p, shape, c_kind, face_flux, kind):
    ctrl, P = oracle_problem(shape, p, c_kind, face_flux, kind, nodes="lgl")
    S = _solver(ctrl, shape, P)
    S.set_metrics(*oracle_metrics_abi(P))
    u = state_for(P, kind)
    U = P.to_internal(u)
    ud = _dev(u)
    R = torch.empty_like(ud)
    D = torch.empty_like(ud)
    S.residual_raw(ud, R)
    S.residual(ud, D)
    torch.cuda.synchronize()
    check_parity(R.cpu().numpy(), P.to_abi(P.residual(U)), TOL, ulp_sensitivity(P.residual_abi, u), what="R")
    check_parity(D.cpu().numpy(), P.to_abi(P.dudt(U)), TOL, ulp_sensitivity(P.dudt_abi, u), what="du/dt")


def test_lgl_rk4_step_matches_oracle():
    shape, p = (3, 2, 2), 4
    ctrl, P = oracle_problem(shape, p, "hu", "ec_roe", nodes="lgl")
    S = _solver(ctrl, shape, P)
    S.set_metrics(*oracle_metrics_abi(P))
    u = state_for(P)
    dt = 2e-3
    u1_ref = P.rk4_step_abi(u, dt)
    ud = _dev(u)
    S.rk_step(ud, dt=dt)
    torch.cuda.synchronize()
    du_ref = u1_ref - u
    sens = ulp_sensitivity(lambda x: P.rk4_step_abi(x, dt) - x, u)
    check_parity(ud.cpu().numpy() - u, du_ref, TOL, sens, difference_floor(u1_ref, du_ref), what="RK4 step")


def test_lgl_entropy_rate_and_bulk_mode():
    shape, p = (4, 4, 4), 3
    ctrl, P = oracle_problem(shape, p, "hu", "ec", nodes="lgl")
    S = _solver(ctrl, shape, P)
    S.set_metrics(*oracle_metrics_abi(P))
    u = state_for(P)
    d = S.entropy(_dev(u))
    assert abs(d["entropy_rate"]) < 1e-13 * d["entropy_rate_scale"]
    for prec in ("fp32_bulk", "fp32_bulk_ff"):
        Sb = _solver(ctrl, shape, P, precision=prec)
        Sb.set_metrics(*oracle_metrics_abi(P))
        D = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        Sb.residual(_dev(u), D)
        torch.cuda.synchronize()
        assert rel_l2(D.cpu().numpy(), P.dudt_abi(u)) < 1e-5, prec


def test_kinetic_energy_lemma_holds_for_the_library_residual(monkeypatch):
    """The kinetic-energy lemma on the library's LGL residual: v_KE . (R - R_p) = 0, with R the
    library's residual and R_p the oracle's residual of the pressure part p_hat n of the
    two-point flux alone (R is linear in the flux function).  On GL the same quantity is
    O(1e-5) of its scale (see tests/test_oracle_lgl.py)."""
    from oracle import physics
    from tests.test_oracle_lgl import pressure_part
    shape, p = (2, 2, 2), 4
    ctrl, P = oracle_problem(shape, p, "hu", "ec", nodes="lgl")
    S = _solver(ctrl, shape, P)
    S.set_metrics(*oracle_metrics_abi(P))
    u = state_for(P)
    R = torch.empty(u.shape, dtype=torch.float64, device="cuda")
    S.residual_raw(_dev(u), R)
    torch.cuda.synchronize()
    monkeypatch.setattr(physics, "chandrashekar", pressure_part)
    Rp = P.to_abi(P.residual(P.to_internal(u)))
    Rnp = R.cpu().numpy() - Rp
    vel = u[:, 1:4] / u[:, 0:1]
    terms = -0.5 * np.sum(vel * vel, axis=1) * Rnp[:, 0] + np.sum(vel * Rnp[:, 1:4], axis=1)
    assert abs(terms.sum()) < 1e-11 * np.abs(terms).sum()
