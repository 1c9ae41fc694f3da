"""GPU parity of the volume source (nsfr_set_source, the manufactured solution of Sec.
"Manufactured Solution Convergence") against the oracle's ManufacturedProblem.

Bars as for the rest of the FP64 path: du/dt with the source and RK4 steps with the
stage times t, t + dt/2, t + dt/2, t + dt at 1e-12 with the oracle's metric terms
injected (per variable and element-wise as ``tests._pairs.check_parity`` states); nsfr_residual_raw stays the source-free R; the stage entry point gives the
same steps and time; FP32-bulk within 1e-5 of FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import manufactured as mm  # noqa: E402
from oracle.operators1d import c_hu  # noqa: E402
from tests._pairs import check_parity, difference_floor, oracle_metrics_abi, rel_l2, ulp_sensitivity  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _case(shape, p, c_kind="dg", face_flux="ec_roe", nodes="gl", precision="fp64", metrics=True):
    from paper_2312_07725_gb300 import Solver
    c = 0.0 if c_kind == "dg" else c_hu(p)
    ctrl = np.ascontiguousarray(wl.control_points(*shape, p, -1.0, 1.0, wl.WARPS["mms"]))
    P = mm.ManufacturedProblem(ctrl, shape, p, c=c, face_flux=face_flux, nodes=nodes)
    S = Solver(ctrl, shape, p, c=c, face_flux=face_flux, nodes=nodes, precision=precision)
    if metrics:
        S.set_metrics(*oracle_metrics_abi(P))
    xyz = S.node_coords()
    assert np.abs(xyz - P.node_coords()).max() < 1e-13
    return P, S, xyz


CASES = [
    ((3, 2, 2), 2, "dg", "ec_roe", "gl"),
    ((2, 2, 3), 3, "hu", "ec", "gl"),
    ((2, 3, 2), 4, "dg", "ec_roe", "lgl"),
    ((3, 3, 1), 5, "hu", "ec_roe", "gl"),     # 9 elements: ragged last CTA
    ((2, 1, 2), 3, "dg", "ec_es", "gl"),
]


@pytest.mark.parametrize("shape,p,c_kind,face_flux,nodes", CASES)
def test_dudt_with_the_manufactured_source_matches_oracle(shape, p, c_kind, face_flux, nodes):
    P, S, xyz = _case(shape, p, c_kind, face_flux, nodes)
    t = 0.3
    f = np.stack(wl.smooth_perturbation(xyz, period=2.0), axis=-2)  # a few % per component
    u = np.ascontiguousarray(wl.manufactured_state(xyz, t) * (1.0 + f))
    S.set_source("manufactured", t)
    ud = torch.from_numpy(u).cuda()
    D, R = torch.empty_like(ud), torch.empty_like(ud)
    S.residual(ud, D)
    S.residual_raw(ud, R)
    torch.cuda.synchronize()
    def dudt_t(x):
        return P.to_abi(P.dudt_t(P.to_internal(x), t))

    def res(x):
        return P.to_abi(P.residual(P.to_internal(x)))

    def dudt(x):
        return P.to_abi(P.dudt(P.to_internal(x)))

    check_parity(D.cpu().numpy(), dudt_t(u), TOL, ulp_sensitivity(dudt_t, u), what="du/dt with source")
    check_parity(R.cpu().numpy(), res(u), TOL, ulp_sensitivity(res, u), what="R (no source)")
    assert S.time == t
    # without the source again: the plain du/dt
    S.set_source("none", t)
    S.residual(ud, D)
    torch.cuda.synchronize()
    check_parity(D.cpu().numpy(), dudt(u), TOL, ulp_sensitivity(dudt, u), what="du/dt")


@pytest.mark.parametrize("nodes", ["gl", "lgl"])
def test_rk4_steps_with_the_source_match_oracle_and_advance_time(nodes):
    P, S, xyz = _case((2, 2, 2), 3, "hu", "ec_roe", nodes)
    t0, dt = 0.1, 4e-3
    u = np.ascontiguousarray(wl.manufactured_state(xyz, t0))
    S.set_source("manufactured", t0)
    ud = torch.from_numpy(u).cuda()
    S.rk_step(ud, dt=dt)
    S.rk_step(ud, dt=dt)
    torch.cuda.synchronize()
    def two_steps(x):
        return P.to_abi(P.rk4_step_t(P.rk4_step_t(P.to_internal(x), t0, dt), t0 + dt, dt))

    ref = two_steps(u)
    du = ref - u
    allv, per = difference_floor(ref, du)  # two steps: twice the rounding of one
    floor = (2 * allv, [(2 * a, 2 * b) for a, b in per])
    sens = ulp_sensitivity(lambda x: two_steps(x) - x, u)
    check_parity(ud.cpu().numpy() - u, du, TOL, sens, floor, what="two RK4 steps")
    assert abs(S.time - (t0 + 2 * dt)) < 1e-15


def test_stage_entry_point_equals_rk_step_with_the_source():
    _, S, xyz = _case((2, 2, 2), 2, "dg", "ec_roe", "gl", metrics=False)
    u0 = torch.from_numpy(np.ascontiguousarray(wl.manufactured_state(xyz, 0.0))).cuda()
    a = u0.clone()
    S.set_source("manufactured", 0.25)
    S.rk_step(a, dt=5e-3)
    t_a = S.time
    b, us, acc = u0.clone(), torch.empty_like(u0), torch.empty_like(u0)
    S.set_source("manufactured", 0.25)
    for st in range(4):
        S.rk_stage(b, us, acc, st, 5e-3)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and S.time == t_a == 0.25 + 5e-3


@pytest.mark.parametrize("precision", ["fp32_bulk", "fp32_bulk_ff"])
def test_fp32_bulk_with_the_source_is_within_1e5_of_fp64(precision):
    _, S64, xyz = _case((3, 2, 2), 4, "hu", "ec_roe", "gl", metrics=False)
    _, S32, _ = _case((3, 2, 2), 4, "hu", "ec_roe", "gl", precision=precision, metrics=False)
    u = torch.from_numpy(np.ascontiguousarray(wl.manufactured_state(xyz, 0.7))).cuda()
    D64, D32 = torch.empty_like(u), torch.empty_like(u)
    for S, D in ((S64, D64), (S32, D32)):
        S.set_source("manufactured", 0.7)
        S.residual(u, D)
    torch.cuda.synchronize()
    assert rel_l2(D32.cpu().numpy(), D64.cpu().numpy()) < 1e-5


def test_source_rejections():
    import ctypes

    from paper_2312_07725_gb300 import NSFRError, Solver
    _, S, xyz = _case((2, 2, 2), 2, face_flux="ec", metrics=False)
    assert S._lib.nsfr_set_source(S._h, 7, 0.0) != 0
    assert S._lib.nsfr_set_source(S._h, 1, float("nan")) != 0
    S.set_source("manufactured", 0.0)
    u = torch.from_numpy(np.ascontiguousarray(wl.manufactured_state(xyz, 0.0))).cuda()
    xb = torch.zeros((S.n_el, 27, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(NSFRError):
        S.vjp(u, torch.ones_like(u), torch.zeros_like(u), xb)
    ctrl = np.ascontiguousarray(wl.mms_mesh(2, 2))
    Su = Solver(ctrl, (2, 2, 2), 2, nq=4)
    with pytest.raises(NSFRError):
        Su.set_source("manufactured", 0.0)
    t = ctypes.c_double(-1.0)
    assert S._lib.nsfr_get_time(S._h, ctypes.byref(t)) == 0 and t.value == 0.0


def test_manufactured_solution_converges_on_the_warped_mesh():
    """The paper's grid study on its warped mesh of [-1, 1]^3 (beta = 1/50), p = 2 and 3,
    CFL 0.2, to t = 0.5: density and pressure errors fall at about p + 1 between
    16^3 and 32^3 elements."""
    from paper_2312_07725_gb300.experiments import manufactured_convergence
    for p in (2, 3):
        r = manufactured_convergence(p, [16, 32], tf=0.5)
        o_rho, o_p = r["orders_rho_p"][-1]
        assert o_rho > p + 0.6 and o_p > p + 0.6, r
