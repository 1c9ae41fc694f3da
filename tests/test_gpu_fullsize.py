"""Parity at the benchmark's full size: 64^3 warped Taylor-Green elements at p = 4
(32.8M nodes), in the launch configuration bench.py times.

* sampled outputs: 4^3-element blocks, each computed by the oracle on a 6^3-element
  patch around it (the halo supplies the neighbours' face states);
    - the library's metric terms on the patch against the oracle's (1e-12);
    - du/dt of the block with the oracle's metric terms injected into the library
      for the patch (nsfr_set_metrics).  At this size the residual itself is
      ill-conditioned: the oracle alone moves du/dt by ~3e-12 for a 1 ulp change
      of the state.  The bar is max(1e-12, 4 x the oracle's measured 1-ulp sensitivity
      (state and elementary functions, ``tests._pairs.ulp_sensitivity``)), for all
      five variables together and, in L2 and element-wise, for each variable
      (``tests._pairs.check_parity``);
* properties that hold at any size: conservation (sum R = 0), the entropy rate of
  the EC scheme and free-stream preservation.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import geometry  # noqa: E402
from oracle.operators1d import Ops1D, c_hu  # noqa: E402
from oracle.problem import Problem  # noqa: E402
from tests._pairs import check_parity, rel_l2, ulp_sensitivity  # noqa: E402

pytestmark = pytest.mark.gpu
NE, P_DEG = 64, 4


@pytest.fixture(scope="module")
def full():
    from paper_2312_07725_gb300 import Solver
    ctrl = wl.tgv_mesh(NE, P_DEG)
    S = Solver(ctrl, (NE,) * 3, P_DEG, c=c_hu(P_DEG))
    ops = Ops1D(P_DEG, c_hu(P_DEG))
    X = geometry.node_coordinates(ctrl, P_DEG, ops)           # oracle's coordinates
    xyz = np.ascontiguousarray(np.moveaxis(X, 0, 1).reshape(NE ** 3, 3, -1))
    u = np.ascontiguousarray(wl.perturbed_tgv_state(xyz))
    ud = torch.from_numpy(u).cuda()
    D = torch.empty_like(ud)
    S.residual(ud, D)
    R = torch.empty_like(ud)
    S.residual_raw(ud, R)
    torch.cuda.synchronize()
    return {"ctrl": ctrl, "S": S, "u": u, "ud": ud, "D": D.cpu().numpy(), "R": R}


def _patch(full, ex0, ey0, ez0):
    """Oracle on the 6^3 patch whose interior 4^3 block starts at (ex0, ey0, ez0)."""
    rng = [(np.arange(-1, 5) + e0) % NE for e0 in (ex0, ey0, ez0)]
    ez, ey, ex = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    idx = (ex + NE * (ey + NE * ez)).ravel()
    P = Problem(full["ctrl"][idx], (6, 6, 6), P_DEG, c=c_hu(P_DEG))
    inner = np.zeros((6, 6, 6), bool)
    inner[1:5, 1:5, 1:5] = True
    return idx, inner.ravel(), P


@pytest.mark.parametrize("corner", [(0, 0, 0), (30, 61, 17), (62, 7, 45)])
def test_sampled_blocks_match_oracle(full, corner):
    from tests._pairs import oracle_metrics_abi
    idx, inner, P = _patch(full, *corner)
    S = full["S"]
    C, J, Cf = S.metrics()
    Co, Jo, Cfo = oracle_metrics_abi(P)
    assert rel_l2(C[idx], Co) < 1e-12
    assert rel_l2(J[idx], Jo) < 1e-12
    assert rel_l2(Cf[idx], Cfo) < 1e-12
    # du/dt with identical metric terms on the patch
    C2, J2, Cf2 = C.copy(), J.copy(), Cf.copy()
    C2[idx], J2[idx], Cf2[idx] = Co, Jo, Cfo
    try:
        S.set_metrics(C2, J2, Cf2)
        D = torch.empty_like(full["ud"])
        S.residual(full["ud"], D)
        torch.cuda.synchronize()
        up = full["u"][idx]
        Dref = P.dudt_abi(up)[inner]
        sens = ulp_sensitivity(lambda x: P.dudt_abi(x)[inner], up)
        check_parity(D.cpu().numpy()[idx[inner]], Dref, 1e-12, sens, what=f"du/dt block {corner}", sens_all=True)
    finally:
        S.set_metrics(C, J, Cf)


def test_conservation_and_entropy_at_full_size(full):
    S = full["S"]
    d = S.entropy(full["ud"])
    scale = full["R"].abs().sum(dim=(0, 2)).cpu().numpy()
    for k in range(5):
        assert abs(d["sum_R"][k]) < 1e-13 * scale[k]
    assert abs(d["entropy_rate"]) < 1e-13 * d["entropy_rate_scale"]


def test_free_stream_at_full_size(full):
    """Free-stream preservation at full size, measured on R (before the division by
    w J): at the round-off level of the fluxes, and within 10x of the oracle's own
    free-stream residual on a sampled patch of the same mesh."""
    S = full["S"]
    xyz = S.node_coords()
    fs = torch.from_numpy(np.ascontiguousarray(wl.free_stream_state(xyz))).cuda()
    R = torch.empty_like(fs)
    S.residual_raw(fs, R)
    torch.cuda.synchronize()
    C, _, _ = S.metrics()
    f_scale = fs.abs().max().item() * np.abs(C).max()
    assert R.abs().max().item() < 1e-13 * f_scale
    rng = [(np.arange(-1, 5) + 62) % NE for _ in range(3)]   # seams in x, y and z
    ez, ey, ex = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    idx = (ex + NE * (ey + NE * ez)).ravel()
    P = Problem(full["ctrl"][idx], (6, 6, 6), P_DEG, c=c_hu(P_DEG))
    inner = np.zeros((6, 6, 6), bool)
    inner[1:5, 1:5, 1:5] = True
    R_or = P.residual_abi(np.ascontiguousarray(wl.free_stream_state(P.node_coords())))[inner.ravel()]
    R_gpu = R.cpu().numpy()[idx[inner.ravel()]]
    assert np.abs(R_gpu).max() < 10 * np.abs(R_or).max() + 1e-20
