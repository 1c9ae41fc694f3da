"""nsfr_residual_static, the entry point for callers that must not allocate device
memory (an application whose memory manager owns the device, or code that cannot
take cudaMalloc's implicit synchronisation).  It must give the same du/dt as the
context-based nsfr_residual, call after call, leave the device's free memory
unchanged, report a bad mesh and recover from it on the next call, and refuse host
buffers and problems larger than its fixed working array before doing anything.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from tests._pairs import check_parity, oracle_metrics_abi, oracle_problem, state_for, ulp_sensitivity  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the FP64 parity bar used throughout the tests


def _rel(a, b):
    return float(torch.linalg.norm((a - b).ravel()) / torch.linalg.norm(b.ravel()))


def _setup(shape, p, c, face_flux):
    from paper_2312_07725_gb300 import Solver
    ctrl = wl.control_points(*shape, p, -np.pi, np.pi, wl.warp_tgv)
    S = Solver(ctrl, shape, p, c=c, face_flux=face_flux)
    C, J, Cf = (torch.from_numpy(x).cuda() for x in S.metrics())
    return S, C, J, Cf


@pytest.mark.parametrize("p,face_flux", [(2, "ec"), (3, "ec_roe"), (4, "ec_es")])
def test_static_entry_matches_nsfr_residual_on_consecutive_calls(p, face_flux):
    from paper_2312_07725_gb300 import nsfr
    shape, c = (3, 2, 4), 8.0e-4
    S, C, J, Cf = _setup(shape, p, c, face_flux)
    xyz = S.node_coords()
    states = [wl.perturbed_tgv_state(xyz, seed) for seed in (11, 12, 13)]
    free = []
    for u_np in states:  # calls in a row, different states
        u = torch.from_numpy(np.ascontiguousarray(u_np)).cuda()
        ref = torch.empty_like(u)
        S.residual(u, ref)
        out = torch.full_like(u, float("nan"))
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        nsfr.residual_static(u, C, J, Cf, shape, p, c=c, face_flux=face_flux, dudt=out)
        torch.cuda.synchronize()
        free.append(before - torch.cuda.mem_get_info()[0])
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < TOL
    # the first call on the device may load the library's module (which holds the
    # fixed array); later calls allocate nothing
    assert free[1:] == [0] * (len(states) - 1), free


def test_static_entry_matches_the_oracle():
    """du/dt of the entry point on the oracle's own metric terms against the oracle's du/dt,
    per variable and element-wise (tests._pairs.check_parity)."""
    from paper_2312_07725_gb300 import nsfr
    shape, p = (3, 2, 2), 4
    ctrl, P = oracle_problem(shape, p, "hu", "ec")
    u_np = state_for(P)
    C, J, Cf = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in oracle_metrics_abi(P))
    u = torch.from_numpy(u_np).cuda()
    out = torch.empty_like(u)
    for _ in range(2):
        out.fill_(float("nan"))
        nsfr.residual_static(u, C, J, Cf, shape, p, c=P.ops.c, face_flux="ec", dudt=out)
        torch.cuda.synchronize()
        check_parity(out.cpu().numpy(), P.dudt_abi(u_np), TOL, ulp_sensitivity(P.dudt_abi, u_np),
                     what="nsfr_residual_static du/dt")


def test_static_entry_reports_a_bad_mesh_then_recovers():
    from paper_2312_07725_gb300 import NSFRError, nsfr
    shape, p, c = (2, 2, 2), 3, 0.0
    S, C, J, Cf = _setup(shape, p, c, "ec")
    u = torch.from_numpy(np.ascontiguousarray(wl.perturbed_tgv_state(S.node_coords()))).cuda()
    out = torch.empty_like(u)
    with pytest.raises(NSFRError) as ei:
        nsfr.residual_static(u, C, -J, Cf, shape, p, c=c, dudt=out)  # J <= 0 everywhere
    assert ei.value.status == -2  # NSFR_ERR_MESH
    # the error word is cleared at the start of every call: a good mesh is fine again
    nsfr.residual_static(u, C, J, Cf, shape, p, c=c, dudt=out)
    ref = torch.empty_like(u)
    S.residual(u, ref)
    torch.cuda.synchronize()
    assert _rel(out, ref) < TOL


def test_static_entry_refuses_host_buffers():
    """A host (numpy) state is refused by the binding and, through the C ABI directly, by
    the library, before any launch: the output stays untouched."""
    from paper_2312_07725_gb300 import NSFRError, nsfr
    shape, p = (2, 2, 2), 2
    S, C, J, Cf = _setup(shape, p, 0.0, "ec")
    u_np = np.ascontiguousarray(wl.perturbed_tgv_state(S.node_coords()))
    out = torch.zeros(u_np.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(NSFRError) as ei:
        nsfr.residual_static(u_np, C, J, Cf, shape, p, dudt=out)
    assert ei.value.status == -1
    st = nsfr.lib().nsfr_residual_static(ctypes.c_void_p(u_np.ctypes.data), C.data_ptr(), J.data_ptr(),
                                         Cf.data_ptr(), *shape, p, 0.0, 0, 1.4, out.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == -1
    assert torch.count_nonzero(out).item() == 0


def test_static_entry_rejects_problems_beyond_its_array():
    from paper_2312_07725_gb300 import nsfr
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 64^3 elements at p = 4 need far more than NSFR_STATIC_SCRATCH_BYTES: refused by the
    # library's size check, called directly, before anything runs
    st = nsfr.lib().nsfr_residual_static(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 64, 64, 64, 4,
                                         0.0, 0, 1.4, x.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == -1
    assert torch.count_nonzero(x).item() == 0
