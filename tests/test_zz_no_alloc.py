"""nsfr_residual_static, the entry point for callers that must not allocate device
memory (an application whose memory manager owns the device, or code that cannot
take cudaMalloc's implicit synchronisation).  It must give the same du/dt as the
context-based nsfr_residual, call after call, and refuse problems larger than its
fixed working array before doing anything.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the FP64 parity bar used throughout the tests


def _rel(a, b):
    return float(torch.linalg.norm((a - b).ravel()) / torch.linalg.norm(b.ravel()))


def test_static_entry_matches_nsfr_residual_on_consecutive_calls():
    from paper_2312_07725_gb300 import Solver, nsfr
    shape, p, c = (3, 2, 4), 3, 8.0e-4
    ctrl = wl.control_points(*shape, p, -np.pi, np.pi, wl.warp_tgv)
    S = Solver(ctrl, shape, p, c=c, face_flux="ec_roe")
    xyz = S.node_coords()
    C, J, Cf = (torch.from_numpy(x).cuda() for x in S.metrics())
    states = [wl.perturbed_tgv_state(xyz, seed) for seed in (11, 12)]
    for u_np in states:  # two calls in a row, different states
        u = torch.from_numpy(np.ascontiguousarray(u_np)).cuda()
        ref = torch.empty_like(u)
        S.residual(u, ref)
        out = torch.full_like(u, float("nan"))
        nsfr.residual_static(u, C, J, Cf, shape, p, c=c, face_flux="ec_roe", dudt=out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < TOL


def test_static_entry_rejects_problems_beyond_its_array():
    from paper_2312_07725_gb300 import NSFRError, nsfr
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 64^3 elements at p = 4 need far more than NSFR_STATIC_SCRATCH_BYTES
    with pytest.raises(NSFRError) as ei:
        nsfr.residual_static(x, x, x, x, (64, 64, 64), 4, dudt=x)
    assert ei.value.status == -1
    assert torch.count_nonzero(x).item() == 0
