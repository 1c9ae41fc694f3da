"""The z-slab decomposition on the GPU against the undecomposed solver, and the host-state
RK step (copies in z-chunks overlapped with kernels) against the device-state one.

A periodic block cut into ws slabs, each with one ghost element layer on either
side filled by the halo exchange before every RK stage, must reproduce the
undecomposed RK4 steps element by element: every kernel computes an element
from its own data and its face neighbours' only, so the interiors agree bit for
bit, and so does the CFL step (the max wave speed over the ranks).  The slabs
run in one process (``LocalSlabs``, copies between them) and, for the
torch.distributed exchanger, as two processes on this one GPU with gloo moving
the layers through host memory (no kernel waits on another process: the ranks
meet on the host between stages).
"""
import json
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mesh(shape, p, kind="tgv"):
    if kind == "tgv":
        return np.ascontiguousarray(wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv))
    return np.ascontiguousarray(wl.control_points(*shape, p, 0.0, 1.0, wl.warp_unit))


def _global_run(ctrl, shape, p, steps, kw, kind="tgv"):
    from paper_2312_07725_gb300 import Solver
    S = Solver(ctrl, shape, p, **kw)
    xs = S.node_coords()
    u0 = wl.perturbed_tgv_state(xs) if kind == "tgv" else wl.perturbed_density_wave_state(xs)
    u0 = np.ascontiguousarray(u0)
    u = torch.from_numpy(u0).cuda()
    dts = [S.rk_step(u, cfl=0.1) for _ in range(steps)]
    torch.cuda.synchronize()
    return u0, u.cpu().numpy(), dts


CASES = [
    ((3, 2, 6), 3, {}, "tgv"),
    ((2, 3, 4), 4, {"c": 0.01}, "tgv"),
    ((2, 2, 6), 2, {"face_flux": "ec_roe"}, "unit"),
    ((2, 2, 4), 3, {"face_flux": "ec_es", "nodes": "lgl"}, "unit"),
    ((3, 1, 4), 4, {"precision": "fp32_bulk"}, "tgv"),
    ((2, 3, 4), 4, {"precision": "fp32_bulk_ff"}, "tgv"),
    ((2, 2, 4), 2, {"nq": 4}, "tgv"),             # uncollocated, overintegrated
]


@pytest.mark.parametrize("shape,p,kw,kind", CASES)
@pytest.mark.parametrize("ws", [1, 2])
def test_local_slabs_reproduce_the_undecomposed_steps(shape, p, kw, kind, ws):
    from paper_2312_07725_gb300.slab import LocalSlabs
    ctrl = _mesh(shape, p, kind)
    steps = 2
    u0, ug, dts = _global_run(ctrl, shape, p, steps, kw, kind)
    D = LocalSlabs(ctrl, shape, p, ws, **kw)
    us = [s.extend(u0) for s in D.slabs]
    dd = [D.step(us, cfl=0.1) for _ in range(steps)]
    torch.cuda.synchronize()
    assert dd == dts
    L = D.slabs[0].layer
    for s, u in zip(D.slabs, us):
        ref = ug[s.z0 * L:(s.z0 + s.nz) * L]
        assert np.array_equal(s.interior(u).cpu().numpy(), ref)


def test_three_local_slabs_of_a_deeper_block():
    from paper_2312_07725_gb300.slab import LocalSlabs
    shape, p = (2, 2, 9), 3
    ctrl = _mesh(shape, p)
    u0, ug, dts = _global_run(ctrl, shape, p, 3, {})
    D = LocalSlabs(ctrl, shape, p, 3)
    us = [s.extend(u0) for s in D.slabs]
    dd = [D.step(us, cfl=0.1) for _ in range(3)]
    torch.cuda.synchronize()
    assert dd == dts
    L = D.slabs[0].layer
    got = np.concatenate([s.interior(u).cpu().numpy() for s, u in zip(D.slabs, us)])
    assert got.shape == ug.shape and np.array_equal(got, ug)
    assert D.slabs[1].ctrl.shape[0] == (3 + 2) * L


def _slab_rank(rank, ws, port, out_dir, shape, p, steps):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import workloads as wl
    from paper_2312_07725_gb300 import Solver
    from paper_2312_07725_gb300.slab import DistExchanger, Slab
    dist.init_process_group("gloo")
    ctrl = np.ascontiguousarray(wl.control_points(*shape, p, -math.pi, math.pi, wl.warp_tgv))
    xs = Solver(ctrl, shape, p).node_coords()
    u0 = np.ascontiguousarray(wl.perturbed_tgv_state(xs))
    s = Slab(ctrl, shape, p, rank, ws, DistExchanger(dist, rank, ws, timeout_s=120.0))
    u = s.extend(u0)
    dts = [s.step(u, cfl=0.1) for _ in range(steps)]
    torch.cuda.synchronize()
    np.save(os.path.join(out_dir, f"slab{rank}.npy"), s.interior(u).cpu().numpy())
    with open(os.path.join(out_dir, f"slab{rank}.json"), "w") as f:
        json.dump({"dts": dts, "z0": s.z0, "nz": s.nz}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_process_slabs_with_the_distributed_exchanger(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    shape, p, steps = (2, 3, 4), 3, 2
    ctrl = _mesh(shape, p)
    _, ug, dts = _global_run(ctrl, shape, p, steps, {})
    mp.start_processes(_slab_rank, args=(2, port, str(tmp_path), shape, p, steps), nprocs=2,
                       join=True, start_method="spawn")
    L = shape[0] * shape[1]
    for r in range(2):
        meta = json.load(open(tmp_path / f"slab{r}.json"))
        assert meta["dts"] == dts
        got = np.load(tmp_path / f"slab{r}.npy")
        assert np.array_equal(got, ug[meta["z0"] * L:(meta["z0"] + meta["nz"]) * L])


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk", "fp32_bulk_ff"])
def test_rk_stage_element_range_updates_only_its_elements(precision):
    from paper_2312_07725_gb300 import NSFRError, Solver
    shape, p = (2, 3, 3), 3
    ctrl = _mesh(shape, p)
    S = Solver(ctrl, shape, p, precision=precision)
    u0 = torch.from_numpy(np.ascontiguousarray(wl.perturbed_tgv_state(S.node_coords()))).cuda()
    L, dt = 6, 1e-3
    full = [torch.empty_like(u0) for _ in range(3)]  # u, ustage, acc of the whole-mesh stages
    full[0].copy_(u0)
    seen = []
    for st in range(4):
        S.rk_stage(*full, st, dt)
        seen.append([t.clone() for t in full])
    b, e = L, 2 * L + 3  # a range that is not a whole layer
    # stage 0: reads u only
    us, acc = torch.full_like(u0, 7.0), torch.full_like(u0, 7.0)
    u = u0.clone()
    S.rk_stage(u, us, acc, 0, dt, elements=(b, e))
    torch.cuda.synchronize()
    assert torch.equal(us[b:e], seen[0][1][b:e]) and torch.equal(acc[b:e], seen[0][2][b:e])
    assert bool((us[:b] == 7.0).all()) and bool((us[e:] == 7.0).all()) and bool((acc[e:] == 7.0).all())
    # stage 3 from the whole-mesh stage-2 arrays: u changes inside the range only
    u, us, acc = (t.clone() for t in seen[2])
    S.rk_stage(u, us, acc, 3, dt, elements=(b, e))
    torch.cuda.synchronize()
    assert torch.equal(u[b:e], seen[3][0][b:e])
    assert torch.equal(u[:b], seen[2][0][:b]) and torch.equal(u[e:], seen[2][0][e:])
    # an empty range launches nothing and changes nothing
    S.rk_stage(u, us, acc, 3, dt, elements=(4, 4))
    torch.cuda.synchronize()
    assert torch.equal(u[:b], seen[2][0][:b])
    with pytest.raises(NSFRError):
        S.rk_stage(u, us, acc, 0, dt, elements=(3, S.n_el + 1))


@pytest.mark.parametrize("shape,p,kw", [
    ((2, 3, 11), 3, {}),                                  # 11 layers in 8 copy chunks
    ((3, 2, 5), 4, {"precision": "fp32_bulk"}),
    ((2, 3, 5), 3, {"precision": "fp32_bulk_ff"}),
    ((2, 2, 3), 2, {"face_flux": "ec_roe", "nodes": "lgl"}),
    ((2, 2, 9), 3, {"c": 1e-3, "source": True}),
])
def test_host_state_step_equals_device_state_step(shape, p, kw):
    """nsfr_rk_step on a host state copies it in z-chunks overlapped with the face-state
    pass and copies stage 3's chunks back while the next is computed: the result, the
    CFL step and the context's time equal those of the step on a device state."""
    from paper_2312_07725_gb300 import Solver
    kw = dict(kw)
    source = kw.pop("source", False)
    ctrl = (np.ascontiguousarray(wl.control_points(*shape, p, -1.0, 1.0, wl.WARPS["mms"])) if source
            else _mesh(shape, p))
    A = Solver(ctrl, shape, p, **kw)
    B = Solver(ctrl, shape, p, **kw)
    xs = A.node_coords()
    u0 = np.ascontiguousarray(wl.manufactured_state(xs, 0.0) if source else wl.perturbed_tgv_state(xs))
    if source:
        A.set_source("manufactured", 0.0)
        B.set_source("manufactured", 0.0)
    ud = torch.from_numpy(u0.copy()).cuda()
    uh = torch.from_numpy(u0.copy()).pin_memory()
    for k in range(3):
        if k < 2:
            da, db = A.rk_step(ud, cfl=0.1), B.rk_step(uh.numpy(), cfl=0.1)
        else:
            da, db = A.rk_step(ud, dt=1e-3), B.rk_step(uh.numpy(), dt=1e-3)
        assert da == db
    torch.cuda.synchronize()
    assert np.array_equal(ud.cpu().numpy(), uh.numpy())
    assert A.time == B.time
    # a pageable numpy state takes the same path
    un = u0.copy()
    A2 = Solver(ctrl, shape, p, **kw)
    if source:
        A2.set_source("manufactured", 0.0)
    A2.rk_step(un, cfl=0.1)
    ud2 = torch.from_numpy(u0.copy()).cuda()
    B2 = Solver(ctrl, shape, p, **kw)
    if source:
        B2.set_source("manufactured", 0.0)
    B2.rk_step(ud2, cfl=0.1)
    torch.cuda.synchronize()
    assert np.array_equal(un, ud2.cpu().numpy())
