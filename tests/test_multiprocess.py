"""The multi-process path of bench.py on the CPU (gloo, world size 2).

Under torchrun every rank runs an independent replica of the workload (weak
scaling, no data-path collective); the ranks meet only in the barriers around
the timed region and in the max-over-ranks reduction of the timings, and rank 0
alone prints the JSON line.  These tests run that plumbing with the gloo
backend: the reduction itself, and the reference arm (the oracle, which needs
no GPU) launched exactly as the driver launches the bench.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(impl="reference")
    r, w, dist = bench.dist_init(args)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, 1.5 + r)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "ws": w, "max": m, "backend": dist.get_backend()}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_with_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [x["rank"] for x in res] == [0, 1]
    assert all(x["ws"] == 2 and x["backend"] == "gloo" for x in res)
    assert all(x["max"] == 2.5 for x in res)  # the slowest rank's time on every rank


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--p", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


# --------------------------------------------------------------------------
# the z-slab decomposition's host logic (paper_2312_07725_gb300.slab)
# --------------------------------------------------------------------------
def test_extended_layers_take_the_neighbour_layers():
    import math

    import workloads as wl
    from paper_2312_07725_gb300.slab import extended_layers, slab_range
    shape = (3, 2, 6)
    ctrl = wl.control_points(*shape, 2, -math.pi, math.pi, wl.warp_tgv)
    L = 6
    for ws in (1, 2, 3):
        for r in range(ws):
            z0, nz = slab_range(6, ws, r)
            ext = extended_layers(ctrl, shape, z0, nz)
            assert ext.shape[0] == (nz + 2) * L
            for k in range(nz + 2):
                z = (z0 - 1 + k) % 6
                assert np.array_equal(ext[k * L:(k + 1) * L], ctrl[z * L:(z + 1) * L])
    with pytest.raises(ValueError):
        slab_range(7, 2, 0)


def _halo_rank(rank, ws, port, out_dir, late):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import time

    import torch
    import torch.distributed as dist
    from paper_2312_07725_gb300.slab import DistExchanger, HaloTimeout
    dist.init_process_group("gloo")
    L, nz = 4, 3
    t = torch.zeros(((nz + 2) * L, 5, 8), dtype=torch.float64)
    for k in range(nz):  # interior layer k of rank r holds 100 r + k
        t[(k + 1) * L:(k + 2) * L] = 100.0 * rank + k
    res = {"rank": rank}
    ex = DistExchanger(dist, rank, ws, timeout_s=2.0 if late else 60.0)
    if late and rank == 1:
        time.sleep(6.0)  # a late neighbour: rank 0 must give up with HaloTimeout
    try:
        ex.exchange(t, L)
        res["top"] = float(t[-L:].mean())
        res["bottom"] = float(t[:L].mean())
        res["max"] = ex.global_max(float(rank) + 0.5)
    except HaloTimeout:
        res["timeout"] = True
    with open(os.path.join(out_dir, f"halo{rank}.json"), "w") as f:
        json.dump(res, f)
    os._exit(0)  # no collective teardown after a deliberately broken exchange


@pytest.mark.parametrize("ws", [2, 3])
def test_halo_exchange_fills_the_ghost_layers_with_gloo(tmp_path, ws):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_halo_rank, args=(r, ws, port, str(tmp_path), False)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    res = [json.load(open(tmp_path / f"halo{r}.json")) for r in range(ws)]
    for r, x in enumerate(res):
        above, below = (r + 1) % ws, (r - 1) % ws
        assert x["top"] == 100.0 * above + 0            # first interior layer of the rank above
        assert x["bottom"] == 100.0 * below + 2         # last interior layer of the rank below
        assert x["max"] == ws - 1 + 0.5


def test_a_late_neighbour_raises_halo_timeout(tmp_path):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_halo_rank, args=(r, 2, port, str(tmp_path), True)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    r0 = json.load(open(tmp_path / "halo0.json"))
    assert r0.get("timeout") is True
