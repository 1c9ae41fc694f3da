"""Benchmark of the NSFR-EC residual hot path on GB300.

Workload (default): the inviscid Taylor-Green vortex on the warped periodic
cube [-pi, pi]^3, 64^3 hexahedra at p = 4 (32,768,000 GL nodes, 5 variables),
Chandrashekar EC volume and face flux, positive FR parameter c (c_HU, see
tests/golden/c_values.json: the paper does not print c_+), classic RK4 at
CFL 0.1.  One bench "step" is one RK4 step = four RK stages; every stage is
the whole hot path (entropy-projected face states, volume/hybrid/surface flux
differencing, weight-adjusted mass inverse, stage update), and the step also
computes its CFL time step from the maximum wave speed.

Metric: GDOF/s per RK stage = (nodes x stages) / time / 1e9, DOF = one
solution node (the paper's count); x5 per conserved component is printed
separately.  The state (1.3 GB) is larger than L2 (129 MB), so no L2 flush is
needed between steps.

With --decomp slab the ranks hold the z-slabs of a periodic stack of N copies
of the mesh (one copy per rank, one ghost element layer per side) and exchange
the boundary layers before every stage; at N = 1 the slab exchanges with
itself, which measures the ghost-layer and exchange overhead on one GPU.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                        [--modes both|fp64] [--n-el E] [--p P] [--nq Q]
                        [--decomp replicas|slab]
"""
from __future__ import annotations

import argparse
import functools
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

# Algorithmic FP64 flops of the volume kernel (an FMA counts 2, a reciprocal or
# division 1): per two-point flux evaluation (the Chandrashekar flux with its
# two log means) and per accumulation of one flux into two residual entries
FLOPS_PER_FLUX = 55
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one volume_kernel<5>
# launch per element, from an ncu --set full capture at 24^3 elements (813.1 + 125.2 MB
# for 13,824 elements, the kernel as it stands: profiles/volume_kernel_p4_tgv24.md; every
# buffer the kernel touches scales with the element count)
VOLUME_DRAM_BYTES_PER_ELEMENT = {4: (813.061120e6 + 125.166336e6) / 13824}
FLOPS_PER_ACC = 20
# the same with Ranocha's pressure terms: the two log means (22), u_bar (3), u_bar.n,
# u_a.n / 2 and u_a.u_b / 4 (15), F_rho (1), p_bar (2), 1/(2 (gamma-1) beta_ln) (2), the
# momentum flux (9) and the energy flux (8)
FLOPS_PER_FLUX_RANOCHA = 62
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--modes", default="both", choices=["both", "fp64"],
                    help="both: the FP64 line plus the fp32_bulk and fp32_bulk_ff objects; fp64: skip them")
    ap.add_argument("--n-el", type=int, default=64)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--cfl", type=float, default=0.1)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the VJP and diagnostics timings")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="replicas: every rank steps its own copy of the mesh; slab: the ranks "
                         "hold the z-slabs of ws stacked copies (halo exchange every stage)")
    ap.add_argument("--nq", type=int, default=None,
                    help="uncollocated scheme: solution on the p+1 Lobatto nodes, NQ Gauss-Legendre "
                         "quadrature points per direction (FP64 only)")
    return ap.parse_args()


def c_value(p):
    with open(os.path.join(ROOT, "tests", "golden", "c_values.json")) as f:
        return float(json.load(f)["c_hu"][str(p)])


def workload_config(args, ws):
    N = args.n_el
    if args.decomp == "slab":
        par = (f"z-slabs: rank r holds layers {N}r..{N}r+{N - 1} of a periodic {N}x{N}x{N * ws} stack "
               f"of {ws} copies, one ghost layer per side, halo exchange before every stage, "
               "all-reduce max for dt")
    else:
        par = f"{ws} independent replica(s), no data-path collective"
    n = args.p + 1
    nodes = args.n_el ** 3 * n ** 3
    quad = "GL collocated" if args.nq is None else f"LGL solution, {args.nq} GL quadrature points per direction"
    return {
        "workload": f"tgv_warped_{args.n_el}^3_p{args.p}" + ("" if args.nq is None else f"_lgl_nq{args.nq}"),
        "elements": args.n_el ** 3, "p": args.p, "nodes": nodes, "variables": 5,
        "c": c_value(args.p), "c_kind": "c_HU (stand-in for c_+)", "volume_flux": "chandrashekar",
        "face_flux": "ec", "quadrature": quad, "cfl": args.cfl, "step": "RK4 step = 4 stages",
        "l2_flush": "not needed: state 40 B/node x nodes > 129 MB L2", "parallelism": par,
    }


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def smi_id(device):
    """nvidia-smi's --id for a torch CUDA device: its PCI bus id, because CUDA
    ordinals follow CUDA_VISIBLE_DEVICES and nvidia-smi's indices do not; the
    ordinal when the bus id is unavailable or nvidia-smi does not accept it."""
    import torch
    ordinal = str(device)
    try:
        pr = torch.cuda.get_device_properties(device)
        bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
    except (AttributeError, RuntimeError, AssertionError):
        return ordinal
    try:
        r = subprocess.run(["nvidia-smi", f"--id={bus}", "--query-gpu=index", "--format=csv,noheader"],
                           capture_output=True, text=True, timeout=20)
        if r.returncode == 0 and r.stdout.strip():
            return bus
    except (OSError, subprocess.TimeoutExpired):
        pass
    return ordinal


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed plumbing: each rank runs an independent replica, or one z-slab of a
# stack of copies (--decomp slab); weak scaling either way
# --------------------------------------------------------------------------
def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# --------------------------------------------------------------------------
# the workloads the oracle is timed on, each on a bounded periodic sample of the same
# element geometry and degree (the oracle's cost per node depends on p, not on the
# mesh size): (label, p, mesh elements per direction, sample elements per direction)
CPU_CONFIGS = [("taylor-green 4^3 p=3", 3, 4, 4), ("taylor-green 32^3 p=3", 3, 32, 6),
               ("taylor-green 16^3 p=7", 7, 16, 3), ("taylor-green 64^3 p=4", 4, 64, 6)]
BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def _oracle_worker(job):
    """One spawned process: the oracle steps its own copy of an n_sample^3 sample (one
    stage = du/dt with the WA inverse + a stage update), after a barrier shared with
    the other workers, for about budget_s of wall time.  Returns (nodes, per-stage
    seconds, wall seconds, CPU seconds)."""
    p, n_sample, budget_s, bar = job
    from oracle.problem import Problem
    ctrl = wl.tgv_mesh(n_sample, p)
    P = Problem(ctrl, (n_sample,) * 3, p, c=c_value(p))
    U = P.to_internal(wl.tgv_state(P.node_coords()))
    U = U + 1e-4 * P.dudt(U)  # warm-up stage
    if bar is not None:
        bar.wait()
    times = []
    t0, c0 = time.perf_counter(), time.process_time()
    while True:
        ts = time.perf_counter()
        U = U + 1e-4 * P.dudt(U)
        times.append(time.perf_counter() - ts)
        if time.perf_counter() - t0 > budget_s:
            break
    return n_sample ** 3 * (p + 1) ** 3, times, time.perf_counter() - t0, time.process_time() - c0


def _pool_run(p, n_sample, budget_s, workers):
    """The oracle on `workers` spawned processes (numpy single-threaded in each), every one
    stepping its own copy of the sample: aggregate GDOF/s, median seconds per stage."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")  # never fork a process that may hold a CUDA context
    saved = {k: os.environ.get(k) for k in BLAS_ENV}
    for k in BLAS_ENV:
        os.environ[k] = "1"
    try:
        with ctx.Manager() as mgr:
            bar = mgr.Barrier(workers)
            with ctx.Pool(workers) as pool:
                out = pool.map(_oracle_worker, [(p, n_sample, budget_s, bar)] * workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    nodes = out[0][0]
    wall = max(o[2] for o in out)
    stages = sum(len(o[1]) for o in out)
    med = statistics.median(t for o in out for t in o[1])
    return nodes * stages / wall / 1e9, med, stages


def host_info():
    info = {"nproc": os.cpu_count()}
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20)
        for ln in r.stdout.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Architecture", "Model name", "CPU(s)", "Thread(s) per core"):
                info[k.strip()] = v.strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return info


def cpu_baseline(p, budget_s=3.0, configs=None, n_mesh_p=64):
    """The FP64 oracle, as it stands, on this host's cores: for each workload of
    ``configs`` (default CPU_CONFIGS, plus degree p's workload if it is not among them)
    a bounded sample timed with one worker (one thread) and with one worker per core.
    Returns the cpu_baseline object (value: all cores on degree p's workload)."""
    host = host_info()
    cores = host["nproc"] or 1
    configs = list(CPU_CONFIGS if configs is None else configs)
    if not any(c[1] == p for c in configs):
        configs.append((f"taylor-green {n_mesh_p}^3 p={p}", p, n_mesh_p, 6 if p <= 4 else 3))
    rows, value, sample = [], None, ""
    for label, pc, n_mesh, n_s in configs:
        r1, m1, s1 = _pool_run(pc, n_s, budget_s, 1)
        rn, mn, sn = _pool_run(pc, n_s, budget_s, cores)
        rows.append({"workload": label, "p": pc, "sample": f"{n_s}^3 elements", "one_thread_gdof_per_s": r1,
                     "one_thread_median_stage_s": m1, "all_cores_gdof_per_s": rn, "all_cores_median_stage_s": mn,
                     "workers": cores, "stages": [s1, sn]})
        if pc == p and (value is None or n_mesh == n_mesh_p):
            value = rn
            sample = (f"{label}: {n_s}^3-element periodic sample, {cores} spawned worker processes (one per "
                      f"core, numpy single-threaded) each stepping its own copy for {budget_s:.0f} s; "
                      f"one-thread rate {r1:.2e} GDOF/s")
    return {"value": value, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample,
            "host": host, "configs": rows}


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return
    cfg = workload_config(args, ws)
    # the oracle on the same workload only: a bounded sample per timed window
    cpu = cpu_baseline(args.p, configs=[], n_mesh_p=args.n_el)
    val = cpu["value"]
    line = {"impl": "reference", "metric": "NSFR-EC residual GDOF/s per RK stage", "value": val,
            "unit": "GDOF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": cpu,
            "e2e": {"value": val, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our implementation
# --------------------------------------------------------------------------
def volume_kernel_flops(n_el, p, has_k=True, nq=None, vol_flux="chandrashekar"):
    """Algorithmic FP64 flops of one volume-kernel launch over n_el elements (for the
    uncollocated scheme the lines have nq points and the epilogue is the dense
    (chi Pi~1)^T, 1/(wJ), Pi~1 sweeps back to the p+1 solution nodes).  With Ranocha's
    pressure terms every flux counts FLOPS_PER_FLUX_RANOCHA, and the node pressures
    rho / (2 beta) 2 flops per node."""
    if vol_flux == "ranocha":
        if nq is not None:
            raise ValueError("the Ranocha model is for the collocated scheme")
        n = p + 1
        fluxes_vol, fluxes_hyb = 3 * n * n * n * (n - 1) // 2, 6 * n ** 3
        per_el = (fluxes_vol + fluxes_hyb) * (FLOPS_PER_FLUX_RANOCHA + FLOPS_PER_ACC)
        per_el += 6 * n * n * (5 + 10 * n) + 5 * n ** 3 + 2 * n ** 3
        if has_k:
            per_el += 6 * 5 * n * n * 4 * n
        return per_el * n_el, {"volume_pairs": fluxes_vol, "hybrid": fluxes_hyb, "flops_per_element": per_el}
    if nq is not None:
        n, ns = nq, p + 1
        per_el = (3 * n * n * n * (n - 1) // 2 + 6 * n ** 3) * (FLOPS_PER_FLUX + FLOPS_PER_ACC)
        per_el += 6 * n * n * (5 + 10 * n) + 5 * n ** 3
        per_el += 5 * 2 * (3 * n ** 4 + ns * n ** 3 + ns * ns * n * n + ns ** 3 * n)
        return per_el * n_el, {"volume_pairs": 3 * n * n * n * (n - 1) // 2, "hybrid": 6 * n ** 3,
                               "flops_per_element": per_el}
    n = p + 1
    fluxes_vol = 3 * n * n * n * (n - 1) // 2      # unordered pairs on every line
    fluxes_hyb = 6 * n ** 3                         # volume node x face node of its line
    # (the face fluxes f* themselves, 3 n^2 per element, are the face-flux kernel's)
    per_el = (fluxes_vol + fluxes_hyb) * (FLOPS_PER_FLUX + FLOPS_PER_ACC)
    per_el += 6 * n * n * (5 + 10 * n)              # face term combination, both faces of each line
    per_el += 5 * n ** 3                            # 1/(w J)
    if has_k:
        per_el += 6 * 5 * n * n * 4 * n             # rank-one Pi~ / Pi~^T sweeps
    return per_el * n_el, {"volume_pairs": fluxes_vol, "hybrid": fluxes_hyb, "flops_per_element": per_el}


class _Replica:
    """The whole mesh on this GPU (every rank an independent replica)."""

    def __init__(self, args, ctrl, u0, precision, dist, rank, ws, vol_flux="chandrashekar"):
        import torch
        from paper_2312_07725_gb300 import Solver
        N = args.n_el
        self.S = Solver(ctrl, (N, N, N), args.p, c=c_value(args.p), face_flux="ec", precision=precision,
                        nq=args.nq, vol_flux=vol_flux)
        self.u0 = u0
        self.u = torch.from_numpy(u0).cuda()
        self.cfl = args.cfl

    def step(self, u):
        self.S.rk_step(u, cfl=self.cfl)

    def e2e_setup(self):
        import torch
        self.uh = torch.from_numpy(self.u0).pin_memory()
        self.S.rk_step(self.uh.numpy(), cfl=self.cfl)  # sizes the library's staging buffers
        return self.uh.numel() * 8

    def e2e_step(self):
        # through the C ABI with pinned host buffers: the library copies in and out
        self.S.rk_step(self.uh.numpy(), cfl=self.cfl)

    def interior(self, t):
        return t


class _SlabRank:
    """One z-slab of a z-stack of ws copies of the mesh (weak scaling), with ghost
    layers refreshed by a halo exchange before every RK stage."""

    def __init__(self, args, ctrl, u0, precision, dist, rank, ws, vol_flux="chandrashekar"):
        from paper_2312_07725_gb300.slab import DistExchanger, Slab
        N = args.n_el
        self.slab = Slab(ctrl, (N, N, N), args.p, rank, ws, DistExchanger(dist, rank, ws), copies=ws,
                         c=c_value(args.p), face_flux="ec", precision=precision, nq=args.nq)
        self.S = self.slab.solver
        self.u = self.slab.extend(u0)
        self.cfl = args.cfl

    def step(self, u):
        self.slab.step(u, cfl=self.cfl)

    def e2e_setup(self):
        import torch
        self.uh = self.u.cpu().pin_memory()
        self.ud = torch.empty_like(self.u)
        return self.uh.numel() * 8

    def e2e_step(self):
        import torch
        self.ud.copy_(self.uh, non_blocking=True)
        self.slab.step(self.ud, cfl=self.cfl)
        self.uh.copy_(self.ud, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def interior(self, t):
        return self.slab.interior(t)


def measure(args, ctrl, u0, precision, dist, rank, ws, steps, vol_flux="chandrashekar"):
    """Time `steps` RK4 steps of one precision mode, plus its e2e variant."""
    import torch

    p, N = args.p, args.n_el
    if vol_flux != "chandrashekar":
        run = _Replica(args, ctrl, u0, precision, dist, rank, ws, vol_flux=vol_flux)
    else:
        run = (_SlabRank if args.decomp == "slab" else _Replica)(args, ctrl, u0, precision, dist, rank, ws)
    S, u = run.S, run.u
    stream = torch.cuda.current_stream()
    nodes = N ** 3 * (p + 1) ** 3  # this rank's own nodes (ghost layers not counted)
    for _ in range(args.warmup):
        run.step(u)
    torch.cuda.synchronize()
    barrier(dist)
    launches0 = S.kernel_launches()
    S.profile(True)
    clocks = ClockSampler(smi_id(torch.cuda.current_device()))
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        run.step(u)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    S.profile(False)
    prof = S.profile_read()
    launches = S.kernel_launches() - launches0
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1))
    value = nodes * 4 * steps * ws / (ms / 1e3) / 1e9
    # e2e: the same RK4 step from and back to pinned host memory
    e2e_bytes = run.e2e_setup()
    run.e2e_step()  # a second untimed step: the timed ones then start from a warm host path
    barrier(dist)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        run.e2e_step()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    e2e = nodes * 4 * args.e2e_steps * ws / e2e_s / 1e9
    # one du/dt of the initial state, to compare the two precision modes
    uin = torch.from_numpy(u0).cuda() if args.decomp != "slab" else run.slab.extend(u0)
    D = torch.empty_like(uin)
    S.residual(uin, D)
    torch.cuda.synchronize()
    # residual only (entropy projection, face fluxes, volume terms and the WA inverse, no RK
    # update): du/dt of the state, device-timed the same way
    for _ in range(2):
        S.residual(uin, D)
    torch.cuda.synchronize()
    barrier(dist)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(4 * steps):
        S.residual(uin, D)
    e1.record(stream)
    torch.cuda.synchronize()
    rms = max_over_ranks(dist, e0.elapsed_time(e1)) / (4 * steps)
    residual_only = nodes * ws / (rms / 1e3) / 1e9
    wa = None
    if precision == "fp64" and vol_flux == "chandrashekar" and args.nq is None:
        # the weight-adjusted inverse is the volume kernel's epilogue: its cost is the
        # kernel storing du/dt (sweeps, 1/(W J)) less the same kernel storing R
        # (nsfr_residual_raw), both from the library's events on the launch stream
        # (into a buffer of its own: D keeps the du/dt the precision modes are compared on)
        vol, Dw = {}, torch.empty_like(uin)
        for name, fn in (("dudt", S.residual), ("raw", S.residual_raw)):
            fn(uin, Dw)
            torch.cuda.synchronize()
            S.profile(True)
            for _ in range(2 * steps):
                fn(uin, Dw)
            torch.cuda.synchronize()
            S.profile(False)
            t_ms, n_l = S.profile_read()["volume"]
            vol[name] = t_ms / n_l
        wa = {"volume_ms_dudt": vol["dudt"], "volume_ms_raw": vol["raw"], "ms": vol["dudt"] - vol["raw"]}
        del Dw
    del uin
    kern = {k: {"ms_total": v[0], "launches": v[1], "ms_avg": v[0] / v[1]} for k, v in prof.items()}
    res = {"value": value, "ms_per_step": ms / steps, "e2e": e2e, "e2e_bytes": e2e_bytes,
           "gpu_launches": launches, "kernels": kern, "clocks": clk,
           "dudt": run.interior(D).cpu().numpy(), "n_el_computed": S.n_el,
           "residual_only": {"value": residual_only, "unit": "GDOF/s", "ms_per_evaluation": rms},
           "wa_inverse": wa}
    S.close()
    del u, D, run
    torch.cuda.empty_cache()
    return res


def measure_adjoint(args, ctrl, u0, residual_ms):
    """The hand-written VJP of du/dt (nsfr_vjp: with respect to the state, and to the
    state and the grid control points) and the diagnostics (nsfr_entropy) on the same
    workload, FP64, device-timed with CUDA events on the launching stream."""
    import torch
    from paper_2312_07725_gb300 import Solver
    N, p = args.n_el, args.p
    S = Solver(ctrl, (N, N, N), p, c=c_value(p), face_flux="ec")
    u = torch.from_numpy(u0).cuda()
    dbar = torch.from_numpy(np.ascontiguousarray(wl.random_cotangent(u0.shape))).cuda()
    ubar = torch.zeros_like(u)
    xbar = torch.zeros((S.n_el, (S.p_geo + 1) ** 3, 3), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the first call allocates the VJP scratch
        S.vjp(u, dbar, ubar, xbar)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def timed(fn, k=3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    S.profile(True)
    t_full = timed(lambda: S.vjp(u, dbar, ubar, xbar))
    S.profile(False)
    prof = S.profile_read()
    t_state = timed(lambda: S.vjp(u, dbar, ubar))
    t_diag = timed(lambda: S.entropy(u))  # synchronises: includes the host-side finish
    nodes = N ** 3 * (p + 1) ** 3
    kern = {k: {"ms_total": v[0], "launches": v[1], "ms_avg": v[0] / v[1]} for k, v in prof.items()}
    S.close()
    del u, dbar, ubar, xbar
    torch.cuda.empty_cache()
    return {"vjp_state_and_grid": {"ms": t_full, "gdof_per_s": nodes / (t_full / 1e3) / 1e9},
            "vjp_state": {"ms": t_state, "gdof_per_s": nodes / (t_state / 1e3) / 1e9},
            "ratio_to_residual": t_full / residual_ms, "kernels": kern,
            "diagnostics": {"ms": t_diag, "gdof_per_s": nodes / (t_diag / 1e3) / 1e9}}


def run_ours(args, rank, ws, dist):
    cfg = workload_config(args, ws)
    p, N = args.p, args.n_el
    ctrl = wl.tgv_mesh(N, p)
    from paper_2312_07725_gb300 import Solver
    S0 = Solver(ctrl, (N, N, N), p, c=cfg["c"], nq=args.nq)
    xyz = S0.node_coords()
    S0.close()
    u0 = np.ascontiguousarray(wl.tgv_state(xyz))
    del xyz

    m64 = measure(args, ctrl, u0, "fp64", dist, rank, ws, args.steps)
    d64 = m64.pop("dudt")
    m32, mff = None, None
    if args.modes == "both":  # the uncollocated scheme has the fp32_bulk form, not the float-float one
        m32 = measure(args, ctrl, u0, "fp32_bulk", dist, rank, ws, args.steps)
        d32 = m32.pop("dudt")
        bulk_err = float(np.linalg.norm((d32 - d64).ravel()) / np.linalg.norm(d64.ravel()))
        del d32
    if args.nq is None and args.modes == "both":
        mff = measure(args, ctrl, u0, "fp32_bulk_ff", dist, rank, ws, args.steps)
        dff = mff.pop("dudt")
        ff_err = float(np.linalg.norm((dff - d64).ravel()) / np.linalg.norm(d64.ravel()))
        del dff
    del d64

    mra = None
    if args.nq is None and args.modes == "both" and args.decomp == "replicas":
        # the paper's EC runs' flux: Chandrashekar's with Ranocha's pressure terms (FP64)
        mra = measure(args, ctrl, u0, "fp64", dist, rank, ws, args.steps, vol_flux="ranocha")
        mra.pop("dudt")

    adj = None
    if args.nq is None and not args.no_adjoint and args.decomp == "replicas":
        adj = measure_adjoint(args, ctrl, u0, m64["residual_only"]["ms_per_evaluation"])

    clk = m64["clocks"]
    vol_ms, vol_n = m64["kernels"]["volume"]["ms_total"], m64["kernels"]["volume"]["launches"]
    ne_launch = m64["n_el_computed"]  # elements one volume launch processes (slabs: with ghost layers)
    flops, counts = volume_kernel_flops(ne_launch, p, cfg["c"] != 0.0, args.nq)
    achieved = flops / (vol_ms / vol_n / 1e3) / 1e12
    peak, peak_src = fp64_peak(clk)
    peaks = measure_fma_peaks() if args.nq is None else None
    probe64 = peaks["fp64"]["tflops"] if peaks else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": (VOLUME_DRAM_BYTES_PER_ELEMENT[p] * ne_launch
                        if p in VOLUME_DRAM_BYTES_PER_ELEMENT and args.nq is None else None),
            "traffic_unit": "bytes per launch", "kernel": f"volume_kernel<{args.nq or p + 1}> (FP64 pipe)",
            "peak_source": peak_src,
            "peak_measured_probe": probe64, "frac_of_measured_probe": achieved / probe64 if probe64 else None,
            "flops_per_launch": flops, "flux_evals_per_element": counts}
    rk = None
    if args.nq is None:  # the stage models are those of the collocated scheme
        rk = {"fp64": roofline_kernels(m64["kernels"], p, ne_launch, "fp64", clk, peaks, cfg["c"] != 0.0)}
        if m64.get("wa_inverse"):
            rk["fp64"]["mass_inverse"] = wa_inverse_roofline(m64["wa_inverse"], p, ne_launch, clk, peaks,
                                                             cfg["c"] != 0.0)
        for nm, m in (("fp32_bulk", m32), ("fp32_bulk_ff", mff)):
            if m is not None:
                rk[nm] = roofline_kernels(m["kernels"], p, ne_launch, nm, m["clocks"], peaks, cfg["c"] != 0.0)
        if mra is not None:
            rk["ranocha"] = roofline_kernels(mra["kernels"], p, ne_launch, "fp64", mra["clocks"], peaks,
                                             cfg["c"] != 0.0, vol_flux="ranocha")
    if adj is not None and rk is not None:
        fp64_nom = peak
        rk["adjoint"] = {}
        for nm, work in adjoint_kernel_models(p, ne_launch, cfg["c"] != 0.0).items():
            if nm in adj["kernels"]:
                t = adj["kernels"][nm]["ms_avg"] / 1e3
                rk["adjoint"][nm] = {"bound": "alu", "pipe": "fp64", "work_per_launch": work, "work_unit": "flops",
                                     "ms_avg": t * 1e3, "achieved": work / t / 1e12, "unit": "TFLOP/s",
                                     "peak": fp64_nom, "frac": work / t / 1e12 / fp64_nom}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, n_mesh_p=N)
    if rank == 0:
        line = {"metric": "NSFR-EC residual GDOF/s per RK stage", "value": m64["value"], "unit": "GDOF/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m64["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg, "gdof_per_s_x5_components": 5 * m64["value"],
                "e2e": {"value": m64["e2e"], "unit": "GDOF/s", "h2d_bytes_per_step": m64["e2e_bytes"],
                        "d2h_bytes_per_step": m64["e2e_bytes"]},
                "gpu_launches": m64["gpu_launches"], "kernels": m64["kernels"], "roofline": roof,
                "roofline_kernels": rk, "fma_probe": peaks, "clocks": clk,
                "residual_only": m64["residual_only"],
                "adjoint": adj,
                "cpu_baseline": cpu,
                "ranocha": None if mra is None else
                {"value": mra["value"], "unit": "GDOF/s", "ms_per_step": mra["ms_per_step"],
                 "vs_chandrashekar": mra["value"] / m64["value"],
                 "e2e": {"value": mra["e2e"], "unit": "GDOF/s", "h2d_bytes_per_step": mra["e2e_bytes"],
                         "d2h_bytes_per_step": mra["e2e_bytes"]},
                 "gpu_launches": mra["gpu_launches"], "kernels": mra["kernels"],
                 "residual_only": mra["residual_only"], "clocks": mra["clocks"],
                 "flux": "Chandrashekar's with Ranocha's pressure terms (volume, hybrid and face), FP64"},
                "fp32_bulk": None if m32 is None else
                {"value": m32["value"], "unit": "GDOF/s", "ms_per_step": m32["ms_per_step"],
                 "speedup_vs_fp64": m32["value"] / m64["value"],
                 "dudt_rel_l2_vs_fp64_path": bulk_err,
                 "e2e": {"value": m32["e2e"], "unit": "GDOF/s", "h2d_bytes_per_step": m32["e2e_bytes"],
                         "d2h_bytes_per_step": m32["e2e_bytes"]},
                 "gpu_launches": m32["gpu_launches"], "kernels": m32["kernels"],
                 "residual_only": m32["residual_only"],
                 "clocks": m32["clocks"],
                 "dtype": "f32 flux arithmetic and contractions; f64 log means, entropy projection, state"},
                "fp32_bulk_ff": None if mff is None else
                {"value": mff["value"], "unit": "GDOF/s", "ms_per_step": mff["ms_per_step"],
                 "speedup_vs_fp64": mff["value"] / m64["value"],
                 "dudt_rel_l2_vs_fp64_path": ff_err,
                 "e2e": {"value": mff["e2e"], "unit": "GDOF/s", "h2d_bytes_per_step": mff["e2e_bytes"],
                         "d2h_bytes_per_step": mff["e2e_bytes"]},
                 "gpu_launches": mff["gpu_launches"], "kernels": mff["kernels"],
                 "residual_only": mff["residual_only"], "clocks": mff["clocks"],
                 "dtype": "f32 flux arithmetic and contractions; float-float log-mean scalars and entropy "
                          "projection (f64 log means across wide jumps); f64 state"}}
        print(json.dumps(line), flush=True)


def fp64_peak(clk):
    """FP64 FMA peak in TFLOP/s: SMs x FP64 FMA lanes per SM per clock x 2 x clock.

    The lane count is the FP64 issue rate ncu reports for this part
    (sm__sass_thread_inst_executed_op_dfma_pred_on peak, 2 per SM per cycle);
    the clock is the median SM clock sampled during the timed region."""
    lanes = FP64_LANES_PER_SM
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    return 152 * lanes * 2 * mhz * 1e6 / 1e12, f"152 SMs x {lanes} FP64 FMA/clk/SM x 2 x {mhz:.0f} MHz"


FP64_LANES_PER_SM = 2.0  # ncu: 2 DFMA thread-instructions per SM per cycle (nominal 1.26 TFLOP/s at 2070 MHz)
FP32_LANES_PER_SM = 128.0  # FP32 FMA lanes per SM (4 sub-partitions x 32)
HBM_FALLBACK_GBS = 6800.0  # the profiling recipe's fallback copy bandwidth, if no measured figure exists


def hbm_peak():
    """Measured copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy, measured)"
    except (OSError, KeyError, ValueError, TypeError):
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def measure_fma_peaks():
    """The FMA pipes' throughput, measured with nsfr_fma_probe (FP64 and FP32 chains on
    every SM, about 0.4 s each, CUDA events on the launching stream), with the SM clock
    sampled during each: TFLOP/s (an FMA = 2 flops) and the clock."""
    import torch
    from paper_2312_07725_gb300 import nsfr
    sink = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    for name, fp32, iters in (("fp64", 0, 100_000), ("fp32", 1, 6_000_000)):
        blocks = 152 * 8
        nsfr.fma_probe(fp32, max(1, iters // 100), blocks, sink)  # warm-up
        torch.cuda.synchronize()
        clocks = ClockSampler(smi_id(torch.cuda.current_device()))
        clocks.start()
        time.sleep(0.2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmas = sum(nsfr.fma_probe(fp32, iters, blocks, sink) for _ in range(2))
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        out[name] = {"tflops": 2.0 * fmas / (ms / 1e3) / 1e12, "ms": ms, "clocks": clk,
                     "probe": f"nsfr_fma_probe: {blocks} CTAs x 256 threads x 8 chains x {iters} steps, 2 launches"}
    return out


def stage_kernel_models(p, ne, precision, has_k=True, vol_flux="chandrashekar"):
    """Algorithmic work of one launch of each kernel of an RK stage over ne elements
    (n = p+1; an FMA counts 2 flops; a division, reciprocal, square root, log or exp 1):
      face_states  v(u) at n^3 nodes (32 each: u, |u|^2, p, beta, ln rho, ln p, s, v,
                   the record fields), t_s . v to the six faces (30 n^3 multiply-adds),
                   u(v~) at 6 n^2 face nodes (22 each: u, |u|^2, s~, ln 2 beta~, rho~ by
                   exp, the record fields)
      face_flux    3 n^2 face fluxes of 55 flops (the EC flux of the bench's faces; with
                   Ranocha's pressure terms 62, plus 4 for the two states' pressures)
      volume       volume_kernel_flops
      max_wavespeed  40 bytes (the state) read per node and launch
    Returns {kernel: (kind, work, unit)}."""
    n = p + 1
    fs = (32 * n ** 3 + 60 * n ** 3 + 6 * n * n * 22) * ne
    vol, _ = volume_kernel_flops(ne, p, has_k, vol_flux=vol_flux)
    ff = FLOPS_PER_FLUX_RANOCHA + 4 if vol_flux == "ranocha" else FLOPS_PER_FLUX
    return {"face_states": ("flops", fs), "face_flux": ("flops", 3 * n * n * ff * ne),
            "volume": ("flops", vol), "max_wavespeed": ("bytes", 40 * n ** 3 * ne)}


def roofline_kernels(kern, p, ne, precision, clk, peaks, has_k=True, vol_flux="chandrashekar"):
    """Per-kernel rooflines of one precision mode's timed step: algorithmic work per launch
    (stage_kernel_models) over the kernel's mean launch time from the library's CUDA events,
    against the bounding resource: the FP64 FMA pipe (nominal from 152 SMs x 2 lanes x the
    sampled clock, and the probe's measured rate), the FP32 FMA pipe (the FP32-bulk kernels'
    float and float-float arithmetic) or HBM (the measured copy bandwidth)."""
    mhz = clk.get("sm_mhz") or 2070.0
    fp64_nom = 152 * FP64_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    fp32_nom = 152 * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    hbm, hbm_src = hbm_peak()
    models = stage_kernel_models(p, ne, precision, has_k, vol_flux)
    out = {}
    for name, (kind, work) in models.items():
        if name not in kern:
            continue
        t = kern[name]["ms_avg"] / 1e3
        if kind == "bytes":
            ach = work / t / 1e9
            out[name] = {"bound": "hbm", "work_per_launch": work, "work_unit": "bytes", "ms_avg": t * 1e3,
                         "achieved": ach, "unit": "GB/s", "peak": hbm, "frac": ach / hbm, "peak_source": hbm_src}
            continue
        ach = work / t / 1e12
        pipe = "fp64"
        # the bulk volume kernels run their flux arithmetic on the FP32 pipe (the log
        # means' series branch included, in float-float); FP64 is left on the rare log
        # branch and the epilogue's conversions
        if precision != "fp64" and name == "volume":
            pipe = "fp32"
        if precision == "fp32_bulk_ff" and name == "face_states":
            pipe = "fp32"
        e = {"bound": "alu", "work_per_launch": work, "work_unit": "flops", "ms_avg": t * 1e3, "achieved": ach,
             "unit": "TFLOP/s"}
        if pipe == "fp64":
            e.update({"pipe": "fp64", "peak": fp64_nom, "frac": ach / fp64_nom,
                      "peak_source": f"152 SMs x 2 FP64 FMA/clk/SM x 2 x {mhz:.0f} MHz"})
        else:
            e.update({"pipe": "fp32 (the flux arithmetic; float-float where the form says so)", "peak": fp32_nom,
                      "frac": ach / fp32_nom, "peak_source": f"152 SMs x 128 FP32 FMA/clk/SM x 2 x {mhz:.0f} MHz"})
        if peaks and pipe == "fp64" and "fp64" in peaks:
            e["frac_of_measured_probe"] = ach / peaks["fp64"]["tflops"]
        out[name] = e
    return out


def wa_inverse_roofline(wa, p, ne, clk, peaks, has_k=True):
    """The weight-adjusted mass inverse, fused into the volume kernel's epilogue: its
    algorithmic flops (the six rank-one sweeps, 120 n^3 per element, and the 1/(W J)
    scaling, 5 n^3) over its marginal time, the volume kernel storing du/dt less the
    same kernel storing R."""
    n = p + 1
    work = (5 * n ** 3 + (120 * n ** 3 if has_k else 0)) * ne
    mhz = clk.get("sm_mhz") or 2070.0
    fp64_nom = 152 * FP64_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    t = wa["ms"] / 1e3
    e = {"bound": "alu", "pipe": "fp64", "work_per_launch": work, "work_unit": "flops", "ms_avg": wa["ms"],
         "how": "marginal: volume kernel with the du/dt epilogue "
                f"({wa['volume_ms_dudt']:.3f} ms) less the same kernel storing R ({wa['volume_ms_raw']:.3f} ms)"}
    if t > 0:
        ach = work / t / 1e12
        e.update({"achieved": ach, "unit": "TFLOP/s", "peak": fp64_nom, "frac": ach / fp64_nom,
                  "peak_source": f"152 SMs x 2 FP64 FMA/clk/SM x 2 x {mhz:.0f} MHz"})
        if peaks and "fp64" in peaks:
            e["frac_of_measured_probe"] = ach / peaks["fp64"]["tflops"]
    return e


def adjoint_kernel_models(p, ne, has_k=True):
    """Algorithmic work of the adjoint kernels (models, n = p+1): the VJP of every two-point
    flux (1,500 volume and hybrid plus 3 n^2 face fluxes at p = 4) as a forward recompute
    (55) plus a reverse sweep counted at twice the forward flops (110) plus the cotangent
    accumulation (20), and the transposed WA-inverse sweeps; the face-state VJP as three
    times the forward face-state flops (recompute and reverse); the metric VJP as the
    reverse of the conservative-curl construction, whose sweeps are linear (90 n^4
    multiply-adds: interpolation, derivatives, curl, transfer to the GL nodes, J)."""
    n = p + 1
    fluxes = 3 * n ** 3 * (n - 1) // 2 + 6 * n ** 3 + 3 * n * n
    vol = fluxes * (FLOPS_PER_FLUX * 3 + FLOPS_PER_ACC) + 6 * n * n * (5 + 10 * n) + 5 * n ** 3
    if has_k:
        vol += 6 * 5 * n * n * 4 * n
    fs = 3 * (32 * n ** 3 + 60 * n ** 3 + 6 * n * n * 22)
    return {"vjp_volume": vol * ne, "vjp_face": fs * ne, "vjp_metrics": 180 * n ** 4 * ne}


def main():
    args = parse()
    rank, ws, dist = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
    else:
        run_ours(args, rank, ws, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
