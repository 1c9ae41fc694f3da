"""Drivers for the studies the scheme is judged by, on the GPU library.

  convergence   L2 error of rho for the exact density wave on the warped unit cube,
                RK4 to t_f (order p+1 expected: the paper's Fig. OOA claim)
  tgv_history   entropy, its semi-discrete rate, kinetic energy and conserved totals
                along a Taylor-Green run, FP64 or FP32-bulk
  adjoint       gradient of the kinetic energy after N RK4 steps with respect to the
                initial state and the mesh control points (checkpointed discrete adjoint)
  manufactured  the paper's grid study with the manufactured solution and its source
                on the warped [-1, 1]^3 (Roe faces, CFL 0.2, t_f = 2): L2 errors of
                density and pressure, orders
  max_cfl       the paper's maximum-CFL study on 4^3 elements (t_f = 1)

Usage: python -m paper_2312_07725_gb300.experiments convergence|tgv|adjoint|manufactured|max_cfl [options]
Each prints one JSON document.  Inputs come from ``workloads``; everything that
computes runs in libnsfr.so.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

import workloads as wl

from .nsfr import Solver


def l2_error_rho(S, u, t):
    xyz = S.node_coords()
    ex = wl.density_wave_state(xyz, t)
    wj = S.quadrature()
    e = u[:, 0] - ex[:, 0]
    return math.sqrt(float(np.sum(wj * e * e)))


def convergence(p, levels, c=0.0, face_flux="ec_roe", tf=0.1, cfl=0.1, precision="fp64"):
    """L2 errors of rho at t_f for N^3 meshes, N in ``levels``, and the observed orders."""
    errs, times = [], []
    for N in levels:
        ctrl = wl.unit_mesh(N, p)
        S = Solver(ctrl, (N, N, N), p, c=c, face_flux=face_flux, precision=precision)
        xyz = S.node_coords()
        u = torch.from_numpy(np.ascontiguousarray(wl.density_wave_state(xyz, 0.0))).cuda()
        dx = 1.0 / (N * (p + 1))
        lam = math.sqrt(3.0) + math.sqrt(1.4 * 1.0 / (2.0 - 0.1))  # max |u| + a of the wave
        nsteps = int(math.ceil(tf / (cfl * dx / lam)))
        dt = tf / nsteps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            S.rk_step(u, dt=dt)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        S.check()
        errs.append(l2_error_rho(S, u.cpu().numpy(), tf))
        S.close()
    orders = [math.log(errs[i - 1] / errs[i]) / math.log(levels[i] / levels[i - 1]) for i in range(1, len(errs))]
    return {"p": p, "levels": list(levels), "c": c, "face_flux": face_flux, "tf": tf, "cfl": cfl,
            "l2_errors": errs, "orders": orders, "seconds": times}


def tgv_history(n_el, p, c, steps, precision="fp64", cfl=0.1, every=10, tf=None, nodes="gl", face_flux="ec",
                warp="tgv"):
    """Entropy, its semi-discrete rate, kinetic energy and conserved totals along a
    Taylor-Green run: ``steps`` RK4 steps, or up to time ``tf`` when given."""
    ctrl = wl.tgv_mesh(n_el, p, warp=warp)
    S = Solver(ctrl, (n_el,) * 3, p, c=c, precision=precision, nodes=nodes, face_flux=face_flux)
    xyz = S.node_coords()
    u = torch.from_numpy(np.ascontiguousarray(wl.tgv_state(xyz))).cuda()
    hist = []
    t = 0.0
    d0 = S.entropy(u)
    n = 0
    dt_prev = 0.0
    t0 = time.perf_counter()
    while True:
        done = (tf is None and n == steps) or (tf is not None and t >= tf - 1e-12)
        if n % every == 0 or done:
            d = S.entropy(u)
            hist.append({"step": n, "t": t, "entropy": d["entropy"], "entropy_rate": d["entropy_rate"],
                         "entropy_rate_rel": abs(d["entropy_rate"]) / d["entropy_rate_scale"],
                         "kinetic_energy": d["kinetic_energy"],
                         # drift of the conserved totals: mass and energy relative to their
                         # totals, momentum (total zero for the vortex) relative to the mass total
                         "Q_drift": [abs(d["Q"][0] - d0["Q"][0]) / abs(d0["Q"][0])]
                         + [abs(d["Q"][k] - d0["Q"][k]) / abs(d0["Q"][0]) for k in (1, 2, 3)]
                         + [abs(d["Q"][4] - d0["Q"][4]) / abs(d0["Q"][4])]})
        if done:
            break
        if tf is not None and n > 0 and t + 1.05 * dt_prev >= tf:
            dt_prev = S.rk_step(u, dt=tf - t)  # last step lands on tf (the CFL step changes slowly)
        else:
            dt_prev = S.rk_step(u, cfl=cfl)
        t += dt_prev
        n += 1
    return {"n_el": n_el, "p": p, "c": c, "precision": precision, "nodes": nodes, "face_flux": face_flux,
            "steps": n, "t_final": t, "seconds": time.perf_counter() - t0, "history": hist}


def adjoint(n_el=16, p=4, steps=50, checkpoint=10, c=None, cfl=0.1):
    from .autograd import rk4_adjoint
    c = c if c is not None else 0.0
    ctrl = wl.tgv_mesh(n_el, p)
    S = Solver(ctrl, (n_el,) * 3, p, c=c)
    xyz = S.node_coords()
    u0 = torch.from_numpy(np.ascontiguousarray(wl.tgv_state(xyz))).cuda()
    wj = torch.from_numpy(S.quadrature()).cuda()
    dt = cfl * (2 * math.pi / (n_el * (p + 1))) / 11.0  # frozen step below the CFL-0.1 step

    def ke(v):
        return float((0.5 * wj * (v[:, 1:4] ** 2).sum(dim=1) / v[:, 0]).sum())

    def ke_grad(v):
        g = torch.zeros_like(v)
        g[:, 0] = -0.5 * wj * (v[:, 1:4] ** 2).sum(dim=1) / v[:, 0] ** 2
        g[:, 1:4] = wj[:, None] * v[:, 1:4] / v[:, 0:1]
        return g

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, xbar, uN = rk4_adjoint(S, u0, dt, steps, ke_grad, checkpoint_every=checkpoint)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    # central finite differences along seeded directions (state, and a mesh amplitude)
    rng = np.random.default_rng(3)
    d = torch.from_numpy(rng.standard_normal(tuple(u0.shape)) * 1e-2).cuda() * u0.abs().amax(dim=(0, 2), keepdim=True)

    def traj(v0, solver):
        v = v0.clone()
        for _ in range(steps):
            solver.rk_step(v, dt=dt)
        return v

    eps = 1e-6
    fd = (ke(traj(u0 + eps * d, S)) - ke(traj(u0 - eps * d, S))) / (2 * eps)
    adj = float((lam * d).sum())
    # the three warp amplitudes A_x = 0.10, A_y = 0.05, A_z = 0.08: ctrl(A) = X0 + sum_k A_k D_k,
    # D_k the displacement of coordinate k per unit amplitude
    X0 = wl.control_points(n_el, n_el, n_el, p, -math.pi, math.pi)
    amps = (0.10, 0.05, 0.08)
    xb = xbar.cpu().numpy()
    out = {"n_el": n_el, "p": p, "steps": steps, "checkpoint_every": checkpoint, "dt": dt,
           "ke_final": ke(uN), "adjoint_seconds": t_adj,
           "state_direction": {"adjoint": adj, "central_fd": fd, "rel_diff": abs(adj - fd) / abs(adj)},
           "warp_amplitudes": []}
    for k, a_k in enumerate(amps):
        Dk = np.zeros_like(ctrl)
        Dk[..., k] = (ctrl - X0)[..., k] / a_k
        adj_a = float((xb * Dk).sum())
        row = {"amplitude": ["x", "y", "z"][k], "adjoint": adj_a}

        def ke_at(h):
            S2 = Solver(np.ascontiguousarray(ctrl + h * Dk), (n_el,) * 3, p, c=c)
            v = ke(traj(u0, S2))
            S2.close()
            return v

        # central differences of second order at h = 1e-6 and 1e-4, and of fourth order
        # (-f(2h) + 8 f(h) - 8 f(-h) + f(-2h)) / 12h at h = 1e-3: dKE/dA is ~1e-6 of KE, so
        # the small step sits at the rounding floor of KE and the large one needs the
        # higher-order stencil
        for h in (1e-6, 1e-4):
            fd_a = (ke_at(h) - ke_at(-h)) / (2 * h)
            row[f"fd2_h{h:g}"] = fd_a
            row[f"rel_diff_fd2_h{h:g}"] = abs(adj_a - fd_a) / abs(adj_a)
        h = 1e-3
        fd4 = (-ke_at(2 * h) + 8 * ke_at(h) - 8 * ke_at(-h) + ke_at(-2 * h)) / (12 * h)
        row["fd4_h0.001"] = fd4
        row["rel_diff_fd4_h0.001"] = abs(adj_a - fd4) / abs(adj_a)
        out["warp_amplitudes"].append(row)
    return out


# --------------------------------------------------------------------------
# the manufactured solution (Sec. "Manufactured Solution Convergence") and the
# maximum CFL study (Sec. "Maximum CFL")
# --------------------------------------------------------------------------
def manufactured_errors(S, u, t, gamma=1.4):
    """L2 errors of density and pressure against the manufactured solution at time t,
    sqrt(sum (u - u_exact)^T W J (u - u_exact)) over the volume nodes."""
    xyz = S.node_coords()
    ex = wl.manufactured_state(xyz, t)
    wj = S.quadrature()
    rho = u[:, 0]
    p = (gamma - 1.0) * (u[:, 4] - 0.5 * (u[:, 1] ** 2 + u[:, 2] ** 2 + u[:, 3] ** 2) / rho)
    p_ex = (gamma - 1.0) * (ex[:, 4] - 1.5 * ex[:, 0])
    return (math.sqrt(float(np.sum(wj * (rho - ex[:, 0]) ** 2))),
            math.sqrt(float(np.sum(wj * (p - p_ex) ** 2))))


def run_manufactured(N, p, c, tf, nodes="gl", face_flux="ec_roe", dt_fixed=None, cfl=None,
                     precision="fp64"):
    """Integrate the manufactured solution on the paper's warped N^3 mesh of [-1, 1]^3
    from its exact state to t_f, with a fixed step dt_fixed or the CFL step of the
    maximum wave speed (the last step shortened to land on t_f); returns (errors, steps)."""
    ctrl = wl.mms_mesh(N, p)
    S = Solver(ctrl, (N, N, N), p, c=c, face_flux=face_flux, nodes=nodes, precision=precision)
    try:
        S.set_source("manufactured", 0.0)
        u = torch.from_numpy(np.ascontiguousarray(wl.manufactured_state(S.node_coords(), 0.0))).cuda()
        dx = S.dx
        t, steps = 0.0, 0
        while tf - t > 1e-12 * tf:
            dt = dt_fixed if dt_fixed is not None else cfl * dx / S.max_wavespeed(u)
            dt = min(dt, tf - t)
            S.rk_step(u, dt=dt)
            t += dt
            steps += 1
        S.check()
        assert abs(S.time - t) <= 1e-12 * tf
        return manufactured_errors(S, u.cpu().numpy(), tf), steps
    finally:
        S.close()


def manufactured_convergence(p, levels, c=0.0, nodes="gl", tf=2.0, cfl=0.2, face_flux="ec_roe"):
    """The paper's grid study: the adaptive step dt = 0.2 dx / max(|u| + a) (its
    "dt = 0.2 dx" read as CFL 0.2: a fixed 0.2 dx would be CFL 0.46 at this solution's
    wave speed of about 2.3), dx = 2 / (N (p+1)), one period (t_f = 2); L2 errors of
    density and pressure and the observed orders."""
    errs, times, steps = [], [], []
    for N in levels:
        t0 = time.perf_counter()
        e, k = run_manufactured(N, p, c, tf, nodes, face_flux, cfl=cfl)
        times.append(time.perf_counter() - t0)
        errs.append(e)
        steps.append(k)
    orders = [[math.log(errs[i - 1][k] / errs[i][k]) / math.log(levels[i] / levels[i - 1]) for k in (0, 1)]
              for i in range(1, len(errs))]
    return {"study": "manufactured", "p": p, "levels": list(levels), "c": c, "nodes": nodes, "tf": tf,
            "cfl": cfl, "face_flux": face_flux, "steps": steps,
            "l2_errors_rho_p": errs, "orders_rho_p": orders, "seconds": times}


def max_cfl(p, c=0.0, nodes="gl", n_el=4, tf=1.0, cfl0=0.1, dcfl=0.01, cfl_max=1.0, digits=7):
    """Sec. "Maximum CFL": the pressure L2 error at t_f = 1 with CFL 0.1 is the reference;
    the CFL grows by 0.01 until the error no longer agrees with it to ``digits``
    significant digits (|e - e_ref| > 0.5 * 10^(1 - digits) |e_ref|) or the run fails;
    the last agreeing CFL is the maximum."""
    from .nsfr import NSFRError
    ref, _ = run_manufactured(n_el, p, c, tf, nodes, cfl=cfl0)
    tol = 0.5 * 10.0 ** (1 - digits) * ref[1]
    rows, best = [], cfl0
    k = 1
    while cfl0 + k * dcfl <= cfl_max + 1e-12:
        cfl = round(cfl0 + k * dcfl, 10)
        try:
            e, steps = run_manufactured(n_el, p, c, tf, nodes, cfl=cfl)
            ok = math.isfinite(e[1]) and abs(e[1] - ref[1]) <= tol
        except NSFRError:
            e, steps, ok = (float("nan"), float("nan")), 0, False
        rows.append({"cfl": cfl, "pressure_error": e[1], "steps": steps, "agrees": ok})
        if not ok:
            break
        best = cfl
        k += 1
    return {"study": "max_cfl", "p": p, "c": c, "nodes": nodes, "n_el": n_el, "tf": tf,
            "reference_pressure_error": ref[1], "max_cfl": best, "sweep": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["convergence", "tgv", "adjoint", "manufactured", "max_cfl"])
    ap.add_argument("--p", type=int, nargs="+", default=[2, 3, 4, 5])
    ap.add_argument("--levels", type=int, nargs="+", default=[4, 8, 16, 32])
    ap.add_argument("--c", default="both", choices=["dg", "hu", "both"])
    ap.add_argument("--n-el", type=int, default=32)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--precision", default="both", choices=["fp64", "fp32_bulk", "fp32_bulk_ff", "both"])
    ap.add_argument("--tf", type=float, default=None, help="TGV: run to this time instead of --steps")
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--nodes", default="gl", choices=["gl", "lgl"])
    ap.add_argument("--face-flux", default=None, choices=["ec", "ec_roe", "ec_es"],
                    help="face flux (default: ec for tgv, ec_roe for convergence)")
    ap.add_argument("--warp", default="tgv", choices=["tgv", "paper", "none"])
    args = ap.parse_args()
    import os
    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                           "c_values.json")) as f:
        c_hu = {int(k): v for k, v in json.load(f)["c_hu"].items()}
    out = []
    if args.study == "convergence":
        for p in args.p:
            for ck in (["dg", "hu"] if args.c == "both" else [args.c]):
                out.append(convergence(p, args.levels, c=0.0 if ck == "dg" else c_hu[p],
                                       face_flux=args.face_flux or "ec_roe"))
                print(json.dumps(out[-1]), flush=True)
    elif args.study == "tgv":
        for p in args.p:
            for ck in (["dg", "hu"] if args.c == "both" else [args.c]):
                for prec in (["fp64", "fp32_bulk"] if args.precision == "both" else [args.precision]):
                    out.append(tgv_history(args.n_el, p, 0.0 if ck == "dg" else c_hu[p], args.steps, prec,
                                           every=args.every, tf=args.tf, nodes=args.nodes,
                                           face_flux=args.face_flux or "ec", warp=args.warp))
                    print(json.dumps(out[-1]), flush=True)
    elif args.study == "manufactured":
        for p in args.p:
            for ck in (["dg", "hu"] if args.c == "both" else [args.c]):
                out.append(manufactured_convergence(p, args.levels, c=0.0 if ck == "dg" else c_hu[p],
                                                    nodes=args.nodes, tf=args.tf or 2.0))
                print(json.dumps(out[-1]), flush=True)
    elif args.study == "max_cfl":
        for p in args.p:
            for nodes in ("gl", "lgl"):
                for ck in (["dg", "hu"] if args.c == "both" else [args.c]):
                    r = max_cfl(p, c=0.0 if ck == "dg" else c_hu[p], nodes=nodes, tf=args.tf or 1.0)
                    r["c_kind"] = ck
                    print(json.dumps(r), flush=True)
    else:
        print(json.dumps(adjoint(n_el=args.n_el, p=args.p[0], steps=args.steps)), flush=True)


if __name__ == "__main__":
    main()
