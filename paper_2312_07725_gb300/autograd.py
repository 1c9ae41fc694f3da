"""Differentiation through the NSFR-EC residual and RK4 (torch.autograd front end).

``dudt(u, solver)``     du/dt as a torch.autograd.Function whose backward calls the
                        library's hand-written VJP (nsfr_vjp) for the state.
``rk4_adjoint(...)``    the discrete adjoint of classic RK4 with a frozen step:
                        gradients of a terminal functional with respect to the
                        initial state and to the mesh control points, with the
                        trajectory checkpointed every ``checkpoint_every`` steps and
                        recomputed segment by segment in the reverse sweep.
The residuals, RK steps and VJPs run in libnsfr.so; the adjoint's stage
combinations (u + a dt k and the cotangent sums) are torch element-wise
operations on the library's outputs.
"""
from __future__ import annotations

import torch


class _Dudt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver):
        out = torch.empty_like(u)
        solver.residual(u, out)
        ctx.solver = solver
        ctx.save_for_backward(u)
        return out

    @staticmethod
    def backward(ctx, grad):
        (u,) = ctx.saved_tensors
        ub = torch.zeros_like(u)
        ctx.solver.vjp(u, grad.contiguous(), ub)
        return ub, None


def dudt(u, solver):
    """du/dt = -(M_m + K_m)^{-1} R(u), differentiable with respect to u."""
    return _Dudt.apply(u, solver)


def _stage_inputs(solver, u, dt):
    """The four RK4 stage inputs y1..y4 and the stage derivatives k1..k3."""
    k = torch.empty_like(u)
    y = [u]
    ks = []
    for a in (0.5, 0.5, 1.0):
        solver.residual(y[-1], k)
        ks.append(k.clone())
        y.append(u + a * dt * ks[-1])
    return y


def rk4_step(solver, u, dt):
    """u + dt/6 (k1 + 2 k2 + 2 k3 + k4) through the library's fused stages (in place on a copy)."""
    v = u.clone()
    solver.rk_step(v, dt=dt)
    return v


def rk4_adjoint(solver, u0, dt, nsteps, terminal_grad, checkpoint_every=10, want_x=True):
    """Gradient of a functional Phi(u_N) of the RK4 trajectory u_{n+1} = RK4(u_n).

    ``terminal_grad(uN)`` returns dPhi/du_N (a tensor shaped like u).  Returns
    (u0_bar, x_bar, uN): the gradient with respect to the initial state, with
    respect to the mesh control points [N_e][(p_geo+1)^3][3] (None unless
    ``want_x``), and the final state.  The step dt is held fixed (a frozen CFL
    step keeps the map smooth).
    """
    # forward sweep: keep every checkpoint_every-th state
    ckpt = {0: u0.clone()}
    u = u0.clone()
    for n in range(nsteps):
        solver.rk_step(u, dt=dt)
        if (n + 1) % checkpoint_every == 0 and (n + 1) < nsteps:
            ckpt[n + 1] = u.clone()
    uN = u.clone()
    lam = terminal_grad(uN).contiguous()
    xbar = None
    if want_x:
        q3 = (solver.p_geo + 1) ** 3
        xbar = torch.zeros((solver.n_el, q3, 3), dtype=torch.float64, device=u0.device)
    starts = sorted(ckpt)
    for si in reversed(range(len(starts))):
        s0 = starts[si]
        s1 = starts[si + 1] if si + 1 < len(starts) else nsteps
        # recompute the segment's states
        states = [ckpt[s0].clone()]
        for _ in range(s0, s1 - 1):
            states.append(rk4_step(solver, states[-1], dt))
        for n in reversed(range(s1 - s0)):
            un = states[n]
            y = _stage_inputs(solver, un, dt)
            kb = [dt / 6.0 * lam, dt / 3.0 * lam, dt / 3.0 * lam, dt / 6.0 * lam]
            new_lam = lam.clone()
            coef = [0.5 * dt, 0.5 * dt, dt]  # y_{s+1} = u + coef[s] k_s
            for s in (3, 2, 1, 0):
                yb = torch.zeros_like(un)
                solver.vjp(y[s], kb[s].contiguous(), yb, xbar)
                new_lam += yb
                if s > 0:
                    kb[s - 1] = kb[s - 1] + coef[s - 1] * yb
            lam = new_lam
    return lam, xbar, uN
