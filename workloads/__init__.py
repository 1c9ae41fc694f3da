"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds only the *definitions of the inputs*: the mesh-warping
formulas, the analytic initial states and a seeded smooth perturbation.  It
contains none of the discretisation's arithmetic (no quadrature, no operators,
no fluxes): the caller supplies the physical coordinates at which a state is
sampled, and the mesh control points sit at equispaced reference positions, so
nothing here depends on Gauss or Lobatto nodes.

Layouts follow the library's C ABI:
  * control points  : [N_e][(p_geo+1)^3][3], xi fastest, element
                      e = ex + nx*(ey + ny*ez);
  * node coordinates: [N_e][3][n^3] (physical x, y, z at solution nodes);
  * conserved state : [N_e][5][n^3] = (rho, rho u, rho v, rho w, rho e).

Workloads (the paper's analytic test problems, Sec. "Results"):
  * the inviscid Taylor-Green vortex initial state (Sec. "Inviscid Taylor
    Green Vortex", Eq. for rho, u, v, w, p) written with the pressure
    p = 100/gamma + (cos2x + cos2y)(cos2z + 2)/16, which is the paper's
    expression (cos2x cos2z + 2cos2x + 2cos2y + cos2y cos2z)/16 factored;
  * a smooth density wave rho = 2 + 0.1 sin(2 pi (x+y+z-3t)), u=v=w=1, p=1,
    an exact solution of the Euler equations used for convergence studies;
  * three warps: the non-symmetric warp of the Taylor-Green benchmark on
    [-pi, pi]^3, the same warp rescaled to [0,1]^3, and the paper's own warp
    (Eq. "warped grid") with amplitude beta on [x_L, x_R]^3.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4
PARITY_SEED = 20231207


# ---------------------------------------------------------------------------
# warps: maps (X, Y, Z) on the undeformed box -> physical (x, y, z)
# ---------------------------------------------------------------------------
def warp_none(X, Y, Z):
    return X, Y, Z


def warp_tgv(X, Y, Z):
    """Non-symmetric warp of the Taylor-Green benchmark on [-pi, pi]^3.

    Every displacement vanishes on the faces of the box and is 2 pi periodic,
    so the warped grid stays periodic.
    """
    x = X + 0.10 * np.sin(X) * np.sin(2 * Y) * np.sin(Z)
    y = Y + 0.05 * np.sin(2 * X) * np.sin(Y) * np.sin(3 * Z)
    z = Z + 0.08 * np.sin(X) * np.sin(3 * Y) * np.sin(2 * Z)
    return x, y, z


def warp_unit(X, Y, Z):
    """The Taylor-Green warp moved to [0, 1]^3 with amplitudes scaled by 1/(2 pi)."""
    tp = 2.0 * math.pi
    Xt, Yt, Zt = tp * X, tp * Y, tp * Z
    s = 1.0 / tp
    x = X + s * 0.10 * np.sin(Xt) * np.sin(2 * Yt) * np.sin(Zt)
    y = Y + s * 0.05 * np.sin(2 * Xt) * np.sin(Yt) * np.sin(3 * Zt)
    z = Z + s * 0.08 * np.sin(Xt) * np.sin(3 * Yt) * np.sin(2 * Zt)
    return x, y, z


def make_warp_paper(beta, x_lo, x_hi):
    """The paper's warp (Sec. "Results", Eq. warped grid) with l=(x_R-x_L)/(2 pi)."""
    l = (x_hi - x_lo) / (2.0 * math.pi)

    def warp(a, b, c):
        x = a + beta * np.sin(a / l) * np.sin(b / l) * np.sin(2 * c / l)
        y = b + beta * np.sin(4 * a / l) * np.sin(b / l) * np.sin(3 * c / l)
        z = c + beta * np.sin(2 * a / l) * np.sin(5 * b / l) * np.sin(c / l)
        return x, y, z

    return warp


def make_warp_scaled(warp, amp):
    """Scale the displacement of ``warp`` by ``amp`` (for mesh-amplitude studies)."""

    def w(X, Y, Z):
        x, y, z = warp(X, Y, Z)
        return X + amp * (x - X), Y + amp * (y - Y), Z + amp * (z - Z)

    return w


WARPS = {"none": warp_none, "tgv": warp_tgv, "unit": warp_unit,
         # the paper's Taylor-Green timing mesh: its warp with beta = 1/5 on [-pi, pi]^3
         "paper": make_warp_paper(0.2, -math.pi, math.pi),
         # the paper's manufactured-solution mesh: its warp with beta = 1/50 on [-1, 1]^3
         "mms": make_warp_paper(0.02, -1.0, 1.0)}


# ---------------------------------------------------------------------------
# mesh control points
# ---------------------------------------------------------------------------
def control_points(nx, ny, nz, p_geo, lo, hi, warp=warp_none, dtype=np.float64):
    """Control points of a structured periodic hexahedral grid.

    Each element is the image of the reference cube [-1,1]^3 under a degree
    ``p_geo`` tensor-product Lagrange map whose control points sit at the
    equispaced reference nodes xi_k = -1 + 2k/p_geo.  The undeformed element
    (ex,ey,ez) covers [lo + ex h_x, lo + (ex+1) h_x] x ... ; ``warp`` moves
    every control point.  Returns an array [N_e][(p_geo+1)^3][3].
    """
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (3,))
    ne = (nx, ny, nz)
    h = (hi - lo) / np.asarray(ne, dtype=np.float64)
    q = p_geo + 1
    s = np.arange(q, dtype=np.float64) / p_geo  # (xi+1)/2 at equispaced nodes
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()  # element order: ex fastest
    sk, sj, si = np.meshgrid(s, s, s, indexing="ij")  # node order: xi fastest
    si, sj, sk = si.ravel(), sj.ravel(), sk.ravel()
    X = lo[0] + (ex[:, None] + si[None, :]) * h[0]
    Y = lo[1] + (ey[:, None] + sj[None, :]) * h[1]
    Z = lo[2] + (ez[:, None] + sk[None, :]) * h[2]
    x, y, z = warp(X, Y, Z)
    return np.ascontiguousarray(np.stack([x, y, z], axis=-1).astype(dtype))


# ---------------------------------------------------------------------------
# analytic states, evaluated at caller-supplied node coordinates
# ---------------------------------------------------------------------------
def conserved_from_primitive(rho, u, v, w, p, gamma=GAMMA):
    """Stack (rho, rho u, rho v, rho w, rho e) with rho e = p/(gamma-1) + rho|u|^2/2."""
    rho_e = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, rho_e], axis=-2)


def tgv_state(xyz, gamma=GAMMA):
    """Inviscid Taylor-Green vortex initial state at coordinates [N_e][3][n^3]."""
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    rho = np.ones_like(x)
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    p = 100.0 / gamma + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return conserved_from_primitive(rho, u, v, w, p, gamma)


def density_wave_state(xyz, t=0.0, gamma=GAMMA):
    """Exact density wave rho = 2 + 0.1 sin(2pi(x+y+z-3t)), u=v=w=1, p=1."""
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    rho = 2.0 + 0.1 * np.sin(2.0 * math.pi * (x + y + z - 3.0 * t))
    one = np.ones_like(x)
    return conserved_from_primitive(rho, one, one, one, one, gamma)


def manufactured_state(xyz, t=0.0):
    """Gassner et al.'s manufactured solution (the paper's convergence test) at
    coordinates [N_e][3][n^3]: rho = 2 + 0.1 sin(pi(x+y+z-2t)), u=v=w=1, rho e = rho^2."""
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    rho = 2.0 + 0.1 * np.sin(math.pi * (x + y + z - 2.0 * t))
    return np.stack([rho, rho, rho, rho, rho * rho], axis=-2)


def free_stream_state(xyz, rho=1.3, vel=(0.7, -0.4, 0.25), p=2.1, gamma=GAMMA):
    x = xyz[..., 0, :]
    o = np.ones_like(x)
    return conserved_from_primitive(rho * o, vel[0] * o, vel[1] * o, vel[2] * o, p * o, gamma)


def smooth_perturbation(xyz, seed=PARITY_SEED, period=2.0 * math.pi, kmax=3,
                        amp_rel=0.01, amp_vel=0.05):
    """Seeded smooth periodic perturbation fields (d rho/rho, du, dv, dw, dp/p).

    Sums of Fourier modes with integer wave numbers |k_i| <= kmax on a box of
    the given period, random phases and amplitudes from numpy's PCG64 seeded
    generator.  Returns five arrays shaped like xyz[..., 0, :].
    """
    rng = np.random.default_rng(seed)
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    kscale = 2.0 * math.pi / period
    out = []
    for comp in range(5):
        f = np.zeros_like(x)
        nmodes = 6
        for _ in range(nmodes):
            k = rng.integers(-kmax, kmax + 1, size=3)
            if not k.any():
                k[0] = 1
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1)
            f = f + a * np.sin(kscale * (k[0] * x + k[1] * y + k[2] * z) + ph)
        f = f / nmodes
        out.append(f * (amp_vel if comp in (1, 2, 3) else amp_rel))
    return out


def perturbed_tgv_state(xyz, seed=PARITY_SEED, gamma=GAMMA):
    """Taylor-Green state plus a seeded smooth perturbation that breaks its symmetries."""
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    drho, du, dv, dw, dp = smooth_perturbation(xyz, seed)
    rho = 1.0 + drho
    u = np.sin(x) * np.cos(y) * np.cos(z) + du
    v = -np.cos(x) * np.sin(y) * np.cos(z) + dv
    w = dw
    p = (100.0 / gamma + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0) * (1.0 + dp)
    return conserved_from_primitive(rho, u, v, w, p, gamma)


def perturbed_density_wave_state(xyz, seed=PARITY_SEED, gamma=GAMMA):
    drho, du, dv, dw, dp = smooth_perturbation(xyz, seed, period=1.0)
    x, y, z = xyz[..., 0, :], xyz[..., 1, :], xyz[..., 2, :]
    rho = (2.0 + 0.1 * np.sin(2.0 * math.pi * (x + y + z))) * (1.0 + drho)
    return conserved_from_primitive(rho, 1.0 + du, 1.0 + dv, 1.0 + dw, 1.0 + dp, gamma)


def random_cotangent(shape, seed=PARITY_SEED + 1):
    """Seeded standard-normal array (cotangent seeds for adjoint checks)."""
    return np.random.default_rng(seed).standard_normal(shape)


# ---------------------------------------------------------------------------
# named workloads (sizes of the paper-derived configurations)
# ---------------------------------------------------------------------------
def tgv_mesh(n_el, p, warp="tgv", p_geo=None):
    """Control points of the warped periodic Taylor-Green cube [-pi, pi]^3."""
    pg = p if p_geo is None else p_geo
    return control_points(n_el, n_el, n_el, pg, -math.pi, math.pi, WARPS[warp])


def mms_mesh(n_el, p, warp="mms", p_geo=None):
    """n_el^3 elements on [-1, 1]^3 (the manufactured solution's period)."""
    pg = p if p_geo is None else p_geo
    return control_points(n_el, n_el, n_el, pg, -1.0, 1.0, WARPS[warp])


def unit_mesh(n_el, p, warp="unit", p_geo=None):
    pg = p if p_geo is None else p_geo
    return control_points(n_el, n_el, n_el, pg, 0.0, 1.0, WARPS[warp])


def warp_x_only(X, Y, Z):
    """A curvilinear warp of [0,1]^3 whose displacement depends on X only.

    Refining in x alone then resolves the map, which makes a cheap
    convergence study on a curved (non-affine, off-diagonal metric) mesh.
    """
    tp = 2.0 * math.pi
    return (X + 0.03 * np.sin(tp * X), Y + 0.05 * np.sin(tp * X), Z - 0.04 * np.sin(2 * tp * X))


def density_wave_x_state(xyz, t=0.0, gamma=GAMMA):
    """Exact wave rho = 2 + 0.1 sin(2 pi (x - t)), u = (1, 0, 0), p = 1."""
    x = xyz[..., 0, :]
    rho = 2.0 + 0.1 * np.sin(2.0 * math.pi * (x - t))
    one, zero = np.ones_like(x), np.zeros_like(x)
    return conserved_from_primitive(rho, one, zero, zero, one, gamma)
