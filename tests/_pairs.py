"""Helpers that set up the same seeded problem for the CUDA library and the oracle."""
import math

import numpy as np

import workloads as wl
from oracle.operators1d import c_hu
from oracle.problem import Problem


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over all entries (all five variables together)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_ctrl(shape, p, kind="tgv", p_geo=None):
    pg = p if p_geo is None else p_geo
    if kind == "tgv":
        return wl.control_points(*shape, pg, -math.pi, math.pi, wl.warp_tgv)
    if kind == "unit":
        return wl.control_points(*shape, pg, 0.0, 1.0, wl.warp_unit)
    if kind == "paper":
        return wl.control_points(*shape, pg, 0.0, 2 * math.pi, wl.make_warp_paper(0.2, 0.0, 2 * math.pi))
    if kind == "affine":
        return wl.control_points(*shape, pg, -math.pi, math.pi)
    raise ValueError(kind)


def c_value(p, c_kind):
    return 0.0 if c_kind == "dg" else c_hu(p)


def oracle_problem(shape, p, c_kind="dg", face_flux="ec", kind="tgv", p_geo=None, nodes="gl"):
    ctrl = make_ctrl(shape, p, kind, p_geo)
    P = Problem(ctrl, shape, p, p_geo=p_geo, c=c_value(p, c_kind), face_flux=face_flux, nodes=nodes)
    return ctrl, P


def state_for(P, kind="tgv", seed=wl.PARITY_SEED):
    xyz = P.node_coords()
    if kind in ("tgv", "paper", "affine"):
        return np.ascontiguousarray(wl.perturbed_tgv_state(xyz, seed))
    return np.ascontiguousarray(wl.perturbed_density_wave_state(xyz, seed))


def oracle_metrics_abi(P):
    """The oracle's metric terms in the library's layouts (C, J, Cf)."""
    ne, n = P.mesh.n_el, P.n
    C = np.ascontiguousarray(np.moveaxis(P.C.reshape(3, 3, ne, n ** 3), 2, 0).reshape(ne, 9, n ** 3))
    J = np.ascontiguousarray(P.J.reshape(ne, n ** 3))
    Cf = np.ascontiguousarray(np.moveaxis(P.geo["Cf"].reshape(3, 3, ne, n * n), 2, 0))
    return C, J, Cf


VARS = ("rho", "rho u", "rho v", "rho w", "rho e")
# The per-variable bars allow this multiple of the oracle's own change under a
# seeded 1-ulp change of the input (see ulp_sensitivity): a different but
# equally valid rounding order moves the result by about that much.
SENS_FACTOR = 4.0


def per_variable_errors(got, ref):
    """Per variable k of [..., 5, n^3] arrays: (||d_k|| / ||ref_k||, max|d_k| / max|ref_k|)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = []
    for k in range(5):
        d = got[..., k, :] - ref[..., k, :]
        r = ref[..., k, :]
        nr, mr = np.linalg.norm(r.ravel()), np.abs(r).max()
        out.append((float(np.linalg.norm(d.ravel()) / nr) if nr > 0 else float(np.linalg.norm(d.ravel())),
                    float(np.abs(d).max() / mr) if mr > 0 else float(np.abs(d).max())))
    return out


ULP_SEED = 977


class _RoundedElementary:
    """numpy with log and exp results moved by -2 ... +2 ulp (seeded; the library's own
    log and exp are held to 2 ulp of libm): stands in for the oracle's numpy inside
    ``ulp_sensitivity``, so that the sensitivity covers the rounding of the elementary
    functions any FP64 evaluation has.  The entropy
    projection amplifies it: ln rho~ = (-s~ - ln 2 beta~)/(gamma-1) is a difference of
    two terms of size |ln p| that nearly cancel, so one ulp of a log is many ulps of
    the face density."""

    def __init__(self, rng):
        self._rng = rng

    def __getattr__(self, name):
        return getattr(np, name)

    def _round(self, y):
        return y + np.spacing(y) * self._rng.integers(-2, 3, size=np.shape(y))

    def log(self, x):
        return self._round(np.log(x))

    def exp(self, x):
        return self._round(np.exp(x))


def ulp_sensitivity(fn, u, seed=ULP_SEED, rel=None):
    """How much the oracle's own result fn(u) moves when the input and the oracle's
    rounding move: every entry of u changes by -1, 0 or +1 ulp (seeded) and every log
    and exp the oracle's physics evaluates by up to 2 ulp; with ``rel`` (2^-24: one
    FP32 ulp) the entries of u change by -rel, 0 or +rel relative instead, and the
    elementary functions are left exact (their rounding is far below that level).
    Returns [(rel-L2, rel-max)] for the five variables, then the all-variable
    (rel-L2, rel-max): the conditioning floor of a comparison between two correct
    evaluations at that precision."""
    from oracle import physics
    u = np.asarray(u, dtype=np.float64)
    rng = np.random.default_rng(seed)
    r = rng.integers(-1, 2, size=u.shape)
    ref = fn(u)
    if rel is None:
        u2 = u + np.spacing(u) * r
        physics.np = _RoundedElementary(rng)
        try:
            got = fn(u2)
        finally:
            physics.np = np
    else:
        got = fn(u * (1.0 + rel * r))
    allv = (rel_l2(got, ref), float(np.abs(np.asarray(got) - ref).max() / np.abs(ref).max()))
    return per_variable_errors(got, ref) + [allv]


def check_parity(got, ref, tol=1e-12, sens=None, floor=None, what="", tol_all=None, sens_all=False):
    """Parity of a [..., 5, n^3] result with the oracle's, element by element:

    * all five variables together: ||got - ref|| / ||ref|| <= tol (or ``tol_all``; with
      ``sens_all``, max(tol, SENS_FACTOR x the all-variable sensitivity));
    * each variable k: ||d_k|| / ||ref_k|| <= bar_k and max|d_k| <= bar_k max|ref_k|,
      bar_k = max(tol, SENS_FACTOR x the oracle's 1-ulp sensitivity of variable k) when
      ``sens`` (from ulp_sensitivity) is given, else tol.

    Returns the per-variable errors."""
    allv = rel_l2(got, ref)
    per = per_variable_errors(got, ref)
    bar_all = tol if tol_all is None else tol_all
    if sens_all:
        bar_all = max(bar_all, SENS_FACTOR * sens[5][0])
    bars = [(max(tol, SENS_FACTOR * s[0]), max(tol, SENS_FACTOR * s[1])) if sens else (tol, tol)
            for s in (sens[:5] if sens else [None] * 5)]
    if floor is not None:
        bar_all = bar_all + floor[0]
        bars = [(b[0] + f[0], b[1] + f[1]) for b, f in zip(bars, floor[1])]
    msg = f"{what}: all-variable {allv:.2e} (bar {bar_all:.1e}); " + "; ".join(
        f"{VARS[k]} L2 {per[k][0]:.2e}/{bars[k][0]:.1e} max {per[k][1]:.2e}/{bars[k][1]:.1e}" for k in range(5))
    assert allv <= bar_all, msg
    for k in range(5):
        assert per[k][0] <= bars[k][0] and per[k][1] <= bars[k][1], msg
    return per


def difference_floor(u1, du):
    """Rounding floor of comparing u1 - u formed from a rounded u1 (|u1| >> |du|): 4 ulp of
    u1 over the norm (all variables, and per variable in L2 and max) of du."""
    eps = np.finfo(np.float64).eps
    u1 = np.asarray(u1)
    du = np.asarray(du)
    allv = 4 * eps * np.linalg.norm(u1) / np.linalg.norm(du)
    per = [(4 * eps * np.linalg.norm(u1[..., k, :]) / np.linalg.norm(du[..., k, :]),
            4 * eps * np.abs(u1[..., k, :]).max() / np.abs(du[..., k, :]).max()) for k in range(5)]
    return allv, per
