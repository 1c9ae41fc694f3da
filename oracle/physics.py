"""Euler physics: entropy variables, EC two-point fluxes, Roe dissipation.

States U have shape (5, ...) = (rho, rho u, rho v, rho w, rho e); normals
nvec have shape (3, ...) and need not be unit vectors (they are rows of the
metric cofactor, so f . nvec is a reference-direction flux).

Paper: Euler equations with rho e = p/(gamma-1) + rho|u|^2/2 (Sec. "Systems
of Equations"); entropy variables v = U'(u) and potential psi^k (same
section, Eq. entropy pot with flux relationship); the EC condition is the
Tadmor shuffle [[v]] . f_s = [[psi]] (Eq. tadmor shuffle / Eq. EC flux); the
paper's two-point flux is Chandrashekar's (Sec. "Nonlinearly Stable Flux
Reconstruction") with Ismail and Roe's stable logarithmic mean, and Roe's
dissipation for the dissipative face flux (Sec. "Nonlinear Stability").

The paper does not print U or the flux; the standard forms used here are
  U = -rho s/(gamma-1),  s = ln p - gamma ln rho,  psi^k = rho u_k,
  v = [(gamma-s)/(gamma-1) - rho|u|^2/(2p), rho u/p, rho v/p, rho w/p, -rho/p],
and Chandrashekar's flux in the variables (rho, u, beta = rho/(2p)), which is
the solution of the shuffle condition written out below.
"""
from __future__ import annotations

import numpy as np

# Branch point of the series form of the log mean.  Ismail and Roe's series
# 1 + u/3 + u^2/5 + u^3/7 leaves a relative error of about u^4/9, so the
# branch point is chosen with eps^4/9 below the FP64 unit roundoff.
LOGMEAN_EPS = 1.0e-4


def _re(x):
    return np.real(x)


def primitive(U, gamma):
    rho = U[0]
    vel = U[1:4] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * np.sum(vel * vel, axis=0))
    return rho, vel, p


def entropy_function(U, gamma):
    """U(u) = -rho s / (gamma - 1), s = ln p - gamma ln rho."""
    rho, vel, p = primitive(U, gamma)
    s = np.log(p) - gamma * np.log(rho)
    return -rho * s / (gamma - 1.0)


def entropy_variables(U, gamma):
    """v = dU/du for U = -rho s/(gamma-1)."""
    rho, vel, p = primitive(U, gamma)
    s = np.log(p) - gamma * np.log(rho)
    q2 = np.sum(vel * vel, axis=0)
    v1 = (gamma - s) / (gamma - 1.0) - 0.5 * rho * q2 / p
    vm = rho * vel / p
    v5 = -rho / p
    return np.concatenate([v1[None], vm, v5[None]], axis=0)


def conserved_from_entropy(V, gamma):
    """Inverse of ``entropy_variables``.

    u = -v_m/v_5,  s = gamma - (gamma-1)(v_1 - |v_m|^2/(2 v_5)),
    rho = ((-v_5)^{-1} e^{-s})^{1/(gamma-1)},  p = -rho/v_5.
    """
    v1, vm, v5 = V[0], V[1:4], V[4]
    vel = -vm / v5
    s = gamma - (gamma - 1.0) * (v1 - np.sum(vm * vm, axis=0) / (2.0 * v5))
    rho = np.exp((-s - np.log(-v5)) / (gamma - 1.0))
    p = -rho / v5
    rho_e = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=0)
    return np.concatenate([rho[None], rho * vel, rho_e[None]], axis=0)


def entropy_potential(U, nvec):
    """psi . n = rho (u . n) for U = -rho s/(gamma-1)."""
    return np.sum(U[1:4] * nvec, axis=0)


def euler_flux(U, nvec, gamma):
    """Physical flux f(u) . n (Sec. "Systems of Equations")."""
    rho, vel, p = primitive(U, gamma)
    un = np.sum(vel * nvec, axis=0)
    F0 = rho * un
    Fm = rho * vel * un + p * nvec
    F4 = (U[4] + p) * un
    return np.concatenate([F0[None], Fm, F4[None]], axis=0)


def log_mean(a, b):
    """(a - b)/(ln a - ln b), Ismail and Roe's stable form.

    zeta = a/b, f = (zeta-1)/(zeta+1), u = f^2; for u < eps the quotient
    ln(zeta)/(2f) is replaced by its series 1 + u/3 + u^2/5 + u^3/7; the mean
    is (a + b)/(2F).
    """
    zeta = a / b
    f = (zeta - 1.0) / (zeta + 1.0)
    u = f * f
    small = _re(u) < LOGMEAN_EPS
    with np.errstate(divide="ignore", invalid="ignore"):
        f_safe = np.where(small, 1.0, f)
        F_log = np.log(zeta) / (2.0 * f_safe)
    F_ser = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0
    F = np.where(small, F_ser, F_log)
    return (a + b) / (2.0 * F)


def chandrashekar(UL, UR, nvec, gamma):
    """Chandrashekar's EC/KEP two-point flux f_s(u_L, u_R) . n.

    With beta = rho/(2p), ln-means rho_ln, beta_ln, arithmetic means (bars):
      F_rho = rho_ln (u_bar . n)
      F_m   = F_rho u_bar + p_hat n,          p_hat = rho_bar / (2 beta_bar)
      F_E   = F_rho (1/(2(gamma-1) beta_ln) - |u|^2_bar / 2) + u_bar . F_m,
    where |u|^2_bar is the mean of |u_L|^2 and |u_R|^2.  These are the unique
    coefficients for which [[v]] . F = [[rho u . n]] holds for every jump.
    """
    rL, uL, pL = primitive(UL, gamma)
    rR, uR, pR = primitive(UR, gamma)
    bL = rL / (2.0 * pL)
    bR = rR / (2.0 * pR)
    r_ln = log_mean(rL, rR)
    b_ln = log_mean(bL, bR)
    r_bar = 0.5 * (rL + rR)
    b_bar = 0.5 * (bL + bR)
    u_bar = 0.5 * (uL + uR)
    q2_bar = 0.5 * (np.sum(uL * uL, axis=0) + np.sum(uR * uR, axis=0))
    p_hat = r_bar / (2.0 * b_bar)
    un = np.sum(u_bar * nvec, axis=0)
    F0 = r_ln * un
    Fm = F0 * u_bar + p_hat * nvec
    F4 = F0 * (1.0 / (2.0 * (gamma - 1.0) * b_ln) - 0.5 * q2_bar) + np.sum(u_bar * Fm, axis=0)
    return np.concatenate([F0[None], Fm, F4[None]], axis=0)


def ranocha(UL, UR, nvec, gamma):
    """Chandrashekar's flux with Ranocha's pressure terms, f_s(u_L, u_R) . n.

    The paper's EC runs use Chandrashekar's flux "with Ranocha's pressure fix"
    (Sec. "Results"; Ranocha and Gassner, Commun. Appl. Math. Comput. 2022).
    Read here as Ranocha's EC/KEP flux (J. Sci. Comput. 2018), which keeps
    Chandrashekar's mass flux and internal-energy term and replaces his pressure
    average p_hat = rho_bar/(2 beta_bar) in the momentum flux by the arithmetic
    mean p_bar, and the pressure work p_hat (u_bar . n) in the energy flux by the
    product mean (p_L (u_R . n) + p_R (u_L . n))/2:
      F_rho = rho_ln (u_bar . n)
      F_m   = F_rho u_bar + p_bar n
      F_E   = F_rho (1/(2(gamma-1) beta_ln) + (u_L . u_R)/2)
              + (p_L (u_R . n) + p_R (u_L . n))/2.
    Both pressure changes contribute rho_bar [[u]] . n to [[v]] . F, as
    Chandrashekar's p_hat terms do, so the Tadmor shuffle still holds; with
    constant u and p both give the pressure-equilibrium values p n and p u . n.
    """
    rL, uL, pL = primitive(UL, gamma)
    rR, uR, pR = primitive(UR, gamma)
    bL = rL / (2.0 * pL)
    bR = rR / (2.0 * pR)
    r_ln = log_mean(rL, rR)
    b_ln = log_mean(bL, bR)
    u_bar = 0.5 * (uL + uR)
    p_bar = 0.5 * (pL + pR)
    un = np.sum(u_bar * nvec, axis=0)
    F0 = r_ln * un
    Fm = F0 * u_bar + p_bar * nvec
    uLuR = np.sum(uL * uR, axis=0)
    work = 0.5 * (pL * np.sum(uR * nvec, axis=0) + pR * np.sum(uL * nvec, axis=0))
    F4 = F0 * (1.0 / (2.0 * (gamma - 1.0) * b_ln) + 0.5 * uLuR) + work
    return np.concatenate([F0[None], Fm, F4[None]], axis=0)


TWO_POINT = ("chandrashekar", "ranocha")


def two_point(vol_flux):
    """The entropy-conserving two-point flux named by ``vol_flux`` (looked up by name at
    call time, so that a test may replace a flux function of this module)."""
    if vol_flux not in TWO_POINT:
        raise ValueError(vol_flux)
    return globals()[vol_flux]


def _cabs(x):
    """|x| written so that complex-step derivatives follow the real branch."""
    return x * np.sign(_re(x))


def roe_matrix_apply(UL, UR, nvec, gamma, absolute=True):
    """|A_n| (u_R - u_L) (or A_n (u_R - u_L) when absolute=False), Roe averages.

    Roe's linearisation A_n = sum_k n_k df^k/du at the Roe-averaged state,
    expanded in its eigenvectors (acoustic waves q -+ a, entropy and shear
    waves q), with q = u_hat . n_hat; the result is scaled by |n|.
    """
    rL, uL, pL = primitive(UL, gamma)
    rR, uR, pR = primitive(UR, gamma)
    nn = np.sqrt(np.sum(nvec * nvec, axis=0))
    nh = nvec / nn
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    wl = sL / (sL + sR)
    wr = 1.0 - wl
    HL = (UL[4] + pL) / rL
    HR = (UR[4] + pR) / rR
    uh = wl * uL + wr * uR
    Hh = wl * HL + wr * HR
    q2h = np.sum(uh * uh, axis=0)
    a2 = (gamma - 1.0) * (Hh - 0.5 * q2h)
    ah = np.sqrt(a2)
    rh = sL * sR
    qh = np.sum(uh * nh, axis=0)
    dr = rR - rL
    dp = pR - pL
    du = uR - uL
    dq = np.sum(du * nh, axis=0)
    al1 = (dp - rh * ah * dq) / (2.0 * a2)
    al5 = (dp + rh * ah * dq) / (2.0 * a2)
    al2 = dr - dp / a2
    dut = du - dq * nh  # shear jump
    lam1, lam2, lam5 = qh - ah, qh, qh + ah
    if absolute:
        lam1, lam2, lam5 = _cabs(lam1), _cabs(lam2), _cabs(lam5)
    one = np.ones_like(qh)
    r1 = np.concatenate([one[None], uh - ah * nh, (Hh - qh * ah)[None]], axis=0)
    r5 = np.concatenate([one[None], uh + ah * nh, (Hh + qh * ah)[None]], axis=0)
    r2 = np.concatenate([one[None], uh, (0.5 * q2h)[None]], axis=0)
    rs = np.concatenate([(0.0 * one)[None], dut, np.sum(uh * dut, axis=0)[None]], axis=0)
    out = lam1 * al1 * r1 + lam5 * al5 * r5 + lam2 * (al2 * r2 + rh * rs)
    return nn * out


def es_matrix_dissipation(UL, UR, nvec, gamma):
    """Entropy-variable matrix dissipation R |Lambda| T R^T [[v]], scaled by |n|.

    [[v]] = v(u_R) - v(u_L) is the jump of the entropy variables.  R holds the
    right eigenvectors of the flux Jacobian along n^ = n/|n| (acoustic waves
    q -+ a, the entropy wave and the shear waves, q = u . n^), Lambda their
    speeds, and T Barth's scaling (rho/(2 gamma), rho (gamma-1)/gamma, p, p,
    rho/(2 gamma)), for which R T R^T = du/dv: the dissipation is then the
    Roe-type |A_n| [[u]] with [[u]] written through [[v]], and
    [[v]] . R |Lambda| T R^T [[v]] >= 0 makes every face dissipate entropy.  The
    matrices are evaluated at the state (rho_ln, u_bar, p_hat = rho_bar /
    (2 beta_bar)) of Chandrashekar's flux.  The shear waves enter through the
    projection P = I - n^ n^T, so no tangent basis is needed.
    """
    rL, uL, pL = primitive(UL, gamma)
    rR, uR, pR = primitive(UR, gamma)
    bL, bR = rL / (2.0 * pL), rR / (2.0 * pR)
    rho = log_mean(rL, rR)
    u = 0.5 * (uL + uR)
    p = 0.5 * (rL + rR) / (bL + bR)
    nn = np.sqrt(np.sum(nvec * nvec, axis=0))
    nh = nvec / nn
    a = np.sqrt(gamma * p / rho)
    qn = np.sum(u * nh, axis=0)
    q2 = np.sum(u * u, axis=0)
    H = a * a / (gamma - 1.0) + 0.5 * q2
    dv = entropy_variables(UR, gamma) - entropy_variables(UL, gamma)
    dv0, dvm, dv4 = dv[0], dv[1:4], dv[4]
    t_ac = rho / (2.0 * gamma)
    t_en = rho * (gamma - 1.0) / gamma

    def wave(r0, rm, r4):  # r . [[v]]
        return r0 * dv0 + np.sum(rm * dvm, axis=0) + r4 * dv4

    r1m, r1e = u - a * nh, H - a * qn
    r5m, r5e = u + a * nh, H + a * qn
    c1 = _cabs(qn - a) * t_ac * wave(1.0, r1m, r1e)
    c2 = _cabs(qn) * t_en * wave(1.0, u, 0.5 * q2)
    c5 = _cabs(qn + a) * t_ac * wave(1.0, r5m, r5e)
    z = dvm + u * dv4
    Pz = z - nh * np.sum(nh * z, axis=0)
    cs = _cabs(qn) * p
    D0 = c1 + c2 + c5
    Dm = c1 * r1m + c2 * u + c5 * r5m + cs * Pz
    D4 = c1 * r1e + c2 * 0.5 * q2 + c5 * r5e + cs * np.sum(u * Pz, axis=0)
    return nn * np.concatenate([D0[None], Dm, D4[None]], axis=0)


def numerical_flux(UL, UR, nvec, gamma, face_flux="ec", vol_flux="chandrashekar"):
    """Face flux f*(u_L, u_R; n), n pointing from L to R.

    The EC baseline is the volume's two-point flux (``vol_flux``).
    "ec": the EC two-point flux itself; "ec_roe": EC flux minus
    (1/2)|A_n|(u_R - u_L) (Roe dissipation added to the EC baseline);
    "ec_es": EC flux minus (1/2) R |Lambda| T R^T [[v]] (entropy-variable
    matrix dissipation, provably entropy dissipative).
    """
    F = two_point(vol_flux)(UL, UR, nvec, gamma)
    if face_flux == "ec":
        return F
    if face_flux == "ec_roe":
        return F - 0.5 * roe_matrix_apply(UL, UR, nvec, gamma, absolute=True)
    if face_flux == "ec_es":
        return F - 0.5 * es_matrix_dissipation(UL, UR, nvec, gamma)
    raise ValueError(face_flux)


def max_wavespeed(U, gamma):
    """|u| + a at every node (used for the CFL time step)."""
    rho, vel, p = primitive(U, gamma)
    return np.sqrt(np.sum(vel * vel, axis=0)) + np.sqrt(gamma * p / rho)
