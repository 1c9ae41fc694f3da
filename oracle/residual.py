"""NSFR residual, Eq. NSFR, for the collocated GL basis (chi(xi_v) = I).

Eq. NSFR:  (M_m + K_m) du/dt + [chi_v^T chi_f^T][(Q~ - Q~^T) o F^r] 1
           + sum_f sum_k chi_fk^T W_fk n^r . f*^r = 0,
with Q~ - Q~^T the hybridised skew operator (Eq. skew-symm qtilde oper) and
(F^r)_ij = f_s(u~_i, u~_j) . (C_i + C_j)/2 (metric split inside the two-point
flux).  ``residual`` returns R, everything but the mass term, so that
(M_m + K_m) du/dt = -R.

Entropy projection (Sec. "Nonlinearly Stable Flux Reconstruction"):
u~ = u(chi v^), v^ = Pi v(chi u^).  With collocation the projection and the
volume interpolation are identities: u~ = u at volume nodes and
u~_f = u(t_s . v) at face nodes (t_s the 1D extrapolation along the line).

Two evaluations are provided:
  * ``residual``: the sum-factorised form (Sec. "Scalable Evaluations"): the
    volume block of Q~ - Q~^T only couples nodes on a common line in the
    direction d, (W D_d - D_d^T W) = w_perp S1 along that line, and the hybrid
    blocks only couple a face node with the line that ends on it.  Per line
    node a in direction d, face side s (s = -1/+1):
      R_a += sum_b w_perp S1[a,b] f_s(u_a, u_b) . (C_a + C_b)/2
      R_a += s w_perp t_s[a] (phi_a + f* - sum_b t_s[b] phi_b),
      phi_a = f_s(u_a, u~_f) . (C_a + C_f)/2,   f* = f*(u~_L, u~_R; C_f).
  * ``dense_residual``: assembles Q~ - Q~^T, chi_f and F^r literally for each
    element (a brute-force check, feasible for small p only).
"""
from __future__ import annotations

import numpy as np

from . import physics
from .operators1d import apply_1d


def _take(X, a, d):
    """Slice X[..., z, y, x] at index a along reference direction d."""
    return np.take(X, a, axis=X.ndim - 1 - d)


def _index(ndim, a, d):
    idx = [slice(None)] * ndim
    idx[ndim - 1 - d] = a
    return tuple(idx)


def face_states(U, ops, gamma):
    """Entropy-projected face states u~_f = u(t_s . v(u)).

    Returns Uf[d][s] with shape (5, N_e, n, n): the face normal to direction d
    at side s (0: xi_d = -1, 1: xi_d = +1), face nodes ordered as the two
    remaining directions (slowest first).
    """
    V = physics.entropy_variables(U, gamma)
    Uf = []
    for d in range(3):
        row = []
        for s in (0, 1):
            vf = apply_1d(ops.t(s)[None, :], V, d)
            vf = _take(vf, 0, d)
            row.append(physics.conserved_from_entropy(vf, gamma))
        Uf.append(row)
    return Uf


def volume_term(U, C, ops, gamma, vol_flux="chandrashekar"):
    """Volume-volume block of Eq. NSFR, summed along lines (all ordered pairs)."""
    fs = physics.two_point(vol_flux)
    n = ops.n
    R = np.zeros_like(U)
    wperp = np.outer(ops.w, ops.w)
    for d in range(3):
        Cd = C[d]
        for a in range(n):
            ua = _take(U, a, d)
            na = _take(Cd, a, d)
            acc = np.zeros_like(ua)
            for b in range(n):
                if b == a:
                    continue
                F = fs(ua, _take(U, b, d), 0.5 * (na + _take(Cd, b, d)), gamma)
                acc = acc + ops.S1[a, b] * F
            R[_index(R.ndim, a, d)] += wperp * acc
    return R


def face_terms(U, C, nf, Uf, mesh, ops, gamma, face_flux="ec", vol_flux="chandrashekar"):
    """Hybrid volume-face blocks and surface term of Eq. NSFR, line by line."""
    fs = physics.two_point(vol_flux)
    n = ops.n
    R = np.zeros_like(U)
    wperp = np.outer(ops.w, ops.w)
    for d in range(3):
        for s in (0, 1):
            t = ops.t(s)
            sgn = 1.0 if s == 1 else -1.0
            nb = mesh.neighbor(d, s)
            uf_own = Uf[d][s]
            uf_nbr = Uf[d][1 - s][:, nb]
            nfs = nf[d][s]
            if s == 1:   # this element is the face's minus side
                fstar = physics.numerical_flux(uf_own, uf_nbr, nfs, gamma, face_flux, vol_flux)
            else:
                fstar = physics.numerical_flux(uf_nbr, uf_own, nfs, gamma, face_flux, vol_flux)
            phi = [fs(_take(U, a, d), uf_own, 0.5 * (_take(C[d], a, d) + nfs), gamma) for a in range(n)]
            tphi = sum(t[b] * phi[b] for b in range(n))
            for a in range(n):
                R[_index(R.ndim, a, d)] += sgn * wperp * t[a] * (phi[a] + fstar - tphi)
    return R


def residual(U, C, nf, mesh, ops, gamma, face_flux="ec", vol_flux="chandrashekar"):
    """R of Eq. NSFR (sum-factorised), so that (M_m + K_m) du/dt = -R."""
    Uf = face_states(U, ops, gamma)
    return (volume_term(U, C, ops, gamma, vol_flux)
            + face_terms(U, C, nf, Uf, mesh, ops, gamma, face_flux, vol_flux))


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------
def _kron3(A, B, Cm):
    return np.kron(A, np.kron(B, Cm))


def dense_operators(ops):
    """Dense 3D pieces: D_d, W, E_(d,s), face weights, face normals n^r."""
    n = ops.n
    I = np.eye(n)
    D = [_kron3(I, I, ops.D), _kron3(I, ops.D, I), _kron3(ops.D, I, I)]
    W = _kron3(np.diag(ops.w), np.diag(ops.w), np.diag(ops.w))
    E = {}
    for s in (0, 1):
        t = ops.t(s)[None, :]
        E[(0, s)] = _kron3(I, I, t)
        E[(1, s)] = _kron3(I, t, I)
        E[(2, s)] = _kron3(t, I, I)
    Wf = np.diag(np.kron(ops.w, ops.w))
    return D, W, E, Wf


def hybrid_qtilde(ops, d):
    """Q~ for direction d (the operator whose skew part appears in Eq. NSFR).

    Q~ = [[Q - 1/2 sum_f E_f^T B_f E_f, 1/2 E^T B], [-1/2 B E, 1/2 B]],
    Q = W D_d, B_f = W_f diag(n^r_f,d); faces ordered (d', s) = (0,0),(0,1),...
    """
    D, W, E, Wf = dense_operators(ops)
    n = ops.n
    nv, nfp = n ** 3, n ** 2
    N = nv + 6 * nfp
    Q = np.zeros((N, N))
    Q[:nv, :nv] = W @ D[d]
    for dd in range(3):
        for s in (0, 1):
            f = 2 * dd + s
            nr = (1.0 if s == 1 else -1.0) if dd == d else 0.0
            B = Wf * nr
            Ef = E[(dd, s)]
            sl = slice(nv + f * nfp, nv + (f + 1) * nfp)
            Q[:nv, :nv] -= 0.5 * Ef.T @ B @ Ef
            Q[:nv, sl] += 0.5 * Ef.T @ B
            Q[sl, :nv] -= 0.5 * B @ Ef
            Q[sl, sl] += 0.5 * B
    return Q


def dense_residual(U, C, nf, mesh, ops, gamma, face_flux="ec", vol_flux="chandrashekar"):
    """Eq. NSFR assembled literally, element by element (small p only)."""
    n = ops.n
    nv, nfp = n ** 3, n ** 2
    N = nv + 6 * nfp
    ne = U.shape[1]
    D, W, E, Wf = dense_operators(ops)
    QmQT = []
    for d in range(3):
        Qt = hybrid_qtilde(ops, d)
        QmQT.append(Qt - Qt.T)
    Uv = U.reshape(5, ne, nv)
    Vv = physics.entropy_variables(Uv, gamma)
    Cv = C.reshape(3, 3, ne, nv)
    # hybrid node states: volume nodes then the faces' entropy-projected states
    Uh = np.zeros((5, ne, N), dtype=U.dtype)
    Uh[:, :, :nv] = Uv
    for dd in range(3):
        for s in (0, 1):
            f = 2 * dd + s
            vf = np.einsum("kv,xev->xek", E[(dd, s)], Vv)
            Uh[:, :, nv + f * nfp: nv + (f + 1) * nfp] = physics.conserved_from_entropy(vf, gamma)
    R = np.zeros((5, ne, nv), dtype=U.dtype)
    for d in range(3):
        # metric at hybrid nodes: volume rows, and on the faces normal to d the
        # shared face row; rows on other faces are extrapolated (their Q~
        # entries vanish)
        Ch = np.zeros((3, ne, N), dtype=C.dtype)
        Ch[:, :, :nv] = Cv[d]
        for dd in range(3):
            for s in (0, 1):
                f = 2 * dd + s
                sl = slice(nv + f * nfp, nv + (f + 1) * nfp)
                if dd == d:
                    Ch[:, :, sl] = nf[d][s].reshape(3, ne, nfp)
                else:
                    Ch[:, :, sl] = np.einsum("kv,xev->xek", E[(dd, s)], Cv[d])
        A = QmQT[d]
        ii, jj = np.nonzero(A)
        F = physics.two_point(vol_flux)(Uh[:, :, ii], Uh[:, :, jj], 0.5 * (Ch[:, :, ii] + Ch[:, :, jj]), gamma)
        h = np.zeros((5, ne, N), dtype=U.dtype)
        np.add.at(h, (slice(None), slice(None), ii), A[ii, jj] * F)
        R += h[:, :, :nv]
        for dd in range(3):
            for s in (0, 1):
                f = 2 * dd + s
                R += np.einsum("kv,xek->xev", E[(dd, s)], h[:, :, nv + f * nfp: nv + (f + 1) * nfp])
    # surface term sum_f chi_f^T W_f n^r . f*^r
    for d in range(3):
        for s in (0, 1):
            f = 2 * d + s
            nb = mesh.neighbor(d, s)
            own = Uh[:, :, nv + f * nfp: nv + (f + 1) * nfp]
            fo = 2 * d + (1 - s)
            nbr = Uh[:, nb, nv + fo * nfp: nv + (fo + 1) * nfp]
            nvec = nf[d][s].reshape(3, ne, nfp)
            if s == 1:
                fs = physics.numerical_flux(own, nbr, nvec, gamma, face_flux, vol_flux)
            else:
                fs = physics.numerical_flux(nbr, own, nvec, gamma, face_flux, vol_flux)
            sgn = 1.0 if s == 1 else -1.0
            R += np.einsum("kv,k,xek->xev", E[(d, s)], np.diag(Wf) * sgn, fs)
    return R.reshape(U.shape)
