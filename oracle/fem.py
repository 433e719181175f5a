"""FP64 element math and per-tet maps of the oracle (test infrastructure).

A map over the ``tets`` relation computes one value per tet from the four
vertex rows its keys point to and reduces (``+=``) the per-corner results into
vertex fields (Section 4.1: kernels over a relation with field reductions;
Section 6.2 "Reductions").  The element math is that of linear tetrahedra:

    Dm = [X1-X0, X2-X0, X3-X0],  B = Dm^-1,  V = det(Dm) / 6
    Ds = [x1-x0, x2-x0, x3-x0],  F = Ds B
    H  = -V P(F) B^T,  f_a = column a of H (a = 1..3),  f_0 = -(f_1+f_2+f_3)

StVK (Section 7.2, Vega's model):
    E = (F^T F - I)/2,  S = 2 mu E + lam tr(E) I,  P = F S,
    Psi = mu E:E + lam tr(E)^2 / 2
Neo-Hookean (Section 7.3):
    J = det F,  Psi = mu (tr(F^T F) - 3)/2 - mu ln J + lam (ln J)^2 / 2,
    P = mu (F - F^-T) + lam ln J F^-T

Stiffness times vector (K = d^2 E / dx^2 = -df/dx), per tet:
    dF = dDs B,  (K w)_a = column a of V dP B^T,  (K w)_0 = -sum
    StVK: dE = (dF^T F + F^T dF)/2,  dP = dF S + F (2 mu dE + lam tr(dE) I)
    NH:   dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T

Arrays: x, X, u, w are (N_v, 3); tets is (N_t, 4) int; per-tet matrices are
(N_t, 3, 3); mu, lam are scalars or (N_t,) arrays.
"""
from __future__ import annotations

import numpy as np

STVK = "stvk"
NEOHOOKEAN = "nh"


class InvertedElement(ValueError):
    """A tet with det <= 0 (rest shape) or J <= 0 (neo-Hookean)."""


def _edges(x, tets):
    """Edge matrix with columns x[t1]-x[t0], x[t2]-x[t0], x[t3]-x[t0]."""
    x0 = x[tets[:, 0]]
    return np.stack([x[tets[:, 1]] - x0, x[tets[:, 2]] - x0, x[tets[:, 3]] - x0], axis=2)


def rest_shape(X, tets):
    """B = Dm^-1 and V = det(Dm)/6 per tet from the rest positions."""
    Dm = _edges(X, tets)
    det = np.linalg.det(Dm)
    if np.any(det <= 0.0):
        raise InvertedElement("rest tet with non-positive volume")
    return np.linalg.inv(Dm), det / 6.0


def lumped_mass(V, tets, rho, n_verts):
    """Lumped vertex mass m_i = sum over tets containing i of rho V / 4."""
    m = np.zeros(n_verts)
    for a in range(4):
        m += np.bincount(tets[:, a], weights=rho * V / 4.0, minlength=n_verts)
    return m


def deformation_gradient(x, tets, B):
    """F = Ds B."""
    return _edges(x, tets) @ B


def _col(a):
    a = np.asarray(a, dtype=np.float64)
    return a if a.ndim == 0 else a[:, None, None]


def _tr(M):
    return np.trace(M, axis1=1, axis2=2)


def _T(M):
    return np.swapaxes(M, 1, 2)


_I = np.eye(3)


def stvk_energy_density(F, mu, lam):
    E = 0.5 * (_T(F) @ F - _I)
    trE = _tr(E)
    return np.asarray(mu) * np.sum(E * E, axis=(1, 2)) + 0.5 * np.asarray(lam) * trE * trE


def stvk_pk1(F, mu, lam):
    E = 0.5 * (_T(F) @ F - _I)
    S = 2.0 * _col(mu) * E + _col(lam) * _tr(E)[:, None, None] * _I
    return F @ S


def stvk_dpk1(F, dF, mu, lam):
    E = 0.5 * (_T(F) @ F - _I)
    S = 2.0 * _col(mu) * E + _col(lam) * _tr(E)[:, None, None] * _I
    dE = 0.5 * (_T(dF) @ F + _T(F) @ dF)
    return dF @ S + F @ (2.0 * _col(mu) * dE + _col(lam) * _tr(dE)[:, None, None] * _I)


def _nh_parts(F):
    J = np.linalg.det(F)
    if np.any(J <= 0.0):
        raise InvertedElement("inverted element (J <= 0) in the neo-Hookean model")
    Finv = np.linalg.inv(F)
    return J, Finv, _T(Finv)


def nh_energy_density(F, mu, lam):
    J, _, _ = _nh_parts(F)
    lnJ = np.log(J)
    I1 = np.sum(F * F, axis=(1, 2))
    mu = np.asarray(mu)
    lam = np.asarray(lam)
    return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ


def nh_pk1(F, mu, lam):
    J, _, FinvT = _nh_parts(F)
    lnJ = np.log(J)[:, None, None]
    return _col(mu) * (F - FinvT) + _col(lam) * lnJ * FinvT


def nh_dpk1(F, dF, mu, lam):
    J, Finv, FinvT = _nh_parts(F)
    lnJ = np.log(J)[:, None, None]
    tr_FinvdF = _tr(Finv @ dF)[:, None, None]
    return (_col(mu) * dF + (_col(mu) - _col(lam) * lnJ) * (FinvT @ _T(dF) @ FinvT)
            + _col(lam) * tr_FinvdF * FinvT)


_PK1 = {STVK: stvk_pk1, NEOHOOKEAN: nh_pk1}
_DPK1 = {STVK: stvk_dpk1, NEOHOOKEAN: nh_dpk1}
_PSI = {STVK: stvk_energy_density, NEOHOOKEAN: nh_energy_density}


def scatter_corners(per_corner, tets, n_verts):
    """Field reduction ``+=`` of per-corner vectors (N_t, 4, 3) into (N_v, 3)."""
    out = np.zeros((n_verts, 3))
    for a in range(4):
        for c in range(3):
            out[:, c] += np.bincount(tets[:, a], weights=per_corner[:, a, c], minlength=n_verts)
    return out


def _corners_from_cols(M):
    """Per-corner vectors from a (N_t,3,3) matrix whose columns are the
    values for corners 1..3; corner 0 receives minus their sum."""
    out = np.empty((M.shape[0], 4, 3))
    out[:, 1:, :] = _T(M)
    out[:, 0, :] = -M.sum(axis=2)
    return out


def elastic_energy(x, tets, B, V, mu, lam, model):
    """Total elastic energy sum_t V_t Psi(F_t)."""
    F = deformation_gradient(x, tets, B)
    return float(np.sum(V * _PSI[model](F, mu, lam)))


def tet_forces(x, tets, B, V, mu, lam, model, n_verts=None):
    """Elastic vertex forces f = -dE/dx reduced over tets."""
    n_verts = x.shape[0] if n_verts is None else n_verts
    F = deformation_gradient(x, tets, B)
    P = _PK1[model](F, mu, lam)
    H = -V[:, None, None] * (P @ _T(B))
    return scatter_corners(_corners_from_cols(H), tets, n_verts)


def tet_Kv(x, w, tets, B, V, mu, lam, model, n_verts=None):
    """Stiffness-times-vector K(x) w reduced over tets."""
    n_verts = x.shape[0] if n_verts is None else n_verts
    F = deformation_gradient(x, tets, B)
    dF = _edges(w, tets) @ B
    dP = _DPK1[model](F, dF, mu, lam)
    Kw = V[:, None, None] * (dP @ _T(B))
    return scatter_corners(_corners_from_cols(Kw), tets, n_verts)


def tet_diagK(x, tets, B, V, mu, lam, model, n_verts=None):
    """Diagonal of K by probing each element with the 12 unit vectors e_(a,c)
    and keeping entry (a,c) of the element product (slow and literal)."""
    n_verts = x.shape[0] if n_verts is None else n_verts
    F = deformation_gradient(x, tets, B)
    nt = tets.shape[0]
    per_corner = np.zeros((nt, 4, 3))
    for a in range(4):
        for c in range(3):
            dDs = np.zeros((nt, 3, 3))
            if a == 0:
                dDs[:, c, :] = -1.0
            else:
                dDs[:, c, a - 1] = 1.0
            dF = dDs @ B
            dP = _DPK1[model](F, dF, mu, lam)
            Kw = _corners_from_cols(V[:, None, None] * (dP @ _T(B)))
            per_corner[:, a, c] = Kw[:, a, c]
    return scatter_corners(per_corner, tets, n_verts)
