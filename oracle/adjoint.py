"""FP64 vector-Jacobian product of the linearised backward-Euler step
(oracle, test infrastructure).  St. Venant-Kirchhoff only.

The paper (Sections 7.2, 7.3) does not differentiate its simulations; this
restates the adjoint of the step in ``implicit.py`` from calculus.  With the
step

    x = X + u,  A = M + dt^2 K(x),  b = dt (f(x) + M g - dt K(x) v),
    A dv = b (pinned rows/cols removed),  v' = v + dv,  u' = u + dt v',

and incoming gradients gu' = dL/du', gv' = dL/dv':

    vbar = gv' + dt gu'                     (through u' = u + dt v')
    A lam = vbar  (pinned rows zero)        (adjoint solve, A symmetric)
    dL/du = gu' - dt K lam - dt^2 d/dx[lam^T K(x) v']
    dL/dv = vbar - dt^2 K lam
    dL/dtheta = dt d/dtheta[lam^T f] - dt^2 d/dtheta[lam^T K v']

(the A-dependence of dv and the K v term of b combine into K(x) v').  Per tet,
with dF_a = Da B for a vertex field a and h(F) = dP(F; dF_w) : dF_lam the
term d/dx[lam^T K w] has corners V Q b (b = rows of B, corner 0 minus their
sum), Q = dh/dF:

    C = 2 mu sym(F^T W) + lam_ tr(F^T W) I
    Q = 2 mu F sym(W^T L) + lam_ tr(W^T L) F + L C + 2 mu W sym(F^T L) + lam_ tr(F^T L) W

and, P and dP being linear in (mu, lam_):
    d/dmu[lam^T f]  = -V (2 F E) : L,          d/dlam_[lam^T f]  = -V tr(E) (F : L)
    d/dmu[lam^T K w] = V (W 2E + F 2 sym(F^T W)) : L,
    d/dlam_[lam^T K w] = V (tr(E) (W : L) + tr(F^T W) (F : L))
with W = dF_w, L = dF_lam, E = (F^T F - I)/2.
"""
from __future__ import annotations

import numpy as np

from . import fem, implicit

_I = np.eye(3)


def _T(M):
    return np.swapaxes(M, 1, 2)


def _sym(M):
    return 0.5 * (M + _T(M))


def _tr(M):
    return np.trace(M, axis1=1, axis2=2)


def _col(a):
    a = np.asarray(a, dtype=np.float64)
    return a if a.ndim == 0 else a[:, None, None]


def _ddot(A, B):
    return np.sum(A * B, axis=(1, 2))


def stvk_Q(F, W, L, mu, lam):
    """dh/dF for h(F) = dP(F; W) : L (StVK)."""
    mu_, lam_ = _col(mu), _col(lam)
    FtW = _T(F) @ W
    C = 2.0 * mu_ * _sym(FtW) + lam_ * _tr(FtW)[:, None, None] * _I
    return (2.0 * mu_ * (F @ _sym(_T(W) @ L)) + lam_ * _tr(_T(W) @ L)[:, None, None] * F + L @ C
            + 2.0 * mu_ * (W @ _sym(_T(F) @ L)) + lam_ * _tr(_T(F) @ L)[:, None, None] * W)


def stvk_theta_terms(F, W, L, V):
    """Per-tet (d/dmu, d/dlam) of lam^T f and of lam^T K w."""
    E = 0.5 * (_T(F) @ F - _I)
    trE = _tr(E)
    FL = _ddot(F, L)
    f_mu = -V * _ddot(2.0 * (F @ E), L)
    f_lam = -V * trE * FL
    dE = _sym(_T(F) @ W)
    k_mu = V * _ddot(W @ (2.0 * E) + F @ (2.0 * dE), L)
    k_lam = V * (trE * _ddot(W, L) + _tr(dE) * FL)
    return f_mu, f_lam, k_mu, k_lam


def _edges(a, tets):
    a0 = a[tets[:, 0]]
    return np.stack([a[tets[:, 1]] - a0, a[tets[:, 2]] - a0, a[tets[:, 3]] - a0], axis=2)


def step_vjp(X, u, v, tets, B, V, mass, mu, lam, dt, gravity, pinned, gu_out, gv_out, max_iters=2000,
             rtol=1e-14):
    """dL/d(u, v, mu, lam) of one step from dL/d(u', v').  Returns
    (gu, gv, gmu, glam, forward) with forward = (u', v', info)."""
    n_verts = X.shape[0]
    u1, v1, info = implicit.implicit_step(X, u, v, tets, B, V, mass, mu, lam, fem.STVK, dt, gravity, pinned,
                                          max_iters, rtol)
    x = X + u
    m = mass[:, None]
    vbar = gv_out + dt * gu_out
    rhs = vbar.copy()
    rhs[pinned] = 0.0
    diag = m + dt * dt * fem.tet_diagK(x, tets, B, V, mu, lam, fem.STVK, n_verts)
    diag[pinned] = 1.0

    def apply_A(p):
        q = m * p + dt * dt * fem.tet_Kv(x, p, tets, B, V, mu, lam, fem.STVK, n_verts)
        q[pinned] = 0.0
        return q

    lam_v, _, _ = implicit.pcg(apply_A, rhs, diag, max_iters, rtol)
    Kl = fem.tet_Kv(x, lam_v, tets, B, V, mu, lam, fem.STVK, n_verts)
    F = fem.deformation_gradient(x, tets, B)
    L = _edges(lam_v, tets) @ B
    W = _edges(v1, tets) @ B
    Q = stvk_Q(F, W, L, mu, lam)
    corners = np.empty((tets.shape[0], 4, 3))
    R = V[:, None, None] * (Q @ _T(B))
    corners[:, 1:, :] = _T(R)
    corners[:, 0, :] = -R.sum(axis=2)
    xq = fem.scatter_corners(corners, tets, n_verts)
    gu = gu_out - dt * Kl - dt * dt * xq
    gv = vbar - dt * dt * Kl
    f_mu, f_lam, k_mu, k_lam = stvk_theta_terms(F, W, L, V)
    gmu = dt * f_mu - dt * dt * k_mu
    glam = dt * f_lam - dt * dt * k_lam
    return gu, gv, gmu, glam, (u1, v1, info)


def rollout(X, u0, v0, tets, B, V, mass, mu, lam, dt, gravity, pinned, steps, max_iters=2000, rtol=1e-14):
    """Forward rollout; returns the list of states [(u_0, v_0), ..., (u_T, v_T)]."""
    states = [(u0, v0)]
    u, v = u0, v0
    for _ in range(steps):
        u, v, _ = implicit.implicit_step(X, u, v, tets, B, V, mass, mu, lam, fem.STVK, dt, gravity, pinned,
                                         max_iters, rtol)
        states.append((u, v))
    return states


def rollout_grad(X, u0, v0, tets, B, V, mass, mu, lam, dt, gravity, pinned, steps, gu_T, gv_T, max_iters=2000,
                 rtol=1e-14):
    """Gradient of a loss of the final state through `steps` steps (all
    states kept; the oracle does not checkpoint)."""
    states = rollout(X, u0, v0, tets, B, V, mass, mu, lam, dt, gravity, pinned, steps, max_iters, rtol)
    gu, gv = gu_T, gv_T
    gmu = np.zeros(tets.shape[0])
    glam = np.zeros(tets.shape[0])
    for k in range(steps - 1, -1, -1):
        u, v = states[k]
        gu, gv, dmu, dlam, _ = step_vjp(X, u, v, tets, B, V, mass, mu, lam, dt, gravity, pinned, gu, gv,
                                        max_iters, rtol)
        gmu = gmu + dmu
        glam = glam + dlam
    return gu, gv, gmu, glam, states
