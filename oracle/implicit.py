"""FP64 linearised backward-Euler step with Jacobi-preconditioned CG
(oracle, test infrastructure).

Section 7.2: each time step computes internal elastic forces and stiffness,
builds a linear system and solves it for the vertex velocities with a
Jacobi-preconditioned conjugate gradient solver; positions follow from the
velocities.  Section 7.3 reuses the same integrator and solver for the
neo-Hookean model.  The paper prints neither the system nor the solver, so
this module writes out the standard one-Newton-step (linearised) backward
Euler:

    A  = M + dt^2 K(x_n)
    b  = dt (f(x_n) + M g - dt K(x_n) v_n)
    A dv = b  (rows and columns of pinned vertices removed)
    v_{n+1} = v_n + dv,   x_{n+1} = x_n + dt v_{n+1}

M is the lumped mass, K the tangent stiffness, f the elastic force.  The
deformed configuration is carried as the displacement u = x - X.

PCG (x_0 = 0, z = r / diag(A)), with the stopping test ||r||_2 <= rtol ||b||_2
checked before every iteration (unpreconditioned 2-norm over free DOFs).
"""
from __future__ import annotations

import numpy as np

from . import fem


class CGBreakdown(RuntimeError):
    """p^T A p <= 0 inside PCG (A not positive definite along p)."""


def pcg(apply_A, b, diag, max_iters, rtol):
    """Jacobi-preconditioned CG for A y = b from y = 0.

    Returns (y, iterations, ||r||/||b||).  ``apply_A`` must already zero the
    rows of constrained DOFs; ``b`` must be zero there.
    """
    y = np.zeros_like(b)
    r = b.copy()
    z = r / diag
    p = z.copy()
    rz = float(np.sum(r * z))
    rr = float(np.sum(r * r))
    bnorm = float(np.sqrt(np.sum(b * b)))
    it = 0
    while it < max_iters and np.sqrt(rr) > rtol * bnorm:
        q = apply_A(p)
        pq = float(np.sum(p * q))
        if not pq > 0.0:
            raise CGBreakdown(f"p^T A p = {pq} at iteration {it}")
        alpha = rz / pq
        y = y + alpha * p
        r = r - alpha * q
        z = r / diag
        rz_new = float(np.sum(r * z))
        rr = float(np.sum(r * r))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        it += 1
    rel = float(np.sqrt(rr) / bnorm) if bnorm > 0 else 0.0
    return y, it, rel


def implicit_step(X, u, v, tets, B, V, mass, mu, lam, model, dt, gravity,
                  pinned, max_iters, rtol):
    """One linearised backward-Euler step.  Returns (u_new, v_new, info).

    X, u, v : (N_v, 3) rest positions, displacement, velocity
    mass    : (N_v,) lumped mass
    pinned  : (N_v,) bool; pinned vertices keep their velocity (dv = 0)
    info    : dict(iters, rel_residual)
    """
    n_verts = X.shape[0]
    x = X + u
    g = np.asarray(gravity, dtype=np.float64).reshape(1, 3)
    m = mass[:, None]
    f = fem.tet_forces(x, tets, B, V, mu, lam, model, n_verts)
    Kv = fem.tet_Kv(x, v, tets, B, V, mu, lam, model, n_verts)
    b = dt * (f + m * g - dt * Kv)
    b[pinned] = 0.0
    diag = m + dt * dt * fem.tet_diagK(x, tets, B, V, mu, lam, model, n_verts)
    diag[pinned] = 1.0

    def apply_A(p):
        q = m * p + dt * dt * fem.tet_Kv(x, p, tets, B, V, mu, lam, model, n_verts)
        q[pinned] = 0.0
        return q

    dv, iters, rel = pcg(apply_A, b, diag, max_iters, rtol)
    v_new = v + dv
    u_new = u + dt * v_new
    return u_new, v_new, dict(iters=iters, rel_residual=rel)
