"""Pins of the oracle's Jacobi PCG and linearised backward-Euler step (CPU).

PCG is pinned against a dense LU solve (numpy.linalg.solve); the step is
pinned by free fall (no stiffness: v gains dt*g, x gains dt*v) and by a dense
direct solve of the same linear system whose stiffness is built by finite
differences of the force (so it does not reuse the oracle's K w code).
"""
import numpy as np
import pytest

import meshgen
from oracle import fem, implicit

MODELS = [fem.STVK, fem.NEOHOOKEAN]


def test_pcg_matches_dense_solve():
    rng = np.random.default_rng(0)
    n = 40
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.normal(size=(n, 1))
    y, it, rel = implicit.pcg(lambda p: A @ p, b, np.diag(A)[:, None].copy(), 500, 1e-14)
    assert rel <= 1e-14 and it <= n + 5
    assert np.max(np.abs(y - np.linalg.solve(A, b))) < 1e-12 * np.max(np.abs(y))


def test_pcg_zero_rhs_and_breakdown():
    A = np.diag([1.0, 2.0, 3.0])
    y, it, rel = implicit.pcg(lambda p: A @ p, np.zeros((3, 1)), np.ones((3, 1)), 10, 1e-8)
    assert it == 0 and np.all(y == 0)
    Aind = np.diag([1.0, -4.0, 1.0])
    with pytest.raises(implicit.CGBreakdown):
        implicit.pcg(lambda p: Aind @ p, np.array([[0.1], [1.0], [0.2]]), np.ones((3, 1)), 10, 1e-12)


def _problem(n=2, model=fem.STVK, seed=1):
    m = meshgen.cube_grid(n, jitter=0.01, seed=seed)
    B, V = fem.rest_shape(m.X, m.tets)
    mu, lam = meshgen.lame_from_young(1e5, 0.45)
    rho = 1000.0
    mass = fem.lumped_mass(V, m.tets, rho, m.n_verts)
    u = meshgen.random_displacement(m.X, n, amp=0.05, seed=seed)
    u[m.pinned] = 0.0
    v = 0.3 * meshgen.random_field(m.n_verts, seed=seed)
    v[m.pinned] = 0.0
    return m, B, V, float(mu), float(lam), mass, u, v


def test_free_fall_without_stiffness():
    m, B, V, _, _, mass, u, v = _problem()
    dt, g = 1e-3, np.array([0.0, 0.0, -9.81])
    u1, v1, info = implicit.implicit_step(m.X, u, v, m.tets, B, V, mass, 0.0, 0.0, fem.STVK,
                                          dt, g, m.pinned, 100, 1e-14)
    free = ~m.pinned
    assert np.max(np.abs(v1[free] - (v[free] + dt * g))) < 1e-14
    assert np.max(np.abs(u1[free] - (u[free] + dt * v1[free]))) < 1e-15
    assert np.all(v1[m.pinned] == 0) and np.all(u1[m.pinned] == 0)
    assert info["iters"] <= 2


@pytest.mark.parametrize("model", MODELS)
def test_step_matches_dense_system_from_fd(model):
    m, B, V, mu, lam, mass, u, v = _problem(model=model)
    dt, g = 2e-3, np.array([0.0, 0.0, -9.81])
    x = m.X + u
    nd = 3 * m.n_verts
    eps = 1e-6 / m.n
    K = np.zeros((nd, nd))
    for j in range(nd):
        xp = x.reshape(-1).copy(); xp[j] += eps
        xm = x.reshape(-1).copy(); xm[j] -= eps
        K[:, j] = -(fem.tet_forces(xp.reshape(-1, 3), m.tets, B, V, mu, lam, model)
                    - fem.tet_forces(xm.reshape(-1, 3), m.tets, B, V, mu, lam, model)).reshape(-1) / (2 * eps)
    Mdiag = np.repeat(mass, 3)
    f = fem.tet_forces(x, m.tets, B, V, mu, lam, model).reshape(-1)
    b = dt * (f + Mdiag * np.tile(g, m.n_verts) - dt * K @ v.reshape(-1))
    free = np.repeat(~m.pinned, 3)
    A = np.diag(Mdiag) + dt * dt * K
    dv = np.zeros(nd)
    dv[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    u1, v1, info = implicit.implicit_step(m.X, u, v, m.tets, B, V, mass, mu, lam, model,
                                          dt, g, m.pinned, 500, 1e-13)
    assert info["rel_residual"] <= 1e-13
    ref_v = v.reshape(-1) + dv
    assert np.max(np.abs(v1.reshape(-1) - ref_v)) < 1e-6 * np.max(np.abs(ref_v))
    assert np.max(np.abs(u1.reshape(-1) - (u.reshape(-1) + dt * ref_v))) < 1e-6 * np.max(np.abs(u))
