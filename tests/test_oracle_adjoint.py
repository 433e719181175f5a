"""Pins of the oracle's adjoint (CPU only): every derivative is checked
against central finite differences of the oracle's forward computation, which
is itself pinned in test_oracle_*.py."""
import numpy as np
import pytest

import meshgen
from oracle import adjoint, fem, implicit


def test_Q_is_derivative_of_dP_contraction():
    rng = np.random.default_rng(0)
    F = np.eye(3)[None] + 0.2 * rng.normal(size=(5, 3, 3))
    W = rng.normal(size=(5, 3, 3))
    L = rng.normal(size=(5, 3, 3))
    mu, lam = rng.uniform(1, 2, 5), rng.uniform(2, 5, 5)
    Q = adjoint.stvk_Q(F, W, L, mu, lam)
    h = 1e-6
    for i in range(3):
        for j in range(3):
            Fp = F.copy(); Fp[:, i, j] += h
            Fm = F.copy(); Fm[:, i, j] -= h
            d = (np.sum(fem.stvk_dpk1(Fp, W, mu, lam) * L, axis=(1, 2))
                 - np.sum(fem.stvk_dpk1(Fm, W, mu, lam) * L, axis=(1, 2))) / (2 * h)
            assert np.max(np.abs(d - Q[:, i, j])) < 1e-6 * (1 + np.max(np.abs(Q)))


def test_theta_terms_are_parameter_derivatives():
    m = meshgen.cube_grid(2, jitter=0.05, seed=3)
    B, V = fem.rest_shape(m.X, m.tets)
    x = m.X + meshgen.random_displacement(m.X, 2, amp=0.2, seed=1)
    lv = meshgen.random_field(m.n_verts, seed=2)
    w = meshgen.random_field(m.n_verts, seed=4)
    F = fem.deformation_gradient(x, m.tets, B)
    L = adjoint._edges(lv, m.tets) @ B
    W = adjoint._edges(w, m.tets) @ B
    f_mu, f_lam, k_mu, k_lam = adjoint.stvk_theta_terms(F, W, L, V)
    rng = np.random.default_rng(5)
    mu = rng.uniform(1e4, 2e4, m.n_tets)
    lam = rng.uniform(3e4, 5e4, m.n_tets)

    def lf(mu_, lam_):
        return np.sum(lv * fem.tet_forces(x, m.tets, B, V, mu_, lam_, fem.STVK))

    def lk(mu_, lam_):
        return np.sum(lv * fem.tet_Kv(x, w, m.tets, B, V, mu_, lam_, fem.STVK))

    for t in (0, 7, 23):
        e = np.zeros(m.n_tets); e[t] = 1.0
        # both quantities are linear in (mu, lam): a unit difference is exact
        assert abs((lf(mu + e, lam) - lf(mu, lam)) - f_mu[t]) < 1e-9 * (1 + abs(f_mu[t]))
        assert abs((lf(mu, lam + e) - lf(mu, lam)) - f_lam[t]) < 1e-9 * (1 + abs(f_lam[t]))
        assert abs((lk(mu + e, lam) - lk(mu, lam)) - k_mu[t]) < 1e-9 * (1 + abs(k_mu[t]))
        assert abs((lk(mu, lam + e) - lk(mu, lam)) - k_lam[t]) < 1e-9 * (1 + abs(k_lam[t]))


def _step_problem(seed=2):
    m = meshgen.cube_grid(2, jitter=0.02, seed=seed)
    B, V = fem.rest_shape(m.X, m.tets)
    mu, lam = meshgen.material_perturbed_lame(m.n_tets, 1e5, 0.45, 0.2, seed)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    u = 0.3 * meshgen.random_displacement(m.X, 2, amp=0.05, seed=seed)
    u[m.pinned] = 0
    v = 0.2 * meshgen.random_field(m.n_verts, seed=seed)
    v[m.pinned] = 0
    return m, B, V, mu, lam, mass, u, v


def test_step_vjp_matches_finite_differences():
    m, B, V, mu, lam, mass, u, v = _step_problem()
    dt, g = 5e-3, np.array([0.0, 0.0, -9.81])
    rng = np.random.default_rng(9)
    gu_out = rng.normal(size=u.shape)
    gv_out = rng.normal(size=v.shape)
    gu, gv, gmu, glam, _ = adjoint.step_vjp(m.X, u, v, m.tets, B, V, mass, mu, lam, dt, g, m.pinned,
                                            gu_out, gv_out)

    def phi(u_, v_, mu_, lam_):
        u1, v1, _ = implicit.implicit_step(m.X, u_, v_, m.tets, B, V, mass, mu_, lam_, fem.STVK, dt, g,
                                           m.pinned, 2000, 1e-14)
        return np.sum(gu_out * u1) + np.sum(gv_out * v1)

    for trial in range(3):
        du = rng.normal(size=u.shape) * 1e-3
        dv = rng.normal(size=v.shape)
        dmu = rng.normal(size=mu.shape) * 1e3
        dlam = rng.normal(size=lam.shape) * 1e3
        h = 1e-6
        fd = (phi(u + h * du, v + h * dv, mu + h * dmu, lam + h * dlam)
              - phi(u - h * du, v - h * dv, mu - h * dmu, lam - h * dlam)) / (2 * h)
        an = np.sum(gu * du) + np.sum(gv * dv) + np.sum(gmu * dmu) + np.sum(glam * dlam)
        assert abs(fd - an) < 1e-5 * abs(an), (trial, fd, an)


def test_rollout_grad_matches_finite_differences():
    m, B, V, mu, lam, mass, u, v = _step_problem(seed=4)
    dt, g = 5e-3, np.array([0.0, 0.0, -9.81])
    steps = 4
    u0 = np.zeros_like(u)
    v0 = np.zeros_like(v)

    def loss(u0_, v0_, mu_, lam_):
        st = adjoint.rollout(m.X, u0_, v0_, m.tets, B, V, mass, mu_, lam_, dt, g, m.pinned, steps)
        return np.sum(st[-1][0] ** 2)

    states = adjoint.rollout(m.X, u0, v0, m.tets, B, V, mass, mu, lam, dt, g, m.pinned, steps)
    uT = states[-1][0]
    gu, gv, gmu, glam, _ = adjoint.rollout_grad(m.X, u0, v0, m.tets, B, V, mass, mu, lam, dt, g, m.pinned,
                                                steps, 2 * uT, np.zeros_like(uT))
    rng = np.random.default_rng(3)
    du = rng.normal(size=u.shape) * 1e-3
    du[m.pinned] = 0
    dmu = rng.normal(size=mu.shape) * 1e3
    dlam = rng.normal(size=lam.shape) * 1e3
    h = 1e-6
    fd = (loss(u0 + h * du, v0, mu + h * dmu, lam + h * dlam) - loss(u0 - h * du, v0, mu - h * dmu,
                                                                      lam - h * dlam)) / (2 * h)
    an = np.sum(gu * du) + np.sum(gmu * dmu) + np.sum(glam * dlam)
    assert abs(fd - an) < 1e-5 * abs(an), (fd, an)
