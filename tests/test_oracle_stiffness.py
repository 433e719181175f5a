"""Pins of the oracle's stiffness product K w and diag(K) (CPU only).

K = d^2 E / dx^2 = -df/dx.  Pinned by: central finite differences of the
(separately pinned) force, symmetry u^T K w = w^T K u, positive
semi-definiteness and the six rigid modes in the null space at the rest
shape, and the diagonal of a dense Jacobian built by finite differences.
"""
import numpy as np
import pytest

import meshgen
from oracle import fem

MODELS = [fem.STVK, fem.NEOHOOKEAN]


def _setup(n=2, jitter=0.08, seed=4, amp=0.15):
    m = meshgen.cube_grid(n, jitter=jitter, seed=seed)
    B, V = fem.rest_shape(m.X, m.tets)
    rng = np.random.default_rng(seed)
    mu = rng.uniform(1e4, 2e4, m.n_tets)
    lam = rng.uniform(3e4, 9e4, m.n_tets)
    x = m.X + meshgen.random_displacement(m.X, m.n, amp=amp, seed=seed)
    return m, B, V, mu, lam, x


def _fd_jacobian(m, B, V, mu, lam, x, model, eps):
    """Dense -df/dx by central differences of the oracle force."""
    nd = 3 * m.n_verts
    K = np.zeros((nd, nd))
    for j in range(nd):
        xp = x.copy().reshape(-1); xp[j] += eps
        xm = x.copy().reshape(-1); xm[j] -= eps
        fp = fem.tet_forces(xp.reshape(-1, 3), m.tets, B, V, mu, lam, model)
        fm = fem.tet_forces(xm.reshape(-1, 3), m.tets, B, V, mu, lam, model)
        K[:, j] = -(fp - fm).reshape(-1) / (2 * eps)
    return K


@pytest.mark.parametrize("model", MODELS)
def test_Kv_matches_force_finite_difference(model):
    m, B, V, mu, lam, x = _setup()
    w = meshgen.random_field(m.n_verts, seed=3)
    Kw = fem.tet_Kv(x, w, m.tets, B, V, mu, lam, model)
    eps = 1e-6 / m.n
    fd = -(fem.tet_forces(x + eps * w, m.tets, B, V, mu, lam, model)
           - fem.tet_forces(x - eps * w, m.tets, B, V, mu, lam, model)) / (2 * eps)
    assert np.max(np.abs(Kw - fd)) < 1e-6 * np.max(np.abs(Kw))


@pytest.mark.parametrize("model", MODELS)
def test_K_is_symmetric(model):
    m, B, V, mu, lam, x = _setup(n=3)
    u = meshgen.random_field(m.n_verts, seed=5)
    w = meshgen.random_field(m.n_verts, seed=6)
    a = np.sum(u * fem.tet_Kv(x, w, m.tets, B, V, mu, lam, model))
    b = np.sum(w * fem.tet_Kv(x, u, m.tets, B, V, mu, lam, model))
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))


def _dense_K(m, B, V, mu, lam, x, model):
    nd = 3 * m.n_verts
    K = np.zeros((nd, nd))
    for j in range(nd):
        e = np.zeros(nd); e[j] = 1.0
        K[:, j] = fem.tet_Kv(x, e.reshape(-1, 3), m.tets, B, V, mu, lam, model).reshape(-1)
    return K


@pytest.mark.parametrize("model", MODELS)
def test_rest_stiffness_psd_with_rigid_null_space(model):
    m, B, V, mu, lam, _ = _setup(n=2)
    K = _dense_K(m, B, V, mu, lam, m.X, model)
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert ev.min() > -1e-9 * ev.max()
    assert np.sum(ev < 1e-9 * ev.max()) == 6       # exactly the rigid modes
    modes = []
    for c in range(3):
        t = np.zeros_like(m.X); t[:, c] = 1.0
        modes.append(t)
        axis = np.zeros(3); axis[c] = 1.0
        modes.append(np.cross(axis, m.X))            # infinitesimal rotation
    for r in modes:
        Kr = fem.tet_Kv(m.X, r, m.tets, B, V, mu, lam, model)
        assert np.max(np.abs(Kr)) < 1e-9 * ev.max()


@pytest.mark.parametrize("model", MODELS)
def test_diagK_matches_fd_jacobian_diagonal(model):
    m, B, V, mu, lam, x = _setup(n=2)
    d = fem.tet_diagK(x, m.tets, B, V, mu, lam, model)
    J = _fd_jacobian(m, B, V, mu, lam, x, model, eps=1e-6 / m.n)
    assert np.max(np.abs(d.reshape(-1) - np.diag(J))) < 1e-6 * np.max(np.abs(d))


def test_stvk_and_nh_agree_at_small_strain():
    """Both models linearise to the same K at the rest shape."""
    m, B, V, mu, lam, _ = _setup(n=2)
    w = meshgen.random_field(m.n_verts, seed=8)
    a = fem.tet_Kv(m.X, w, m.tets, B, V, mu, lam, fem.STVK)
    b = fem.tet_Kv(m.X, w, m.tets, B, V, mu, lam, fem.NEOHOOKEAN)
    assert np.max(np.abs(a - b)) < 1e-9 * np.max(np.abs(a))


def test_nh_inverted_element_raises():
    m, B, V, mu, lam, _ = _setup(n=1, jitter=0.0)
    x = m.X.copy()
    x[:, 2] = -x[:, 2]                               # reflect: every J < 0
    with pytest.raises(fem.InvertedElement):
        fem.tet_forces(x, m.tets, B, V, mu, lam, fem.NEOHOOKEAN)
