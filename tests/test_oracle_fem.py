"""Pins of the FP64 oracle's element math and maps (CPU only).

The paper prints no FEM formulas or worked values (Sections 7.2 and 7.3 only
name StVK and neo-Hookean), so the oracle is pinned by what mathematics and
mechanics fix independently of its own code: the rest shape reproduces affine
maps, volumes agree with the divergence theorem, forces vanish at rest and
under rigid motions, net force and torque balance, forces are minus the
energy gradient, a uniform deformation produces exactly the boundary
tractions of the analytic stress, both models reduce to linear elasticity at
small strain, and K is the symmetric Jacobian of -f.
"""
import json
import os

import numpy as np
import pytest

import meshgen
from oracle import fem

MODELS = [fem.STVK, fem.NEOHOOKEAN]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh(n=3, jitter=0.05, seed=7, permute=False):
    m = meshgen.cube_grid(n, jitter=jitter, seed=seed, permute=permute)
    B, V = fem.rest_shape(m.X, m.tets)
    return m, B, V


def _boundary_triangles(tets):
    """Faces used by exactly one tet, oriented outward (positive tets)."""
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 3, 2]],
                            tets[:, [0, 1, 3]], tets[:, [0, 2, 1]]])
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return faces[cnt[inv.ravel()] == 1], cnt


def test_mesh_is_conforming_and_counts():
    for n in (1, 2, 3, 5):
        m = meshgen.cube_grid(n)
        assert m.n_verts == (n + 1) ** 3 and m.n_tets == 5 * n ** 3
        bt, cnt = _boundary_triangles(m.tets.astype(np.int64))
        assert cnt.max() <= 2                       # a face is shared by at most 2 tets
        assert bt.shape[0] == 12 * n * n            # 2 triangles per boundary square


def test_volumes_match_divergence_theorem():
    m, B, V = _mesh(4, jitter=0.1, seed=3)
    assert np.all(V > 0)
    bt, _ = _boundary_triangles(m.tets.astype(np.int64))
    X = m.X
    vol = np.sum(np.einsum("ij,ij->i", X[bt[:, 0]], np.cross(X[bt[:, 1]], X[bt[:, 2]]))) / 6.0
    assert abs(V.sum() - vol) < 1e-13
    m0, _, V0 = _mesh(4, jitter=0.0)
    assert abs(V0.sum() - 1.0) < 1e-13             # unit cube
    assert abs(fem.lumped_mass(V0, m0.tets, 1000.0, m0.n_verts).sum() - 1000.0) < 1e-9


def test_single_tet_volume_against_convex_hull():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(11)
    for _ in range(5):
        P = rng.normal(size=(4, 3))
        tets = np.array([[0, 1, 2, 3]])
        if np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1)) < 0:
            tets = np.array([[0, 1, 3, 2]])
        _, V = fem.rest_shape(P, tets)
        assert abs(V[0] - spatial.ConvexHull(P).volume) < 1e-12


def test_rest_shape_reproduces_affine_maps():
    m, B, V = _mesh(3, jitter=0.1)
    rng = np.random.default_rng(1)
    A = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    x = m.X @ A.T + rng.normal(size=3)
    F = fem.deformation_gradient(x, m.tets, B)
    assert np.max(np.abs(F - A)) < 1e-12


@pytest.mark.parametrize("model", MODELS)
def test_force_zero_at_rest_and_rigid_motion(model):
    m, B, V = _mesh(3, jitter=0.08)
    mu, lam = 3.4e4, 3.1e5
    scale = (mu + lam) / 9.0          # per-tet force scale at unit strain, h = 1/3
    f0 = fem.tet_forces(m.X, m.tets, B, V, mu, lam, model)
    assert np.max(np.abs(f0)) < 1e-12 * scale
    R = meshgen.random_rotation(4)
    x = m.X @ R.T + np.array([0.3, -2.0, 1.5])
    fr = fem.tet_forces(x, m.tets, B, V, mu, lam, model)
    assert np.max(np.abs(fr)) < 1e-11 * scale


@pytest.mark.parametrize("model", MODELS)
def test_net_force_and_torque_vanish(model):
    m, B, V = _mesh(3, jitter=0.08)
    u = meshgen.random_displacement(m.X, m.n, amp=0.2, seed=5, smooth=0.05)
    x = m.X + u
    mu, lam = np.full(m.n_tets, 2e4), np.full(m.n_tets, 9e4)
    f = fem.tet_forces(x, m.tets, B, V, mu, lam, model)
    s = np.max(np.abs(f))
    assert s > 0
    assert np.max(np.abs(f.sum(0))) < 1e-12 * s * m.n_verts
    assert np.max(np.abs(np.cross(x, f).sum(0))) < 1e-12 * s * m.n_verts


@pytest.mark.parametrize("model", MODELS)
def test_force_is_minus_energy_gradient(model):
    m, B, V = _mesh(2, jitter=0.08)
    rng = np.random.default_rng(2)
    mu = rng.uniform(1e4, 2e4, m.n_tets)
    lam = rng.uniform(5e4, 9e4, m.n_tets)
    x = m.X + meshgen.random_displacement(m.X, m.n, amp=0.15, seed=9)
    f = fem.tet_forces(x, m.tets, B, V, mu, lam, model)
    eps = 1e-6 / m.n
    fd = np.zeros_like(f)
    for i in range(m.n_verts):
        for c in range(3):
            xp = x.copy(); xp[i, c] += eps
            xm = x.copy(); xm[i, c] -= eps
            fd[i, c] = -(fem.elastic_energy(xp, m.tets, B, V, mu, lam, model)
                         - fem.elastic_energy(xm, m.tets, B, V, mu, lam, model)) / (2 * eps)
    assert np.max(np.abs(f - fd)) < 1e-6 * np.max(np.abs(f))


def _analytic_pk1_diag(model, s, mu, lam):
    """P for F = diag(s1, s2, s3), derived by hand from the energy densities:
    StVK  P_ii = s_i (mu (s_i^2 - 1) + lam/2 sum_j (s_j^2 - 1));
    NH    P_ii = mu (s_i - 1/s_i) + lam ln(s1 s2 s3) / s_i."""
    s = np.asarray(s, dtype=np.float64)
    if model == fem.STVK:
        return np.diag(s * (mu * (s * s - 1.0) + 0.5 * lam * np.sum(s * s - 1.0)))
    return np.diag(mu * (s - 1.0 / s) + lam * np.log(np.prod(s)) / s)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("rotate", [False, True])
def test_patch_uniform_deformation_gives_boundary_tractions(model, rotate):
    """x = F X with F uniform: every vertex force equals -P g_i, where g_i is
    the area-weighted outward normal of the rest boundary triangles at i over
    3 (the integral of the hat function times n); interior vertices get 0."""
    m, B, V = _mesh(3, jitter=0.06, seed=21)
    mu, lam = 1.3e4, 6.1e4
    s = np.array([1.12, 0.93, 1.05])
    F = np.diag(s)
    P = _analytic_pk1_diag(model, s, mu, lam)
    if rotate:
        R = meshgen.random_rotation(8)
        F, P = R @ F, R @ P            # frame indifference: P(RF) = R P(F)
    x = m.X @ F.T
    f = fem.tet_forces(x, m.tets, B, V, mu, lam, model)
    bt, _ = _boundary_triangles(m.tets.astype(np.int64))
    X = m.X
    an = 0.5 * np.cross(X[bt[:, 1]] - X[bt[:, 0]], X[bt[:, 2]] - X[bt[:, 0]])
    g = np.zeros_like(X)
    for k in range(3):
        np.add.at(g, bt[:, k], an / 3.0)
    expect = -g @ P.T
    assert np.max(np.abs(f - expect)) < 1e-10 * np.max(np.abs(expect))


@pytest.mark.parametrize("model", MODELS)
def test_small_strain_limit_is_linear_elasticity(model):
    """At infinitesimal strain both models give sigma = 2 mu eps + lam tr(eps) I;
    with (mu, lam) from (E, nu), uniaxial stress E*eps goes with lateral
    strain -nu*eps and zero lateral stress."""
    E, nu = 2.5e5, 0.31
    mu, lam = meshgen.lame_from_young(E, nu)
    eps = 1e-7
    F = np.diag([1 + eps, 1 - nu * eps, 1 - nu * eps])[None]
    P = fem.stvk_pk1(F, mu, lam) if model == fem.STVK else fem.nh_pk1(F, mu, lam)
    assert abs(P[0, 0, 0] / eps - E) < 1e-5 * E
    assert abs(P[0, 1, 1] / eps) < 1e-5 * E and abs(P[0, 2, 2] / eps) < 1e-5 * E
    # shear: P_01 = 2 mu * (gamma / 2) for F = I + gamma e0 e1^T
    F = (np.eye(3) + eps * np.outer([1, 0, 0], [0, 1, 0]))[None]
    P = fem.stvk_pk1(F, mu, lam) if model == fem.STVK else fem.nh_pk1(F, mu, lam)
    assert abs(P[0, 0, 1] / eps - mu) < 1e-5 * mu


@pytest.mark.parametrize("model", MODELS)
def test_pk1_is_energy_derivative(model):
    rng = np.random.default_rng(3)
    F = np.eye(3)[None] + 0.2 * rng.normal(size=(6, 3, 3))
    mu, lam = 1.7, 4.2
    psi = fem.stvk_energy_density if model == fem.STVK else fem.nh_energy_density
    P = fem.stvk_pk1(F, mu, lam) if model == fem.STVK else fem.nh_pk1(F, mu, lam)
    h = 1e-6
    for i in range(3):
        for j in range(3):
            Fp = F.copy(); Fp[:, i, j] += h
            Fm = F.copy(); Fm[:, i, j] -= h
            d = (psi(Fp, mu, lam) - psi(Fm, mu, lam)) / (2 * h)
            assert np.max(np.abs(d - P[:, i, j])) < 1e-7 * (1 + np.max(np.abs(P)))
    assert np.max(np.abs(psi(np.eye(3)[None], mu, lam))) < 1e-15


def test_single_tet_closed_form_golden():
    """Hand-derived forces on the unit right tet (tests/golden/single_tet_closed_form.json)."""
    with open(os.path.join(GOLDEN, "single_tet_closed_form.json")) as fh:
        gold = json.load(fh)
    X = np.array(gold["X"], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3]])
    B, V = fem.rest_shape(X, tets)
    for case in gold["cases"]:
        F = np.array(case["F"], dtype=np.float64)
        x = X @ F.T
        f = fem.tet_forces(x, tets, B, V, case["mu"], case["lam"], case["model"])
        assert np.max(np.abs(f - np.array(case["f"]))) < 1e-13, case["name"]


def test_lumped_mass_of_one_tet_is_a_quarter_at_each_vertex():
    """A single rest tet: each of its four vertices carries rho V / 4, and a
    vertex outside the tet carries nothing (per vertex, not just the total)."""
    rng = np.random.default_rng(5)
    P = rng.normal(size=(5, 3))
    tets = np.array([[4, 2, 0, 3]])
    if np.linalg.det(np.stack([P[2] - P[4], P[0] - P[4], P[3] - P[4]], 1)) < 0:
        tets = np.array([[4, 2, 3, 0]])
    _, V = fem.rest_shape(P, tets)
    m = fem.lumped_mass(V, tets, 1000.0, 5)
    vol = abs(np.linalg.det(np.stack([P[2] - P[4], P[0] - P[4], P[3] - P[4]], 1))) / 6.0
    assert np.array_equal(m == 0, np.array([False, True, False, False, False]))
    assert np.allclose(m[[0, 2, 3, 4]], 1000.0 * vol / 4.0, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_lumped_mass_per_vertex_on_an_unjittered_grid(n):
    """Closed form on an unjittered grid of spacing h = 1/n.  In the 5-tet
    split of a cube the central tet has volume h^3/3 and each corner tet
    h^3/6.  A cube corner of the central tet lies in it and in three corner
    tets (5 h^3/6 in all), a cube corner of a corner tet lies in that tet
    alone (h^3/6).  The central tet takes the corners whose global index sum
    i + j + k is odd in both cube parities, so every vertex gets rho h^3/24
    per adjacent cube, times 5 if i + j + k is odd."""
    m = meshgen.cube_grid(n, jitter=0.0)
    _, V = fem.rest_shape(m.X, m.tets)
    rho = 1000.0
    mass = fem.lumped_mass(V, m.tets, rho, m.n_verts)
    h = 1.0 / n
    idx = np.arange(m.n_verts)
    i, j, k = idx % (n + 1), (idx // (n + 1)) % (n + 1), idx // (n + 1) ** 2
    assert np.allclose(m.X, np.stack([i, j, k], 1) * h, atol=1e-15)
    cubes = np.ones(m.n_verts)
    for g in (i, j, k):
        cubes *= np.where((g == 0) | (g == n), 1, 2)
    want = rho * h ** 3 / 24.0 * cubes * np.where((i + j + k) % 2 == 1, 5.0, 1.0)
    assert np.max(np.abs(mass - want)) < 1e-12 * rho * h ** 3
