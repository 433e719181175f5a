"""Pins of the oracle's spring-mass system (CPU): edge extraction, rest
state, Newton's third law (net force and net torque vanish, momentum is
conserved), a two-mass harmonic oscillator against its analytic motion with
first-order convergence in dt, the kinetic energy of a uniform motion, and
the degenerate readings (zero-length edge, massless vertex)."""
import numpy as np

import meshgen
from oracle import springs


def test_tet_edges_of_one_tet_and_a_grid():
    e = springs.tet_edges(np.array([[0, 1, 2, 3]]))
    assert e.shape == (12, 2)
    assert {tuple(x) for x in e} == {(a, b) for a in range(4) for b in range(4) if a != b}
    m = meshgen.cube_grid(2, seed=1)
    e = springs.tet_edges(m.tets)
    fwd = {tuple(x) for x in e}
    assert all((b, a) in fwd for a, b in fwd)                  # both directions
    assert len(fwd) == e.shape[0]                               # no repeats
    assert all(a != b for a, b in fwd)


def test_rest_state_has_no_force():
    m = meshgen.cube_grid(3, jitter=0.05, seed=2)
    e = springs.tet_edges(m.tets)
    rest = springs.rest_lengths(m.X, e)
    f = springs.internal_forces(m.X, e, rest, 3.0)
    assert np.max(np.abs(f)) < 1e-13


def test_newton_third_law_and_momentum():
    m = meshgen.cube_grid(2, jitter=0.05, seed=3)
    e = springs.tet_edges(m.tets)
    rest = springs.rest_lengths(m.X, e)
    rng = np.random.default_rng(0)
    q = m.X + 0.05 * rng.normal(size=m.X.shape)
    f = springs.internal_forces(q, e, rest, 2.0)
    scale = np.max(np.abs(f))
    assert np.max(np.abs(f.sum(axis=0))) < 1e-13 * scale * len(f)
    torque = np.cross(q, f).sum(axis=0)
    assert np.max(np.abs(torque)) < 1e-12 * scale * len(f)
    mass = rng.uniform(0.5, 2.0, size=m.n_verts)
    qd = 0.1 * rng.normal(size=m.X.shape)
    p0 = (mass[:, None] * qd).sum(axis=0)
    q1, qd1 = springs.run(q, qd, mass, e, rest, 2.0, 1e-3, 20)
    p1 = (mass[:, None] * qd1).sum(axis=0)
    assert np.max(np.abs(p1 - p0)) < 1e-12


def test_two_masses_oscillate_harmonically():
    """One spring (both directions) between equal masses m: the separation is
    L0 + A cos(w t) with w = sqrt(2 k / m).  The update is first order in dt:
    halving dt halves the error."""
    k, mass, L0, A = 4.0, 2.0, 1.0, 0.05
    w = np.sqrt(2 * k / mass)
    edges = np.array([[0, 1], [1, 0]])
    rest = np.array([L0, L0])
    q0 = np.array([[0.0, 0.0, 0.0], [L0 + A, 0.0, 0.0]])
    T = 2 * np.pi / w
    errs = []
    for n in (4000, 8000):
        dt = T / n
        q, qd = springs.run(q0, np.zeros((2, 3)), np.array([mass, mass]), edges, rest, k, dt, n // 4)
        t = (n // 4) * dt
        sep = q[1, 0] - q[0, 0]
        errs.append(abs(sep - (L0 + A * np.cos(w * t))))
        assert abs(q[0, 0] + q[1, 0] - (L0 + A)) < 1e-12            # centre of mass fixed
    assert errs[0] < 2e-3 * A
    assert 1.6 < errs[0] / errs[1] < 2.4


def test_kinetic_energy_of_uniform_motion():
    rng = np.random.default_rng(1)
    mass = rng.uniform(0.5, 1.5, size=10)
    v = np.array([0.3, -0.4, 1.2])
    e = springs.kinetic_energy(np.tile(v, (10, 1)), mass)
    assert abs(e - 0.5 * mass.sum() * v @ v) < 1e-14 * e


def test_degenerate_readings():
    edges = np.array([[0, 1], [1, 0]])
    q = np.zeros((2, 3))
    f = springs.internal_forces(q, edges, np.array([1.0, 1.0]), 5.0)
    assert np.array_equal(f, np.zeros((2, 3)))                   # zero-length edge
    q = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    q1, qd1 = springs.run(q, np.zeros((2, 3)), np.array([0.0, 1.0]), edges, np.array([1.0, 1.0]), 5.0, 0.01, 3)
    assert np.array_equal(q1[0], q[0]) and np.array_equal(qd1[0], np.zeros(3))   # massless vertex stays
    assert q1[1, 0] < 2.0
