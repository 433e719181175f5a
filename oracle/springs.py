"""FP64 spring-mass system on the edges of a tet mesh (oracle, test
infrastructure).

The paper's introductory example (Section 4.1, Figure 1) extends a tetmesh
domain with per-edge rest lengths and per-vertex mass, position q, velocity
qd and force, and runs four kernels:

  initLen                 per edge: rest_len = |head.pos - tail.pos|
  computeInternalForces   per vertex v, over the directed edges e leaving v:
                          v.force += K (e.rest_len dir - dq), dir = dq / |dq|
  applyForces             per vertex: qdd = force / mass,
                          q += qd dt + qdd dt^2 / 2, qd += qdd dt, force = 0
  measureTotalEnergy      E += mass |qd|^2 / 2 over vertices (a global +=)

Readings: the figure takes dq = e.head.q - v.q, which makes the force push
the ends of a stretched spring apart (K (L0 - |dq|) along dq); the system is
read as the spring-mass system the text describes, with the restoring Hooke
force, i.e. the same expression with dq = v.q - e.head.q (force on v
K (|q_h - q_v| - L0) towards the head).  The edges of the mesh are its
distinct vertex pairs that share a tet, each present in both directions; a
zero-length dq contributes no direction (dir = 0, so the force term is
-K dq = 0); a vertex with mass <= 0 does not move (its acceleration is taken
as zero).

Arrays: X, q, qd are (N_v, 3); edges is (N_e, 2) int (tail, head); mass is
(N_v,).  Every step evaluates all forces from the positions at the start of
the step, then moves every vertex.
"""
from __future__ import annotations

import numpy as np


def tet_edges(tets: np.ndarray) -> np.ndarray:
    """Directed edges (tail, head) of a tet mesh: every pair of distinct
    vertices of a tet, both directions, without repeats, sorted."""
    t = np.asarray(tets, dtype=np.int64)
    pairs = []
    for a in range(4):
        for b in range(4):
            if a != b:
                pairs.append(np.stack([t[:, a], t[:, b]], axis=1))
    e = np.unique(np.concatenate(pairs, axis=0), axis=0)
    return e


def rest_lengths(X: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """initLen: |head.pos - tail.pos| per edge."""
    d = X[edges[:, 1]] - X[edges[:, 0]]
    return np.sqrt(np.sum(d * d, axis=1))


def internal_forces(q: np.ndarray, edges: np.ndarray, rest: np.ndarray, k: float) -> np.ndarray:
    """computeInternalForces: force on each tail vertex from its edges."""
    f = np.zeros_like(q, dtype=np.float64)
    for i in range(edges.shape[0]):
        v, h = int(edges[i, 0]), int(edges[i, 1])
        dq = q[v] - q[h]
        n = np.sqrt(np.dot(dq, dq))
        direction = dq / n if n > 0.0 else np.zeros(3)
        f[v] += k * (rest[i] * direction - dq)
    return f


def apply_forces(q: np.ndarray, qd: np.ndarray, f: np.ndarray, mass: np.ndarray, dt: float):
    """applyForces: returns the new (q, qd)."""
    m = np.asarray(mass, dtype=np.float64)
    inv = np.where(m > 0.0, 1.0 / np.where(m > 0.0, m, 1.0), 0.0)
    qdd = f * inv[:, None]
    q_new = q + qd * dt + 0.5 * qdd * dt * dt
    qd_new = qd + qdd * dt
    return q_new, qd_new


def kinetic_energy(qd: np.ndarray, mass: np.ndarray) -> float:
    """measureTotalEnergy: sum of mass |qd|^2 / 2."""
    return float(np.sum(0.5 * np.asarray(mass, dtype=np.float64) * np.sum(qd * qd, axis=1)))


def run(q0, qd0, mass, edges, rest, k, dt, steps):
    """`steps` iterations of computeInternalForces then applyForces."""
    q = np.array(q0, dtype=np.float64)
    qd = np.array(qd0, dtype=np.float64)
    for _ in range(steps):
        f = internal_forces(q, edges, rest, k)
        q, qd = apply_forces(q, qd, f, mass, dt)
    return q, qd
