"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module only *generates* inputs: cube-grid tetrahedral meshes, rest-shape
jitter, per-tet material parameters, id permutations, pinned-vertex masks and
random deformation / direction fields.  It holds none of the finite-element
arithmetic of the method (no Dm^-1, volumes, masses, stresses, forces or
solves); that lives separately in the oracle and in the CUDA library, which
share no code with each other.

Mesh model (Ebb's tetmesh domain, Section 5.2 "Example: FEM tetmesh"): a
``verts`` relation and a ``tets`` relation with a 4-wide key-field
``tets.v[4]`` into ``verts``.  Keys are emitted as int32 (every workload here
has fewer than 2^31 rows).

All random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# 5-tet decomposition of a unit cube.  Corners are (di, dj, dk) in {0,1}^3.
# Even cubes ((i+j+k) even) use the odd-sum corners as the central tet and cut
# one corner tet at each even-sum corner; odd cubes use the mirror split.
# Neighbouring cubes have opposite parity, so shared faces are cut along the
# same diagonal and the mesh is conforming.
# ---------------------------------------------------------------------------
_EVEN_CUBE = (
    ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)),  # central
    ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((1, 1, 0), (0, 1, 0), (1, 0, 0), (1, 1, 1)),
    ((1, 0, 1), (0, 0, 1), (1, 1, 1), (1, 0, 0)),
    ((0, 1, 1), (1, 1, 1), (0, 0, 1), (0, 1, 0)),
)
_ODD_CUBE = (
    ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)),  # central
    ((1, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1)),
    ((0, 1, 0), (1, 1, 0), (0, 0, 0), (0, 1, 1)),
    ((0, 0, 1), (1, 0, 1), (0, 1, 1), (0, 0, 0)),
    ((1, 1, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)),
)


def _orient_template(tmpl):
    """Order each local tet's corners so the integer lattice triple product
    of (c1-c0, c2-c0, c3-c0) is positive (swap the last two keys otherwise).
    Pure integer bookkeeping on lattice offsets: it fixes key order only."""
    out = []
    for t in tmpl:
        c = np.array(t, dtype=np.int64)
        e = c[1:] - c[0]
        s = (e[0, 0] * (e[1, 1] * e[2, 2] - e[1, 2] * e[2, 1])
             - e[0, 1] * (e[1, 0] * e[2, 2] - e[1, 2] * e[2, 0])
             + e[0, 2] * (e[1, 0] * e[2, 1] - e[1, 1] * e[2, 0]))
        assert s != 0
        out.append(t if s > 0 else (t[0], t[1], t[3], t[2]))
    return tuple(out)


EVEN_CUBE = _orient_template(_EVEN_CUBE)
ODD_CUBE = _orient_template(_ODD_CUBE)


@dataclasses.dataclass
class TetMesh:
    """A cube-grid tet mesh over [0,1]^3 with n cubes per side.

    X      : (N_v, 3) float64 rest positions (jittered if requested)
    tets   : (N_t, 4) int32 keys into the vertex relation
    n      : cubes per side
    pinned : (N_v,) bool, True on the bottom face (grid index k == 0)
    grid_k : (N_v,) int64 grid index k of each vertex (after any permutation)
    """
    X: np.ndarray
    tets: np.ndarray
    n: int
    pinned: np.ndarray
    grid_k: np.ndarray

    @property
    def n_verts(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def cube_grid(n: int, jitter: float = 0.0, seed: int = 0,
              permute: bool = False) -> TetMesh:
    """Build the n x n x n cube grid, 5 tets per cube, spacing h = 1/n.

    Vertex id = i + (n+1) * (j + (n+1) * k); tets are listed cube by cube
    (i fastest), 5 per cube.  ``jitter`` is the standard deviation of the
    Gaussian perturbation of every rest coordinate, as a fraction of h.
    ``permute`` applies seeded random permutations to vertex ids and tet ids
    (a mesh with poor locality).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    n1 = n + 1
    h = 1.0 / n
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    # vertex id = i + n1*(j + n1*k)  -> order arrays with i fastest
    ii = ii.transpose(2, 1, 0).reshape(-1)
    jj = jj.transpose(2, 1, 0).reshape(-1)
    kk = kk.transpose(2, 1, 0).reshape(-1)
    X = np.stack([ii, jj, kk], axis=1).astype(np.float64) * h

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci = ci.transpose(2, 1, 0).reshape(-1)
    cj = cj.transpose(2, 1, 0).reshape(-1)
    ck = ck.transpose(2, 1, 0).reshape(-1)
    parity = (ci + cj + ck) & 1
    n_cubes = n * n * n
    tets = np.empty((n_cubes, 5, 4), dtype=np.int64)
    for tmpl, par in ((EVEN_CUBE, 0), (ODD_CUBE, 1)):
        sel = parity == par
        for t, tet in enumerate(tmpl):
            for c, (di, dj, dk) in enumerate(tet):
                tets[sel, t, c] = (ci[sel] + di) + n1 * ((cj[sel] + dj) + n1 * (ck[sel] + dk))
    tets = tets.reshape(-1, 4)

    rng = np.random.Generator(np.random.PCG64(seed))
    if jitter > 0.0:
        X = X + rng.normal(0.0, jitter * h, size=X.shape)
    pinned = kk == 0
    grid_k = kk.astype(np.int64)
    if permute:
        # new vertex id of old vertex o is vperm_inv[o]
        vperm = rng.permutation(X.shape[0])          # new -> old
        vinv = np.empty_like(vperm)
        vinv[vperm] = np.arange(vperm.size)
        X = X[vperm]
        pinned = pinned[vperm]
        grid_k = grid_k[vperm]
        tets = vinv[tets]
        tperm = rng.permutation(tets.shape[0])
        tets = tets[tperm]
    return TetMesh(X=np.ascontiguousarray(X), tets=np.ascontiguousarray(tets.astype(np.int32)),
                   n=n, pinned=pinned, grid_k=grid_k)


def lame_from_young(E, nu):
    """Lame parameters (mu, lambda) of an isotropic material with Young's
    modulus E and Poisson ratio nu (material specification of the inputs)."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def material_loguniform_E(n_tets: int, E_lo: float, E_hi: float, nu: float, seed: int):
    """Per-tet (mu, lambda) with E log-uniform in [E_lo, E_hi] and fixed nu."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    E = np.exp(rng.uniform(math.log(E_lo), math.log(E_hi), size=n_tets))
    return lame_from_young(E, np.full(n_tets, nu))


def material_perturbed_lame(n_tets: int, E: float, nu: float, rel: float, seed: int):
    """Per-tet (mu, lambda), each drawn uniformly within +-rel of the values
    given by (E, nu)."""
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    mu0, lam0 = lame_from_young(E, nu)
    mu = float(mu0) * rng.uniform(1.0 - rel, 1.0 + rel, size=n_tets)
    lam = float(lam0) * rng.uniform(1.0 - rel, 1.0 + rel, size=n_tets)
    return mu, lam


def random_displacement(X: np.ndarray, n: int, amp: float, seed: int,
                        smooth: float = 0.0) -> np.ndarray:
    """A seeded displacement field u (N_v, 3): i.i.d. uniform noise of
    amplitude ``amp * h`` plus, if ``smooth`` > 0, a smooth sinusoidal bend
    of amplitude ``smooth`` (absolute units)."""
    rng = np.random.Generator(np.random.PCG64(seed + 3000))
    h = 1.0 / n
    u = rng.uniform(-amp * h, amp * h, size=X.shape)
    if smooth > 0.0:
        a = rng.uniform(0.5, 1.5, size=3)
        u[:, 0] += smooth * np.sin(math.pi * a[0] * X[:, 2]) * X[:, 1]
        u[:, 1] += smooth * np.sin(math.pi * a[1] * X[:, 0]) * X[:, 2]
        u[:, 2] += smooth * np.cos(math.pi * a[2] * X[:, 1]) * X[:, 0]
    return u


def random_field(n_verts: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded (N_v, 3) vector field with entries uniform in [-scale, scale]."""
    rng = np.random.Generator(np.random.PCG64(seed + 4000))
    return rng.uniform(-scale, scale, size=(n_verts, 3))


def random_rotation(seed: int) -> np.ndarray:
    """A seeded random proper rotation matrix (QR of a Gaussian matrix)."""
    rng = np.random.Generator(np.random.PCG64(seed + 5000))
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def batched_sizes(count: int, n_lo: int, n_hi: int, seed: int) -> np.ndarray:
    """Mesh sides n = round(exp(U(ln n_lo, ln n_hi))) for a batch of meshes."""
    rng = np.random.Generator(np.random.PCG64(seed + 6000))
    return np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)


@dataclasses.dataclass
class MeshBatch:
    """Independent meshes concatenated into one vertex / tet relation pair.

    X, tets, pinned : as in TetMesh, for all meshes (tets offset per mesh)
    batch           : (N_v,) int32 mesh id of each vertex (non-decreasing)
    sides           : cube count per side of each mesh
    vert_off, tet_off : (count+1,) row offsets of each mesh
    """
    X: np.ndarray
    tets: np.ndarray
    pinned: np.ndarray
    batch: np.ndarray
    sides: np.ndarray
    vert_off: np.ndarray
    tet_off: np.ndarray

    def mesh(self, m):
        """(X, tets, pinned) of mesh m alone, keys rebased to its vertices."""
        a, b = self.vert_off[m], self.vert_off[m + 1]
        ta, tb = self.tet_off[m], self.tet_off[m + 1]
        return self.X[a:b], self.tets[ta:tb] - a, self.pinned[a:b]


def cube_grid_batch(sides, jitter: float = 0.01, seed: int = 0) -> MeshBatch:
    """Concatenate one cube grid per entry of ``sides`` (mesh m jittered
    with seed ``seed + m``)."""
    Xs, Ts, Ps, Bs = [], [], [], []
    voff, toff = [0], [0]
    for m, n in enumerate(sides):
        g = cube_grid(int(n), jitter=jitter, seed=seed + m)
        Ts.append(g.tets.astype(np.int64) + voff[-1])
        Xs.append(g.X)
        Ps.append(g.pinned)
        Bs.append(np.full(g.n_verts, m, dtype=np.int32))
        voff.append(voff[-1] + g.n_verts)
        toff.append(toff[-1] + g.n_tets)
    return MeshBatch(X=np.ascontiguousarray(np.concatenate(Xs)),
                     tets=np.ascontiguousarray(np.concatenate(Ts).astype(np.int32)),
                     pinned=np.concatenate(Ps), batch=np.concatenate(Bs), sides=np.asarray(sides),
                     vert_off=np.asarray(voff), tet_off=np.asarray(toff))



@dataclasses.dataclass
class HubMesh:
    """Tets (0, r_i, r_{i+1}, a_j) around a hub vertex (see ``hub_fan``).

    X    : (N_v, 3) float64 rest positions: hub at 0, ring vertices 1..K+1,
           apex vertices after them
    tets : (K * J, 4) int32 keys
    """
    X: np.ndarray
    tets: np.ndarray

    @property
    def n_verts(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def hub_fan(segments: int, apexes: int, seed: int) -> HubMesh:
    """A mesh of high vertex valence (non-conforming: tets overlap).

    The hub vertex sits at the origin and an open ring of ``segments + 1``
    vertices lies in the plane z = 0 at unit radius, at increasing angles (a
    span of at most 5.5 rad); ``apexes`` vertices lie above the plane (z in
    [0.5, 1.5], x and y in [-1, 1]).  Every pair (ring segment, apex) is one
    tet (hub, r_i, r_{i+1}, apex): the triangle (hub, r_i, r_{i+1}) turns
    counter-clockwise seen from above and the apex lies above it, so every
    tet is positively oriented by construction.  The hub is a corner of all
    segments * apexes tets, ring vertices of up to 2 * apexes, apexes of
    ``segments``.  With segments = 1 it is a fan of tets around one shared
    triangle."""
    rng = np.random.Generator(np.random.PCG64(seed + 7000))
    span = min(0.5 * segments, 5.5)
    ang = np.linspace(0.0, span, segments + 1)
    ring = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
    ap = np.stack([rng.uniform(-1, 1, apexes), rng.uniform(-1, 1, apexes), rng.uniform(0.5, 1.5, apexes)], axis=1)
    X = np.concatenate([np.zeros((1, 3)), ring, ap])
    i = np.repeat(np.arange(segments), apexes)
    j = np.tile(np.arange(apexes), segments)
    tets = np.stack([np.zeros_like(i), 1 + i, 2 + i, segments + 2 + j], axis=1)
    # tets listed apex-major in a seeded random order, so that tiles mix
    # segments and apexes
    tets = tets[rng.permutation(tets.shape[0])]
    return HubMesh(X=np.ascontiguousarray(X), tets=np.ascontiguousarray(tets.astype(np.int32)))

# Workload recipes.  They stand in for the paper's FEM workloads (Section 7.2,
# Vega: StVK, implicit backward Euler, Jacobi PCG on tet meshes; Section 7.3,
# FreeFem++: neo-Hookean, implicit CG), whose meshes are not available: cube
# grids of the listed sizes replace them.
WORKLOADS = {
    "stvk_fp64_n8": dict(n=8, model="stvk", E=1e5, nu=0.45, rho=1000.0, seed=1,
                         dt=1e-3, cg_iters=50, precision="f64"),
    "nh_mixed_n64": dict(n=64, model="nh", E_lo=1e4, E_hi=1e6, nu=0.4, rho=1000.0,
                         seed=2, dt=1e-3, steps=10, rtol=1e-8, precision="mixed"),
    "stvk_adjoint_n32": dict(n=32, model="stvk", E=1e5, nu=0.45, rel=0.2, rho=1000.0,
                             seed=3, dt=1e-3, steps=20, checkpoint=5),
    "nh_batched_256": dict(count=256, n_lo=4, n_hi=24, model="nh", E=1e5, nu=0.45,
                           rho=1000.0, seed=4, dt=1e-3),
    "stvk_permuted_n128": dict(n=128, model="stvk", E=1e5, nu=0.45, rho=1000.0,
                               seed=5, permute=True, precision="f32"),
}
