"""Seeded test problems shared by the GPU parity tests (inputs from meshgen,
expected values from the FP64 oracle only)."""
import numpy as np

import meshgen
from oracle import fem

MODELS = {"stvk": fem.STVK, "nh": fem.NEOHOOKEAN}


def problem(n, model="stvk", seed=11, jitter=0.05, amp=0.2, smooth=0.05, per_tet=True, permute=False):
    m = meshgen.cube_grid(n, jitter=jitter, seed=seed, permute=permute)
    if per_tet:
        mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, seed)
    else:
        mu, lam = (float(a) for a in meshgen.lame_from_young(1e5, 0.45))
    u = meshgen.random_displacement(m.X, n, amp=amp, seed=seed, smooth=smooth)
    w = meshgen.random_field(m.n_verts, seed=seed + 1)
    return m, mu, lam, u, w


def oracle_maps(m, mu, lam, u, w, model):
    B, V = fem.rest_shape(m.X, m.tets)
    x = m.X + u
    mdl = MODELS[model]
    f = fem.tet_forces(x, m.tets, B, V, mu, lam, mdl)
    Kw = fem.tet_Kv(x, w, m.tets, B, V, mu, lam, mdl)
    d = fem.tet_diagK(x, m.tets, B, V, mu, lam, mdl)
    return f, Kw, d


def rel_err(a, b):
    """max-norm relative error ||a - b||_inf / ||b||_inf over the whole field."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a)))


def submesh_for_vertices(tets, sample):
    """Tets incident to the sampled vertices: reducing over these alone gives
    the exact field value at every sampled vertex."""
    mask = np.isin(tets, sample).any(axis=1)
    return tets[mask]
