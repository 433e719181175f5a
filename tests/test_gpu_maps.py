"""GPU parity of the element maps against the FP64 oracle, through the C ABI.

Tolerances (relative max-norm over the whole vertex field): 1e-12 for the
FP64 path, 1e-5 for the FP32 path.  Meshes span several 128-tet blocks with a
ragged tail (n = 6: 1080 tets; n = 7: 1715 tets).
"""
import numpy as np
import pytest
import torch

from _problems import oracle_maps, problem, rel_err, submesh_for_vertices

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _mesh(m, mu, lam, colour=True):
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    return DeviceTetMesh(m.X, m.tets, mu if np.ndim(mu) else None, lam if np.ndim(lam) else None, colour=colour)


def _run_maps(dm, u, w, model, prec, reduce, mu, lam):
    abi = _abi()
    dt = torch.float64 if prec == "f64" else torch.float32
    dm.vertex_field("u", dt, value=u)
    dm.vertex_field("w", dt, value=w)
    out = {k: dm.vertex_field(k, dt) for k in ("f", "Kw", "d", "f2", "Kw2")}
    mdl = abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN
    mu0 = 0.0 if np.ndim(mu) else mu
    lam0 = 0.0 if np.ndim(lam) else lam
    opts = abi.map_opts(mdl, mu0, lam0, abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32,
                        reduce, abi.EBB_MAP_ZERO_OUT)
    abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", opts)
    abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "Kw", opts)
    abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", opts)
    abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f2", "Kw2", opts)
    abi.ebb_ctx_sync(dm.ctx)
    return {k: v.double().cpu().numpy().T for k, v in out.items()}


@pytest.mark.parametrize("model", ["stvk", "nh"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("reduce", ["atomic", "colour", "tiled", "gather", "ordered", "coop"])
@pytest.mark.parametrize("per_tet", [True, False])
def test_maps_match_oracle(model, prec, reduce, per_tet):
    abi = _abi()
    m, mu, lam, u, w = problem(6 if per_tet else 7, model, seed=13, per_tet=per_tet)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, model)
    red = {"atomic": abi.EBB_REDUCE_ATOMIC, "colour": abi.EBB_REDUCE_COLOR, "tiled": abi.EBB_REDUCE_TILED,
           "gather": abi.EBB_REDUCE_GATHER, "ordered": abi.EBB_REDUCE_TILED_ORDERED,
           "coop": abi.EBB_REDUCE_COOP}[reduce]
    with _mesh(m, mu, lam) as dm:
        got = _run_maps(dm, u, w, model, prec, red, mu, lam)
    tol = TOL[prec]
    assert rel_err(got["f"], f) < tol
    assert rel_err(got["Kw"], Kw) < tol
    assert rel_err(got["d"], d) < tol
    assert rel_err(got["f2"], f) < tol
    assert rel_err(got["Kw2"], Kw) < tol


def test_small_strain_fp32_relative_accuracy():
    """FP32 forces stay within 1e-5 of FP64 at strains of 1e-4 (the G = F - I
    formulation avoids cancellation)."""
    abi = _abi()
    for model in ("stvk", "nh"):
        m, mu, lam, u, w = problem(6, model, seed=5, amp=1e-4, smooth=1e-5)
        f, Kw, _ = oracle_maps(m, mu, lam, u, w, model)
        with _mesh(m, mu, lam, colour=False) as dm:
            for red in (abi.EBB_REDUCE_ATOMIC, abi.EBB_REDUCE_TILED):
                got = _run_maps(dm, u, w, model, "f32", red, mu, lam)
                assert rel_err(got["f"], f) < 1e-5
                assert rel_err(got["Kw"], Kw) < 1e-5


@pytest.mark.parametrize("reduce", ["colour", "gather", "ordered"])
def test_atomic_free_variants_are_bitwise_deterministic(reduce):
    abi = _abi()
    red = {"colour": abi.EBB_REDUCE_COLOR, "gather": abi.EBB_REDUCE_GATHER,
           "ordered": abi.EBB_REDUCE_TILED_ORDERED}[reduce]
    m, mu, lam, u, w = problem(7, "nh", seed=3)
    with _mesh(m, mu, lam) as dm:
        a = _run_maps(dm, u, w, "nh", "f32", red, mu, lam)
        b = _run_maps(dm, u, w, "nh", "f32", red, mu, lam)
    for k in ("f", "Kw", "d", "f2", "Kw2"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gather_needs_no_colouring(prec):
    """The gather variant on a relation finalized without a colouring (its
    order comes from the vertex index alone): it matches the oracle and
    repeats bit for bit, in both precisions."""
    abi = _abi()
    m, mu, lam, u, w = problem(3, "stvk", seed=17)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "stvk")
    with _mesh(m, mu, lam, colour=False) as dm:
        got = _run_maps(dm, u, w, "stvk", prec, abi.EBB_REDUCE_GATHER, mu, lam)
        again = _run_maps(dm, u, w, "stvk", prec, abi.EBB_REDUCE_GATHER, mu, lam)
    tol = TOL[prec]
    assert rel_err(got["f"], f) < tol and rel_err(got["Kw"], Kw) < tol and rel_err(got["d"], d) < tol
    for k in got:
        assert np.array_equal(got[k], again[k])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ordered_tiles_repeat_at_every_tile_size(prec):
    """The ordered tiled variant without a colouring: at tiles of 128, 61 and
    1 tet (the partial index is rebuilt with the tiles) it matches the oracle
    and repeats bit for bit."""
    abi = _abi()
    m, mu, lam, u, w = problem(4, "nh", seed=19)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "nh")
    tol = TOL[prec]
    p = abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32
    with _mesh(m, mu, lam, colour=False) as dm:
        for cap in (128, 61, 1):
            abi.ebb_relation_set_tuning(dm.ctx, dm.tets, abi.EBB_NEOHOOKEAN, p, abi.EBB_REDUCE_TILED, cap, 0)
            got = _run_maps(dm, u, w, "nh", prec, abi.EBB_REDUCE_TILED_ORDERED, mu, lam)
            again = _run_maps(dm, u, w, "nh", prec, abi.EBB_REDUCE_TILED_ORDERED, mu, lam)
            assert rel_err(got["f"], f) < tol and rel_err(got["Kw"], Kw) < tol and rel_err(got["d"], d) < tol
            for k in got:
                assert np.array_equal(got[k], again[k])


def test_permuted_ids_match_oracle():
    abi = _abi()
    m, mu, lam, u, w = problem(5, "stvk", seed=8, permute=True)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "stvk")
    with _mesh(m, mu, lam) as dm:
        for red in (abi.EBB_REDUCE_ATOMIC, abi.EBB_REDUCE_TILED, abi.EBB_REDUCE_COLOR, abi.EBB_REDUCE_GATHER,
                    abi.EBB_REDUCE_TILED_ORDERED):
            got = _run_maps(dm, u, w, "stvk", "f32", red, mu, lam)
            assert rel_err(got["f"], f) < 1e-5 and rel_err(got["Kw"], Kw) < 1e-5


@pytest.mark.parametrize("n,model,prec,reorder,reduce", [(64, "nh", "f32", False, "tiled"),
                                                         (64, "nh", "f32", False, "gather"),
                                                         (64, "nh", "f32", False, "ordered"),
                                                         (128, "stvk", "f32", False, "tiled"),
                                                         (128, "stvk", "f32", True, "tiled"),
                                                         (32, "stvk", "f64", False, "tiled")])
def test_full_size_sampled_vertices(n, model, prec, reorder, reduce):
    """At the benchmark sizes the oracle checks sampled vertices: each is
    recomputed exactly from its incident tets only."""
    abi = _abi()
    from oracle import fem
    m, mu, lam, u, w = problem(n, model, seed=2, amp=0.05, smooth=0.01, permute=(n == 128))
    rng = np.random.default_rng(0)
    sample = rng.choice(m.n_verts, size=64, replace=False)
    sub = submesh_for_vertices(m.tets, sample)
    sel = np.isin(m.tets, sample).any(axis=1)
    mu_s = mu[sel] if np.ndim(mu) else mu
    lam_s = lam[sel] if np.ndim(lam) else lam
    B, V = fem.rest_shape(m.X, sub)
    mdl = fem.STVK if model == "stvk" else fem.NEOHOOKEAN
    x = m.X + u
    f = fem.tet_forces(x, sub, B, V, mu_s, lam_s, mdl)[sample]
    Kw = fem.tet_Kv(x, w, sub, B, V, mu_s, lam_s, mdl)[sample]
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    with DeviceTetMesh(m.X, m.tets, mu if np.ndim(mu) else None, lam if np.ndim(lam) else None,
                       reorder_verts=reorder) as dm:
        red = {"tiled": abi.EBB_REDUCE_TILED, "gather": abi.EBB_REDUCE_GATHER,
               "ordered": abi.EBB_REDUCE_TILED_ORDERED}[reduce]
        got = _run_maps(dm, u, w, model, prec, red, mu, lam)
    tol = TOL[prec]
    assert rel_err(got["f"][sample], f) < tol
    assert rel_err(got["Kw"][sample], Kw) < tol
    assert rel_err(got["f2"][sample], f) < tol
    assert rel_err(got["Kw2"][sample], Kw) < tol
