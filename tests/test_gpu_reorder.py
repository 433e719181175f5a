"""Vertex renumbering (EBB_FINALIZE_REORDER_VERTS) on meshes with scattered
vertex ids: maps and the implicit step must give the oracle's results in
the caller's vertex order."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import fem, implicit
from _problems import oracle_maps, problem, rel_err

pytestmark = pytest.mark.gpu


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("reduce", ["atomic", "colour", "tiled", "gather", "ordered"])
def test_reordered_maps_match_oracle(prec, reduce):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, "nh", seed=17, permute=True)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "nh")
    dt = torch.float64 if prec == "f64" else torch.float32
    red = {"atomic": abi.EBB_REDUCE_ATOMIC, "colour": abi.EBB_REDUCE_COLOR, "tiled": abi.EBB_REDUCE_TILED,
           "gather": abi.EBB_REDUCE_GATHER, "ordered": abi.EBB_REDUCE_TILED_ORDERED}[reduce]
    with DeviceTetMesh(m.X, m.tets, mu, lam, colour=True, reorder_verts=True) as dm:
        dm.vertex_field("u", dt, value=u)
        dm.vertex_field("w", dt, value=w)
        out = {k: dm.vertex_field(k, dt) for k in ("f", "Kw", "d", "f2", "Kw2")}
        out["f2"].fill_(1.0)     # maps accumulate into what is there
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32,
                         reduce=red, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", o)
        abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "Kw", o)
        abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", o)
        o.flags = 0
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f2", "Kw2", o)
        abi.ebb_ctx_sync(dm.ctx)
        got = {k: v.double().cpu().numpy().T for k, v in out.items()}
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel_err(got["f"], f) < tol
    assert rel_err(got["Kw"], Kw) < tol
    assert rel_err(got["d"], d) < tol
    assert rel_err(got["f2"] - 1.0, f) < tol
    assert rel_err(got["Kw2"], Kw) < tol


def test_reordered_step_matches_oracle():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m = meshgen.cube_grid(6, jitter=0.01, seed=3, permute=True)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=1)
    v0[m.pinned] = 0
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    uo, vo, u_ = np.zeros_like(m.X), v0.copy(), None
    for _ in range(2):
        uo, vo, _ = implicit.implicit_step(m.X, uo, vo, m.tets, B, V, mass, mu, lam, fem.STVK, 1e-3,
                                           np.array([0, 0, -9.81]), m.pinned, 400, 1e-14)
    for prec, tol in ((abi.EBB_PREC_F64, 1e-12), (abi.EBB_PREC_F32, 1e-5)):
        with DeviceTetMesh(m.X, m.tets, reorder_verts=True) as dm:
            uu = dm.vertex_field("u", torch.float64)
            vv = dm.vertex_field("v", torch.float64, value=v0)
            dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.int32)).to(dm.device))
            prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, mu, lam, precision=prec, max_iters=400,
                                  rtol=1e-14 if prec == abi.EBB_PREC_F64 else 1e-8)
            for _ in range(2):
                abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
            assert rel_err(vv.cpu().numpy().T, vo) < tol
            assert rel_err(uu.cpu().numpy().T, uo) < tol


def test_reordered_relation_refuses_batched_and_vjp():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    b = meshgen.cube_grid_batch([2, 2], seed=1)
    with pytest.raises(abi.EbbError) as ei:
        DeviceTetMesh(b.X, b.tets, batch=b.batch, reorder_verts=True)
    assert ei.value.status == abi.EBB_ERR_ARG
    m = meshgen.cube_grid(2, permute=True, seed=2)
    with DeviceTetMesh(m.X, m.tets, reorder_verts=True) as dm:
        for name in ("u", "v", "gu", "gv"):
            dm.vertex_field(name, torch.float64)
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1e4, 1e4, precision=abi.EBB_PREC_F64)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step_vjp(dm.ctx, dm.tets, "u", "v", None, "gu", "gv", None, None, prm)
        assert ei.value.status == abi.EBB_ERR_STATE


# ---- EBB_FINALIZE_RENUMBER_VERTS: the relation's own row order -------------

@pytest.mark.parametrize("prec", ["f64", "f32", "x4"])
@pytest.mark.parametrize("reduce", ["atomic", "tiled", "gather", "ordered"])
def test_renumbered_maps_match_oracle(prec, reduce):
    """Vertex fields held in the relation's row order (after renumbering):
    the maps' results, put back in the caller's order, are the oracle's."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, "nh", seed=19, permute=True)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "nh")
    x4 = prec == "x4"
    dt = torch.float64 if prec == "f64" else torch.float32
    red = {"atomic": abi.EBB_REDUCE_ATOMIC, "tiled": abi.EBB_REDUCE_TILED, "gather": abi.EBB_REDUCE_GATHER,
           "ordered": abi.EBB_REDUCE_TILED_ORDERED}[reduce]
    with DeviceTetMesh(m.X, m.tets, mu, lam, renumber_verts=True) as dm:
        order = dm.order
        assert np.array_equal(np.sort(order), np.arange(m.n_verts)) and not np.array_equal(order, np.arange(m.n_verts))
        info = abi.ebb_relation_info(dm.ctx, dm.tets)
        assert info.reordered == 2
        dm.vertex_field("u", dt, value=u, x4=x4)
        dm.vertex_field("w", dt, value=w, x4=x4)
        out = {k: dm.vertex_field(k, dt, x4=x4) for k in ("f", "Kw", "d", "f2", "Kw2")}
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32,
                         reduce=red, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", o)
        abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "Kw", o)
        abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", o)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f2", "Kw2", o)
        abi.ebb_ctx_sync(dm.ctx)
        got = {k: dm.caller((v[:, :3] if x4 else v.T).double().cpu().numpy()) for k, v in out.items()}
    tol = 1e-12 if prec == "f64" else 1e-5
    for k, want in (("f", f), ("Kw", Kw), ("d", d), ("f2", f), ("Kw2", Kw)):
        assert rel_err(got[k], want) < tol, k


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_renumbered_step_matches_oracle(prec):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m = meshgen.cube_grid(6, jitter=0.01, seed=23, permute=True)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=3)
    v0[m.pinned] = 0
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    uo, vo = np.zeros_like(m.X), v0.copy()
    rtol = 1e-14 if prec == "f64" else 1e-8
    for _ in range(2):
        uo, vo, _ = implicit.implicit_step(m.X, uo, vo, m.tets, B, V, mass, mu, lam, fem.STVK, 1e-3,
                                           np.array([0, 0, -9.81]), m.pinned, 400, 1e-14)
    with DeviceTetMesh(m.X, m.tets, renumber_verts=True) as dm:
        uu = dm.vertex_field("u", torch.float64)
        vv = dm.vertex_field("v", torch.float64, value=v0)
        dm.bind("pinned", torch.from_numpy(dm.rows(m.pinned).astype(np.uint8)).to(dm.device))
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, mu, lam,
                              precision=abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32, max_iters=400,
                              rtol=rtol)
        for _ in range(2):
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
        tol = 1e-12 if prec == "f64" else 1e-5
        assert rel_err(dm.caller(vv.cpu().numpy().T), vo) < tol
        assert rel_err(dm.caller(uu.cpu().numpy().T), uo) < tol


def test_renumber_flag_refusals_and_identity_order():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m = meshgen.cube_grid(2, permute=True, seed=2)
    with pytest.raises(abi.EbbError) as ei:          # the two vertex orders exclude each other
        DeviceTetMesh(m.X, m.tets, reorder_verts=True, renumber_verts=True)
    assert ei.value.status == abi.EBB_ERR_ARG
    b = meshgen.cube_grid_batch([2, 2], seed=1)
    with pytest.raises(abi.EbbError) as ei:
        DeviceTetMesh(b.X, b.tets, batch=b.batch, renumber_verts=True)
    assert ei.value.status == abi.EBB_ERR_ARG
    for kw in ({}, {"reorder_verts": True}):        # fields keep the caller's order
        with DeviceTetMesh(m.X, m.tets, **kw) as dm:
            assert np.array_equal(dm.order, np.arange(m.n_verts))
            with pytest.raises(abi.EbbError) as ei:
                abi.ebb_relation_vertex_order(dm.ctx, dm.tets, m.n_verts - 1)
            assert ei.value.status == abi.EBB_ERR_ARG
