"""The autotuner (ebb_relation_autotune): it times every candidate, leaves the
relation on the fastest tile size, and the maps and the implicit step still
match the oracle afterwards (through EBB_REDUCE_AUTO and explicit variants)."""
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


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_autotune_report_and_parity(prec):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(7, "nh", seed=21)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "nh")
    dt = torch.float32 if prec == "f32" else torch.float64
    p = abi.EBB_PREC_F32 if prec == "f32" else abi.EBB_PREC_F64
    with DeviceTetMesh(m.X, m.tets, mu, lam, colour=True) as dm:
        dm.vertex_field("u", dt, value=u)
        dm.vertex_field("w", dt, value=w)
        rep = abi.ebb_relation_autotune(dm.ctx, dm.tets, "u", "w", abi.map_opts(abi.EBB_NEOHOOKEAN, precision=p))
        cands = [(rep.cand[i].reduce, rep.cand[i].tile_tets, rep.cand[i].us) for i in range(rep.ncand)]
        # tiled at 3 tile sizes with row records (FP32: then staged interleaved at the best size), the
        # best tiled configuration with plane records, atomic, gather, cooperative, colour
        assert rep.ncand == (9 if prec == "f32" else 8)
        assert {c[0] for c in cands} == {abi.EBB_REDUCE_TILED, abi.EBB_REDUCE_ATOMIC, abi.EBB_REDUCE_GATHER,
                                         abi.EBB_REDUCE_COOP, abi.EBB_REDUCE_COLOR}
        tiled_c = [rep.cand[i] for i in range(rep.ncand) if rep.cand[i].reduce == abi.EBB_REDUCE_TILED]
        staged = [c.us for c in tiled_c if c.interleaved and not c.record_planes]
        assert len(staged) == (1 if prec == "f32" else 0)
        in_place = [c.us for c in tiled_c if not c.interleaved and not c.record_planes]
        assert len(in_place) == 3
        assert rep.interleaved == (1 if staged and staged[0] < min(in_place) else 0)
        planes = [c.us for c in tiled_c if c.record_planes]
        assert len(planes) == 1
        assert rep.record_planes == (1 if planes[0] < min(in_place + staged) else 0)
        assert {c[1] for c in cands if c[0] == abi.EBB_REDUCE_TILED} == {128, 96, 64}
        assert all(c[2] > 0 for c in cands)
        best = min(cands, key=lambda c: c[2])
        assert rep.reduce == best[0]
        tiled = [c for c in cands if c[0] == abi.EBB_REDUCE_TILED]
        assert rep.tile_tets == min(tiled, key=lambda c: c[2])[1]
        tol = 1e-12 if prec == "f64" else 1e-5
        out = {k: dm.vertex_field(k, dt) for k in ("f", "Kw", "d")}
        for red in (abi.EBB_REDUCE_AUTO, abi.EBB_REDUCE_TILED):
            o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=p, reduce=red, flags=abi.EBB_MAP_ZERO_OUT)
            abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "Kw", o)
            abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", o)
            abi.ebb_ctx_sync(dm.ctx)
            got = {k: v.double().cpu().numpy().T for k, v in out.items()}
            assert rel_err(got["f"], f) < tol
            assert rel_err(got["Kw"], Kw) < tol
            assert rel_err(got["d"], d) < tol


def test_step_after_retiling_matches_oracle():
    """A step captured before the autotuner re-cuts the tiles is re-captured
    afterwards (the layout generation is part of the graph key)."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m = meshgen.cube_grid(5, jitter=0.01, seed=3)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    uo, vo = np.zeros_like(m.X), np.zeros_like(m.X)
    for _ in range(3):
        uo, vo, _ = implicit.implicit_step(m.X, uo, vo, m.tets, B, V, mass, mu, lam, fem.STVK, 1e-3,
                                           np.array([0, 0, -9.81]), m.pinned, 400, 1e-14)
    with DeviceTetMesh(m.X, m.tets) as dm:
        uu = dm.vertex_field("u", torch.float64)
        vv = dm.vertex_field("v", torch.float64)
        dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dm.device))
        dm.vertex_field("pu", torch.float64, value=0.01 * meshgen.random_field(m.n_verts, seed=1))
        dm.vertex_field("pw", torch.float64, value=meshgen.random_field(m.n_verts, seed=2))
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, mu, lam, max_iters=400, rtol=1e-14)
        abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
        gen_tiles = abi.ebb_relation_autotune(dm.ctx, dm.tets, "pu", "pw", abi.map_opts(abi.EBB_STVK, mu, lam))
        assert gen_tiles.tile_tets in (128, 96, 64)
        # the candidates were timed on re-cut tiles (and the winner re-cut once
        # more unless it was the last one tried), so the blobs the first
        # step's graph captured are gone
        for _ in range(2):
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
        assert rel_err(vv.cpu().numpy().T, vo) < 1e-12
        assert rel_err(uu.cpu().numpy().T, uo) < 1e-12


@pytest.mark.parametrize("reorder", [False, True])
@pytest.mark.parametrize("tile_tets", [128, 64, 37])
def test_hand_tuning_staged_interleaved_maps(reorder, tile_tets):
    """Maps on a relation set by hand to stage FP32 operands vertex-interleaved
    (and to re-cut tiles, including a tile size that is not a warp multiple)
    still match the oracle, with and without reordered vertices."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, "nh", seed=31, permute=reorder)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, "nh")
    with DeviceTetMesh(m.X, m.tets, mu, lam, reorder_verts=reorder) as dm:
        dm.vertex_field("u", torch.float32, value=u)
        dm.vertex_field("w", torch.float32, value=w)
        out = {k: dm.vertex_field(k, torch.float32) for k in ("f", "Kw", "d", "f2")}
        out["f2"].fill_(2.0)
        abi.ebb_relation_set_tuning(dm.ctx, dm.tets, abi.EBB_NEOHOOKEAN, abi.EBB_PREC_F32, abi.EBB_REDUCE_TILED,
                                    tile_tets, 1)
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "Kw", o)
        abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", o)
        o.flags = 0
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f2", o)   # accumulates onto 2.0
        abi.ebb_ctx_sync(dm.ctx)
        got = {k: v.double().cpu().numpy().T for k, v in out.items()}
    assert rel_err(got["f"], f) < 1e-5
    assert rel_err(got["Kw"], Kw) < 1e-5
    assert rel_err(got["d"], d) < 1e-5
    assert rel_err(got["f2"] - 2.0, f) < 1e-5


def test_set_tuning_rejects_bad_values():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m = meshgen.cube_grid(2, seed=1)
    with DeviceTetMesh(m.X, m.tets) as dm:
        for args in ((abi.EBB_STVK, abi.EBB_PREC_F32, abi.EBB_REDUCE_TILED, 0, 0),
                     (abi.EBB_STVK, abi.EBB_PREC_F32, abi.EBB_REDUCE_TILED, 129, 0),
                     (abi.EBB_STVK, abi.EBB_PREC_F32, abi.EBB_REDUCE_AUTO, 128, 0),
                     (abi.EBB_STVK, 7, abi.EBB_REDUCE_TILED, 128, 0),
                     (abi.EBB_STVK, abi.EBB_PREC_F32, abi.EBB_REDUCE_TILED, 128, 4)):
            with pytest.raises(abi.EbbError) as ei:
                abi.ebb_relation_set_tuning(dm.ctx, dm.tets, *args)
            assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError) as ei:   # finalized without colouring
            abi.ebb_relation_set_tuning(dm.ctx, dm.tets, abi.EBB_STVK, abi.EBB_PREC_F32, abi.EBB_REDUCE_COLOR, 128, 0)
        assert ei.value.status == abi.EBB_ERR_STATE


@pytest.mark.parametrize("model", ["stvk", "nh"])
@pytest.mark.parametrize("per_tet", [True, False])
def test_record_planes_match_oracle(model, per_tet):
    """Tile blobs with per-tet data as field planes (SoA) instead of row
    records (AoSoA): every map in both precisions, with and without per-tet
    material, on tiles of 128 and 37 tets."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, model, seed=37, per_tet=per_tet)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, model)
    mdl = abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN
    mu0, lam0 = (0.0, 0.0) if per_tet else (mu, lam)
    with DeviceTetMesh(m.X, m.tets, mu if per_tet else None, lam if per_tet else None) as dm:
        for tile in (128, 37):
            for prec, dt, tol in ((abi.EBB_PREC_F64, torch.float64, 1e-12), (abi.EBB_PREC_F32, torch.float32, 1e-5)):
                abi.ebb_relation_set_tuning(dm.ctx, dm.tets, mdl, prec, abi.EBB_REDUCE_TILED, tile,
                                            abi.EBB_TUNE_RECORD_PLANES)
                assert abi.ebb_relation_info(dm.ctx, dm.tets).record_planes == 1
                dm.vertex_field("u", dt, value=u)
                dm.vertex_field("w", dt, value=w)
                out = {k: dm.vertex_field(k, dt) for k in ("f", "Kw", "d")}
                o = abi.map_opts(mdl, mu0, lam0, prec, abi.EBB_REDUCE_AUTO, abi.EBB_MAP_ZERO_OUT)
                abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "Kw", o)
                abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", o)
                abi.ebb_ctx_sync(dm.ctx)
                got = {k: v.double().cpu().numpy().T for k, v in out.items()}
                assert rel_err(got["f"], f) < tol and rel_err(got["Kw"], Kw) < tol and rel_err(got["d"], d) < tol
        # back to row records
        abi.ebb_relation_set_tuning(dm.ctx, dm.tets, mdl, abi.EBB_PREC_F32, abi.EBB_REDUCE_TILED, 128, 0)
        assert abi.ebb_relation_info(dm.ctx, dm.tets).record_planes == 0


def test_autotune_reports_both_record_layouts():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(8, "nh", seed=39)
    with DeviceTetMesh(m.X, m.tets, mu, lam) as dm:
        dm.vertex_field("u", torch.float64, value=u)
        dm.vertex_field("w", torch.float64, value=w)
        rep = abi.ebb_relation_autotune(dm.ctx, dm.tets, "u", "w",
                                        abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F64))
        tiled = [rep.cand[i] for i in range(rep.ncand) if rep.cand[i].reduce == abi.EBB_REDUCE_TILED]
        assert {c.record_planes for c in tiled} == {0, 1}
        assert rep.record_planes == abi.ebb_relation_info(dm.ctx, dm.tets).record_planes
