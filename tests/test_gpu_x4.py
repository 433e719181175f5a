"""EBB_F32X4 vertex fields (3-vectors stored element by element as four
floats): every map and reduction variant against the FP64 oracle at the FP32
tolerance, with and without reordered vertices; maps accumulate; a map's
fields must share one layout; a misaligned pointer is refused at bind."""
import numpy as np
import pytest
import torch

from _problems import oracle_maps, problem, rel_err

pytestmark = pytest.mark.gpu


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _got(t):
    return t[:, :3].double().cpu().numpy()


@pytest.mark.parametrize("model", ["stvk", "nh"])
@pytest.mark.parametrize("reduce", ["tiled", "atomic", "colour", "gather", "ordered", "coop"])
@pytest.mark.parametrize("reorder", [False, True])
def test_x4_maps_match_oracle(model, reduce, reorder):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, model, seed=41, permute=reorder)
    f, Kw, d = oracle_maps(m, mu, lam, u, w, model)
    red = {"atomic": abi.EBB_REDUCE_ATOMIC, "colour": abi.EBB_REDUCE_COLOR, "tiled": abi.EBB_REDUCE_TILED,
           "gather": abi.EBB_REDUCE_GATHER, "ordered": abi.EBB_REDUCE_TILED_ORDERED,
           "coop": abi.EBB_REDUCE_COOP}[reduce]
    mdl = abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN
    with DeviceTetMesh(m.X, m.tets, mu, lam, colour=True, reorder_verts=reorder) as dm:
        dm.vertex_field("u", value=u, x4=True)
        dm.vertex_field("w", value=w, x4=True)
        out = {k: dm.vertex_field(k, x4=True) for k in ("f", "Kw", "d", "f2", "Kw2", "k3")}
        out["f2"][:, :3] = 1.0
        torch.cuda.synchronize()
        o = abi.map_opts(mdl, precision=abi.EBB_PREC_F32, reduce=red, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", o)
        abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "Kw", o)
        abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", o)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "k3", "Kw2", o)   # k3: force, zeroed
        o.flags = 0
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f2", o)                # accumulates onto 1.0
        abi.ebb_ctx_sync(dm.ctx)
        got = {k: _got(v) for k, v in out.items()}
    assert rel_err(got["f"], f) < 1e-5
    assert rel_err(got["Kw"], Kw) < 1e-5
    assert rel_err(got["d"], d) < 1e-5
    assert rel_err(got["k3"], f) < 1e-5
    assert rel_err(got["Kw2"], Kw) < 1e-5
    assert rel_err(got["f2"] - 1.0, f) < 1e-5


def test_x4_layout_rules_and_autotune():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(5, "nh", seed=43)
    f, Kw, _ = oracle_maps(m, mu, lam, u, w, "nh")
    with DeviceTetMesh(m.X, m.tets, mu, lam) as dm:
        dm.vertex_field("u", value=u, x4=True)
        dm.vertex_field("w", value=w, x4=True)
        dm.vertex_field("wp", torch.float32, value=w)            # planes
        tf = dm.vertex_field("f", x4=True)
        tk = dm.vertex_field("k", x4=True)
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, flags=abi.EBB_MAP_ZERO_OUT)
        with pytest.raises(abi.EbbError) as ei:                  # mixed layouts
            abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "wp", "k", o)
        assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError) as ei:                  # same field read and reduced into
            abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "w", o)
        assert ei.value.status == abi.EBB_ERR_PHASE
        with pytest.raises(abi.EbbError) as ei:                  # F64 maps need F64 planes
            abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f",
                                   abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F64))
        assert ei.value.status == abi.EBB_ERR_ARG
        rep = abi.ebb_relation_autotune(dm.ctx, dm.tets, "u", "w", abi.map_opts(abi.EBB_NEOHOOKEAN,
                                                                               precision=abi.EBB_PREC_F32))
        # tiled x3 (fields already interleaved), tiled with plane records, atomic, gather, cooperative
        assert rep.interleaved == 1 and rep.ncand == 7
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o)
        abi.ebb_ctx_sync(dm.ctx)
        assert rel_err(_got(tf), f) < 1e-5
        assert rel_err(_got(tk), Kw) < 1e-5
        # a pointer off a 16-byte boundary is refused at bind
        raw = torch.zeros(4 * m.n_verts + 1, dtype=torch.float32, device=dm.device)
        bad = raw[1:].view(m.n_verts, 4)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_field_bind(dm.ctx, dm.verts, "bad", bad, x4=True)
        assert ei.value.status == abi.EBB_ERR_ARG
