"""GPU parity of the element maps on meshes of high vertex valence (Section
6.2, field reductions into vertices that many elements share).

A fan of 700 tets around one triangle puts three vertices in every tet, and a
hub mesh puts one vertex in 384 tets and ring vertices in 48 each.  In the
tiled kernels such a vertex fills the most reduction units a tile allows, its
run of units crosses warp boundaries, and tiles close on the unit limit rather
than on tets or slots; the gather and atomic variants sum hundreds of entries
into one vertex.  Every reduction variant is compared with the FP64 oracle,
element by element over the whole field (1e-12 FP64, 1e-5 FP32).
"""
import numpy as np
import pytest
import torch

import meshgen
from oracle import fem
from _problems import rel_err

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
CASES = {"fan700": (1, 700), "hub384": (16, 24)}


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _problem(case, model, per_tet):
    m = meshgen.hub_fan(*CASES[case], seed=3)
    if per_tet:
        mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, seed=3)
    else:
        mu, lam = (float(a) for a in meshgen.lame_from_young(1e5, 0.45))
    u = meshgen.random_field(m.n_verts, seed=5, scale=0.02)
    w = meshgen.random_field(m.n_verts, seed=6)
    B, V = fem.rest_shape(m.X, m.tets)
    x = m.X + u
    mdl = fem.STVK if model == "stvk" else fem.NEOHOOKEAN
    want = {"f": fem.tet_forces(x, m.tets, B, V, mu, lam, mdl),
            "Kw": fem.tet_Kv(x, w, m.tets, B, V, mu, lam, mdl),
            "d": fem.tet_diagK(x, m.tets, B, V, mu, lam, mdl)}
    return m, mu, lam, u, w, want


def _run(m, mu, lam, u, w, model, prec, reduce, x4=False):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    per_tet = np.ndim(mu) > 0
    dt = torch.float64 if prec == "f64" else torch.float32
    with DeviceTetMesh(m.X, m.tets, mu if per_tet else None, lam if per_tet else None) as dm:
        dm.vertex_field("u", dt, value=u, x4=x4)
        dm.vertex_field("w", dt, value=w, x4=x4)
        out = {k: dm.vertex_field(k, dt, x4=x4) for k in ("f", "Kw", "d", "f2", "Kw2")}
        opts = abi.map_opts(abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN,
                            0.0 if per_tet else mu, 0.0 if per_tet else lam,
                            abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32, reduce, abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", opts)
        abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "Kw", opts)
        abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "d", opts)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f2", "Kw2", opts)
        abi.ebb_ctx_sync(dm.ctx)
        if x4:
            return {k: v[:, :3].double().cpu().numpy() for k, v in out.items()}
        return {k: v.double().cpu().numpy().T for k, v in out.items()}


def _check(got, want, tol):
    assert rel_err(got["f"], want["f"]) < tol
    assert rel_err(got["Kw"], want["Kw"]) < tol
    assert rel_err(got["d"], want["d"]) < tol
    assert rel_err(got["f2"], want["f"]) < tol
    assert rel_err(got["Kw2"], want["Kw"]) < tol


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("model", ["stvk", "nh"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("reduce", ["tiled", "ordered", "gather", "atomic", "coop"])
def test_high_valence_maps_match_oracle(case, model, prec, reduce):
    abi = _abi()
    red = {"tiled": abi.EBB_REDUCE_TILED, "ordered": abi.EBB_REDUCE_TILED_ORDERED,
           "gather": abi.EBB_REDUCE_GATHER, "atomic": abi.EBB_REDUCE_ATOMIC,
           "coop": abi.EBB_REDUCE_COOP}[reduce]
    m, mu, lam, u, w, want = _problem(case, model, per_tet=True)
    # the hub vertex really is shared by more tets than a tile holds
    assert np.bincount(m.tets.ravel()).max() > 128
    _check(_run(m, mu, lam, u, w, model, prec, red), want, TOL[prec])


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("reduce", ["tiled", "ordered", "gather", "atomic", "coop"])
def test_high_valence_interleaved_fields_uniform_material(case, reduce):
    """The same on 4-float vector elements (one 16-byte copy and one vector
    atomic per vertex in the tiled kernels), uniform material."""
    abi = _abi()
    red = {"tiled": abi.EBB_REDUCE_TILED, "ordered": abi.EBB_REDUCE_TILED_ORDERED,
           "gather": abi.EBB_REDUCE_GATHER, "atomic": abi.EBB_REDUCE_ATOMIC,
           "coop": abi.EBB_REDUCE_COOP}[reduce]
    m, mu, lam, u, w, want = _problem(case, "stvk", per_tet=False)
    _check(_run(m, mu, lam, u, w, "stvk", "f32", red, x4=True), want, TOL["f32"])
