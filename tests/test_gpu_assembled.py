"""Assembled stiffness on the edge relation (EBB_FINALIZE_EDGES): K(u)
assembled from the closed-form element blocks and applied by the block-sparse
product equals the oracle's matrix-free K w; K is symmetric; the product is
bitwise reproducible; the implicit step with EBB_STEP_ASSEMBLED matches the
oracle; the calls refuse what they do not support."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import fem, implicit
from _problems import oracle_maps, problem, rel_err

pytestmark = pytest.mark.gpu

G = (0.0, 0.0, -9.81)
TOL = {"f64": 1e-12, "f32": 1e-5}


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _mesh(m, mu, lam, **kw):
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    return DeviceTetMesh(m.X, m.tets, mu if np.ndim(mu) else None, lam if np.ndim(lam) else None, **kw)


def _spmv(dm, u, ws, model, prec, x4=False, mu=0.0, lam=0.0):
    """Assemble K(u) and return K w for every w in ws (host arrays, N x 3)."""
    abi = _abi()
    dt = torch.float64 if prec == "f64" else torch.float32
    dm.vertex_field("u", dt, value=u, x4=x4)
    o = abi.map_opts(abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN, mu, lam,
                     abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32, flags=abi.EBB_MAP_ZERO_OUT)
    abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u", o)
    out = []
    for i, w in enumerate(ws):
        dm.vertex_field(f"w{i}", dt, value=w, x4=x4)
        k = dm.vertex_field(f"k{i}", dt, x4=x4)
        abi.ebb_spmv_tet_K(dm.ctx, dm.tets, f"w{i}", f"k{i}", o)
        abi.ebb_ctx_sync(dm.ctx)
        out.append((k[:, :3] if x4 else k.T).double().cpu().numpy().copy())
    return out


@pytest.mark.parametrize("model", ["stvk", "nh"])
@pytest.mark.parametrize("prec,x4", [("f64", False), ("f32", False), ("f32", True)])
@pytest.mark.parametrize("reorder", [False, True])
def test_spmv_matches_oracle_Kv(model, prec, x4, reorder):
    m, mu, lam, u, w = problem(5, model, seed=61, permute=reorder)
    _, Kw, _ = oracle_maps(m, mu, lam, u, w, model)
    with _mesh(m, mu, lam, edges=True, reorder_verts=reorder) as dm:
        (got,) = _spmv(dm, u, [w], model, prec, x4)
    assert rel_err(got, Kw) < TOL[prec]


@pytest.mark.parametrize("model", ["stvk", "nh"])
def test_assembled_K_is_symmetric_and_reproducible(model):
    m, mu, lam, u, _ = problem(4, model, seed=62)
    w1 = meshgen.random_field(m.n_verts, seed=1)
    w2 = meshgen.random_field(m.n_verts, seed=2)
    with _mesh(m, mu, lam, edges=True) as dm:
        k1, k2, k1b = _spmv(dm, u, [w1, w2, w1], model, "f64")
    a, b = float(np.sum(w2 * k1)), float(np.sum(w1 * k2))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert np.array_equal(k1, k1b)


def test_assembled_diagonal_matches_diag_map():
    """Unit probes e_(v,c) on the assembled K give its diagonal, which equals
    the oracle's diag(K) (the closed form the Jacobi preconditioner uses)."""
    m, mu, lam, u, w = problem(2, "nh", seed=63)
    _, _, d = oracle_maps(m, mu, lam, u, w, "nh")
    n = m.n_verts
    probes = []
    for v in range(n):
        for c in range(3):
            e = np.zeros((n, 3))
            e[v, c] = 1.0
            probes.append(e)
    with _mesh(m, mu, lam, edges=True) as dm:
        outs = _spmv(dm, u, probes, "nh", "f64")
    diag = np.array([[outs[3 * v + c][v, c] for c in range(3)] for v in range(n)])
    assert rel_err(diag, d) < 1e-12


def _steps(m, mu, lam, model, steps, prec, flags, reduce="tiled", max_iters=400, rtol=1e-12):
    abi = _abi()
    per_tet = np.ndim(mu) > 0
    with _mesh(m, mu, lam, edges=True) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64)
        dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dm.device))
        prm = abi.step_params(abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN, 1e-3, 1000.0,
                              0.0 if per_tet else mu, 0.0 if per_tet else lam, G,
                              abi.EBB_PREC_F64 if prec == "f64" else abi.EBB_PREC_F32,
                              {"tiled": abi.EBB_REDUCE_TILED, "gather": abi.EBB_REDUCE_GATHER}[reduce],
                              max_iters, rtol, flags=flags)
        reps = [abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm) for _ in range(steps)]
        return dm._tensors["u"].cpu().numpy().T.copy(), dm._tensors["v"].cpu().numpy().T.copy(), reps


def _oracle(m, mu, lam, model, steps, max_iters, rtol):
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    u, v = np.zeros_like(m.X), np.zeros_like(m.X)
    infos = []
    for _ in range(steps):
        u, v, info = implicit.implicit_step(m.X, u, v, m.tets, B, V, mass, mu, lam,
                                            fem.STVK if model == "stvk" else fem.NEOHOOKEAN, 1e-3, np.array(G),
                                            m.pinned, max_iters, rtol)
        infos.append(info)
    return u, v, infos


def test_assembled_fp64_step_matches_oracle():
    abi = _abi()
    m = meshgen.cube_grid(6, jitter=0.01, seed=64)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    uo, vo, io = _oracle(m, mu, lam, "stvk", 2, 400, 1e-14)
    ug, vg, rg = _steps(m, mu, lam, "stvk", 2, "f64", abi.EBB_STEP_ASSEMBLED, rtol=1e-14)
    assert rel_err(vg, vo) < 1e-12 and rel_err(ug, uo) < 1e-12
    assert all(abs(a.iters - b["iters"]) <= 2 for a, b in zip(rg, io))


@pytest.mark.parametrize("reduce", ["tiled", "gather"])
def test_assembled_mixed_step_matches_oracle(reduce):
    abi = _abi()
    m = meshgen.cube_grid(6, jitter=0.01, seed=65)
    mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, 65)
    uo, vo, _ = _oracle(m, mu, lam, "nh", 3, 1000, 1e-8)
    ug, vg, rg = _steps(m, mu, lam, "nh", 3, "f32", abi.EBB_STEP_ASSEMBLED, reduce, 1000, 1e-8)
    assert all(r.rel_residual <= 1e-8 for r in rg)
    assert rel_err(vg, vo) < 1e-5 and rel_err(ug, uo) < 1e-5


def test_assembled_calls_refuse_what_they_do_not_support():
    abi = _abi()
    m, mu, lam, u, w = problem(2, "stvk", seed=66)
    o = abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F64)
    with _mesh(m, mu, lam) as dm:                      # no edge relation
        dm.vertex_field("u", torch.float64, value=u)
        dm.vertex_field("w", torch.float64, value=w)
        dm.vertex_field("k", torch.float64)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u", o)
        assert ei.value.status == abi.EBB_ERR_STATE
        dm.vertex_field("v", torch.float64)
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, flags=abi.EBB_STEP_ASSEMBLED)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", None, prm)
        assert ei.value.status == abi.EBB_ERR_STATE
    with _mesh(m, mu, lam, edges=True) as dm:
        dm.vertex_field("u", torch.float64, value=u)
        dm.vertex_field("w", torch.float64, value=w)
        dm.vertex_field("k", torch.float64)
        with pytest.raises(abi.EbbError) as ei:        # product before any assembly
            abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w", "k", o)
        assert ei.value.status == abi.EBB_ERR_STATE
        abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u", o)
        with pytest.raises(abi.EbbError) as ei:        # FP32 not assembled yet
            abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w", "k", abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F32))
        assert ei.value.status == abi.EBB_ERR_STATE
        with pytest.raises(abi.EbbError) as ei:        # phase rule
            abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w", "w", o)
        assert ei.value.status == abi.EBB_ERR_PHASE
        dm.vertex_field("v", torch.float64)
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, flags=4)
        with pytest.raises(abi.EbbError) as ei:        # unknown flag
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", None, prm)
        assert ei.value.status == abi.EBB_ERR_ARG
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, flags=abi.EBB_STEP_ASSEMBLED)
        dm.vertex_field("gu", torch.float64)
        dm.vertex_field("gv", torch.float64)
        with pytest.raises(abi.EbbError) as ei:        # the VJP takes no flags
            abi.ebb_cg_implicit_step_vjp(dm.ctx, dm.tets, "u", "v", None, "gu", "gv", None, None, prm)
        assert ei.value.status == abi.EBB_ERR_ARG
