"""Error behaviour of the C ABI on a GPU: bad keys, inverted elements, the
phase rule, dtype and ordering errors, and empty relations.  Every failure is
made on the host side or detected by the kernels' own checks; nothing here
faults the device."""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _mesh(tets=None, X=None, **kw):
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m = meshgen.cube_grid(2, jitter=0.02, seed=1)
    return m, DeviceTetMesh(m.X if X is None else X, m.tets if tets is None else tets, **kw)


@pytest.mark.parametrize("bad", [-1, 27, 1 << 20])
def test_out_of_range_key_rejected_at_finalize(bad):
    abi = _abi()
    m = meshgen.cube_grid(2)
    tets = m.tets.copy()
    tets[17, 2] = bad
    with pytest.raises(abi.EbbError) as ei:
        _mesh(tets=tets)
    assert ei.value.status == abi.EBB_ERR_KEY
    assert "row 17" in str(ei.value)


def test_repeated_vertex_rejected():
    abi = _abi()
    m = meshgen.cube_grid(2)
    tets = m.tets.copy()
    tets[3, 1] = tets[3, 0]
    with pytest.raises(abi.EbbError) as ei:
        _mesh(tets=tets)
    assert ei.value.status == abi.EBB_ERR_KEY


def test_inverted_rest_tet_rejected():
    abi = _abi()
    m = meshgen.cube_grid(2)
    tets = m.tets.copy()
    tets[5, [2, 3]] = tets[5, [3, 2]]
    with pytest.raises(abi.EbbError) as ei:
        _mesh(tets=tets)
    assert ei.value.status == abi.EBB_ERR_INVERTED


def test_phase_rule():
    abi = _abi()
    m, dm = _mesh()
    with dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("w", torch.float64)
        dm.vertex_field("f", torch.float64)
        opts = abi.map_opts(abi.EBB_STVK, 1e4, 1e4)
        for call in (lambda: abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "u", opts),
                     lambda: abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "w", opts),
                     lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "f", opts)):
            with pytest.raises(abi.EbbError) as ei:
                call()
            assert ei.value.status == abi.EBB_ERR_PHASE
        # an alias of the same storage under another name is caught too
        dm.bind("u_alias", dm._tensors["u"])
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "u_alias", opts)
        assert ei.value.status == abi.EBB_ERR_PHASE


def test_dtype_and_name_errors():
    abi = _abi()
    m, dm = _mesh()
    with dm:
        dm.vertex_field("u32", torch.float32)
        dm.vertex_field("f64", torch.float64)
        opts = abi.map_opts(abi.EBB_STVK, 1e4, 1e4, abi.EBB_PREC_F64)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u32", "f64", opts)
        assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_forces(dm.ctx, dm.tets, "nope", "f64", opts)
        assert ei.value.status == abi.EBB_ERR_ARG
        # colour variant needs a coloured finalize
        dm.vertex_field("u", torch.float64)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f64",
                                   abi.map_opts(abi.EBB_STVK, 1e4, 1e4, reduce=abi.EBB_REDUCE_COLOR))
        assert ei.value.status == abi.EBB_ERR_STATE


def test_map_before_finalize_is_state_error():
    abi = _abi()
    ctx = abi.ebb_ctx_create(0, None)
    try:
        verts = abi.ebb_relation_create(ctx, "verts", 4)
        tets = abi.ebb_relation_create(ctx, "tets", 1)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_forces(ctx, tets, "u", "f", abi.map_opts(abi.EBB_STVK, 1.0, 1.0))
        assert ei.value.status == abi.EBB_ERR_STATE
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_relation_create(ctx, "bad", -1)
        assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError):
            abi.ebb_relation_finalize(ctx, tets)      # no key-field bound
    finally:
        abi.ebb_ctx_destroy(ctx)


def test_nh_inverted_deformation_raises_at_sync():
    abi = _abi()
    m, dm = _mesh()
    with dm:
        u = -2.0 * m.X                               # x = -X: every tet inverted
        dm.vertex_field("u", torch.float64, value=u)
        dm.vertex_field("f", torch.float64)
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", abi.map_opts(abi.EBB_NEOHOOKEAN, 1e4, 1e4))
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_ctx_sync(dm.ctx)
        assert ei.value.status == abi.EBB_ERR_INVERTED
        abi.ebb_ctx_sync(dm.ctx)                     # the status word was cleared


def test_empty_relations():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    X = np.zeros((0, 3))
    tets = np.zeros((0, 4), np.int32)
    with DeviceTetMesh(X, tets, colour=True) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("f", torch.float64)
        dm.vertex_field("v", torch.float64)
        abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", abi.map_opts(abi.EBB_STVK, 1.0, 1.0))
        rep = abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", None,
                                       abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1.0, 1.0))
        assert rep.iters == 0
    # vertices without tets: the step is free fall
    X = np.random.default_rng(0).normal(size=(5, 3))
    with DeviceTetMesh(X, tets) as dm:
        dm.vertex_field("u", torch.float64)
        v = dm.vertex_field("v", torch.float64)
        rep = abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", None,
                                       abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1.0, 1.0))
        # lumped mass is zero without tets: A = 0 on those rows -> breakdown or no-op, never a hang
        assert rep.iters <= 1


def test_empty_relations_gather_assembled_springs():
    """The gather and ordered tiled variants, the assembled K and the
    springs on relations without tets (and without vertices): no error, zero
    products, free flight of the vertices."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    tets = np.zeros((0, 4), np.int32)
    o = abi.map_opts(abi.EBB_STVK, 1.0, 1.0, reduce=abi.EBB_REDUCE_GATHER)
    for nv in (0, 5):
        X = np.random.default_rng(1).normal(size=(nv, 3))
        with DeviceTetMesh(X, tets, edges=True) as dm:
            w = np.random.default_rng(2).normal(size=(nv, 3))
            dm.vertex_field("u", torch.float64)
            dm.vertex_field("w", torch.float64, value=w)
            f = dm.vertex_field("f", torch.float64)
            k = dm.vertex_field("k", torch.float64)
            abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o)
            abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k",
                                     abi.map_opts(abi.EBB_STVK, 1.0, 1.0, reduce=abi.EBB_REDUCE_TILED_ORDERED))
            abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u", o)
            abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w", "k", o)
            abi.ebb_ctx_sync(dm.ctx)
            assert not f.any() and not k.any()
            abi.ebb_springs_init(dm.ctx, dm.tets, "X")
            q = dm.vertex_field("q", torch.float64, value=X)
            qd = dm.vertex_field("qd", torch.float64, value=w)
            dm.vertex_field("mass", torch.float64, ncomp=1, value=np.ones(nv))
            e = abi.ebb_springs_run(dm.ctx, dm.tets, "q", "qd", "mass", 1.0, 0.01, 3, energy=True)
            assert np.allclose(q.cpu().numpy().T, X + 0.03 * w, rtol=0, atol=1e-14)
            assert abs(e - 0.5 * float(np.sum(w * w))) <= 1e-14 * max(1.0, e)


def test_single_tet_matches_hand_derived_forces():
    import json, os
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "single_tet_closed_form.json")))
    X = np.array(gold["X"], np.float64)
    for case in gold["cases"]:
        F = np.array(case["F"])
        u = X @ F.T - X
        with DeviceTetMesh(X, np.array([[0, 1, 2, 3]], np.int32)) as dm:
            dm.vertex_field("u", torch.float64, value=u)
            f = dm.vertex_field("f", torch.float64)
            mdl = abi.EBB_STVK if case["model"] == "stvk" else abi.EBB_NEOHOOKEAN
            abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", abi.map_opts(mdl, case["mu"], case["lam"]))
            abi.ebb_ctx_sync(dm.ctx)
            assert np.max(np.abs(f.cpu().numpy().T - np.array(case["f"]))) < 1e-14


def test_bounded_wait_times_out_and_context_survives():
    """Failure detection without a fault: the tiled map is told to skip one
    tile's bulk copy (EBB_MAP_TEST_DROP_TILE), so that CTA's bounded wait
    runs out; the next synchronising call reports EBB_ERR_TIMEOUT, and the
    same context then runs the map correctly."""
    abi = _abi()
    from _problems import oracle_maps, problem, rel_err
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, "stvk", seed=3)
    f, Kw, _ = oracle_maps(m, mu, lam, u, w, "stvk")
    with DeviceTetMesh(m.X, m.tets, mu, lam) as dm:
        dm.vertex_field("u", torch.float32, value=u)
        dm.vertex_field("w", torch.float32, value=w)
        tf = dm.vertex_field("f", torch.float32)
        tk = dm.vertex_field("k", torch.float32)
        o = abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED,
                         flags=abi.EBB_MAP_ZERO_OUT | abi.EBB_MAP_TEST_DROP_TILE)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_ctx_sync(dm.ctx)
        assert ei.value.status == abi.EBB_ERR_TIMEOUT
        abi.ebb_ctx_sync(dm.ctx)   # the status word was consumed
        o.flags = abi.EBB_MAP_ZERO_OUT
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o)
        abi.ebb_ctx_sync(dm.ctx)
        assert rel_err(tf.double().cpu().numpy().T, f) < 1e-5
        assert rel_err(tk.double().cpu().numpy().T, Kw) < 1e-5
        # the flag is refused outside the tiled variant
        o.flags = abi.EBB_MAP_TEST_DROP_TILE
        o.reduce = abi.EBB_REDUCE_ATOMIC
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o)
        assert ei.value.status == abi.EBB_ERR_ARG
