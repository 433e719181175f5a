"""The fused map on host buffers (ebb_map_tet_force_Kv_host): against the
FP64 oracle and bit for bit against the device-buffer call (ordered tiled
reduction), in every field layout; accumulation and refusals."""
import numpy as np
import pytest
import torch

from _problems import oracle_maps, problem, rel_err

pytestmark = pytest.mark.gpu


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _host(arr, layout):
    """Host copy of an (N_v, 3) array in a field's layout, page-locked."""
    if layout == "x4":
        t = torch.zeros((arr.shape[0], 4), dtype=torch.float32)
        t[:, :3] = torch.from_numpy(arr.astype(np.float32))
    else:
        dt = torch.float64 if layout == "f64" else torch.float32
        t = torch.from_numpy(np.ascontiguousarray(arr.T)).to(dt)
    return t.pin_memory()


def _vec(t, layout):
    return (t[:, :3] if layout == "x4" else t.T).double().cpu().numpy()


@pytest.mark.parametrize("layout", ["x4", "f32", "f64"])
def test_host_map_matches_oracle_and_device_call(layout):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(6, "nh", seed=47)
    f, Kw, _ = oracle_maps(m, mu, lam, u, w, "nh")
    x4 = layout == "x4"
    dt = torch.float64 if layout == "f64" else torch.float32
    prec = abi.EBB_PREC_F64 if layout == "f64" else abi.EBB_PREC_F32
    tol = 1e-12 if layout == "f64" else 1e-5
    with DeviceTetMesh(m.X, m.tets, mu, lam) as dm:
        for name in ("u", "w", "f", "k", "ud", "wd", "fd", "kd"):
            dm.vertex_field(name, dt, x4=x4)
        uh, wh = _host(u, layout), _host(w, layout)
        fh, kh = torch.zeros_like(uh).pin_memory(), torch.zeros_like(uh).pin_memory()
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=prec, reduce=abi.EBB_REDUCE_TILED_ORDERED,
                         flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
        # the same map through device buffers
        dm._tensors["ud"].copy_(uh)
        dm._tensors["wd"].copy_(wh)
        torch.cuda.synchronize()
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "ud", "wd", "fd", "kd", o)
        abi.ebb_ctx_sync(dm.ctx)
        assert torch.equal(fh, dm._tensors["fd"].cpu()) and torch.equal(kh, dm._tensors["kd"].cpu())
        assert torch.equal(dm._tensors["f"].cpu(), fh)       # device fields keep the results
        # accumulation without EBB_MAP_ZERO_OUT
        o.flags = 0
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
    assert rel_err(_vec(fh, layout), 2 * f) < tol
    assert rel_err(_vec(kh, layout), 2 * Kw) < tol


def test_host_map_refusals_leave_fields_untouched():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(3, "stvk", seed=48)
    with DeviceTetMesh(m.X, m.tets, mu, lam) as du:
        tu = du.vertex_field("u", torch.float64, value=u)
        du.vertex_field("w", torch.float64, value=w)
        du.vertex_field("f", torch.float64)
        du.vertex_field("k", torch.float64)
        du.vertex_field("k32", torch.float32)
        before = tu.clone()
        uh = _host(np.zeros_like(u), "f64")
        wh, fh, kh = uh.clone(), uh.clone(), uh.clone()
        o = abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F64)
        with pytest.raises(abi.EbbError) as ei:              # u is also a reduce target
            abi.ebb_map_tet_force_Kv_host(du.ctx, du.tets, "u", "w", "u", "k", uh, wh, fh, kh, o)
        assert ei.value.status == abi.EBB_ERR_PHASE
        with pytest.raises(abi.EbbError) as ei:              # null host buffer
            abi.ebb_map_tet_force_Kv_host(du.ctx, du.tets, "u", "w", "f", "k", uh, None, fh, kh, o)
        assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError) as ei:              # an FP32 field in an FP64 map
            abi.ebb_map_tet_force_Kv_host(du.ctx, du.tets, "u", "w", "f", "k32", uh, wh, fh, kh, o)
        assert ei.value.status == abi.EBB_ERR_ARG
        # u and w name one device field but come from two host buffers: the
        # second copy would overwrite the first
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_force_Kv_host(du.ctx, du.tets, "u", "u", "f", "k", uh, wh, fh, kh, o)
        assert ei.value.status == abi.EBB_ERR_PHASE
        # the same for two names bound to one tensor
        du.bind("u_alias", tu)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_map_tet_force_Kv_host(du.ctx, du.tets, "u", "u_alias", "f", "k", uh, wh, fh, kh, o)
        assert ei.value.status == abi.EBB_ERR_PHASE
        torch.cuda.synchronize()
        assert torch.equal(tu, before)                       # nothing was copied in


def test_host_map_one_field_for_u_and_w():
    """u and w may be one field filled from one host buffer: K(u) u."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, _ = problem(4, "stvk", seed=49)
    f, Ku, _ = oracle_maps(m, mu, lam, u, u, "stvk")
    with DeviceTetMesh(m.X, m.tets, mu, lam) as dm:
        for name in ("u", "f", "k"):
            dm.vertex_field(name, torch.float64)
        uh = _host(u, "f64")
        fh, kh = torch.zeros_like(uh).pin_memory(), torch.zeros_like(uh).pin_memory()
        o = abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F64, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "u", "f", "k", uh, uh, fh, kh, o)
    assert rel_err(_vec(fh, "f64"), f) < 1e-12
    assert rel_err(_vec(kh, "f64"), Ku) < 1e-12


@pytest.mark.parametrize("layout", ["x4", "f32", "f64"])
@pytest.mark.parametrize("renumber", [True, False])
def test_chunked_host_map_matches_oracle(layout, renumber):
    """With the tiled reduction on a mesh of many tiles the host-buffer map
    runs in tile chunks whose copies overlap the map (on renumbered vertices
    the chunks touch nearly disjoint row ranges; on scattered ids the first
    chunk waits for almost every row): same results as the oracle, the
    accumulating call adds, and the host outputs equal the device fields."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(12, "stvk", seed=51, permute=True)
    f, Kw, _ = oracle_maps(m, mu, lam, u, w, "stvk")
    x4 = layout == "x4"
    dt = torch.float64 if layout == "f64" else torch.float32
    prec = abi.EBB_PREC_F64 if layout == "f64" else abi.EBB_PREC_F32
    tol = 1e-12 if layout == "f64" else 1e-5
    with DeviceTetMesh(m.X, m.tets, mu, lam, renumber_verts=renumber) as dm:
        assert abi.ebb_relation_info(dm.ctx, dm.tets).ntiles >= 16
        for name in ("u", "w", "f", "k"):
            dm.vertex_field(name, dt, x4=x4)
        uh, wh = _host(dm.rows(u), layout), _host(dm.rows(w), layout)
        fh, kh = torch.zeros_like(uh).pin_memory(), torch.zeros_like(uh).pin_memory()
        o = abi.map_opts(abi.EBB_STVK, precision=prec, reduce=abi.EBB_REDUCE_TILED, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
        assert rel_err(dm.caller(_vec(fh, layout)), f) < tol
        assert rel_err(dm.caller(_vec(kh, layout)), Kw) < tol
        assert torch.equal(dm._tensors["f"].cpu(), fh) and torch.equal(dm._tensors["k"].cpu(), kh)
        o.flags = 0
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
        assert rel_err(dm.caller(_vec(fh, layout)), 2 * f) < tol
        assert rel_err(dm.caller(_vec(kh, layout)), 2 * Kw) < tol


def _host_xyz(arr):
    """Host copy of an (N_v, 3) array as packed FP32 (x, y, z) rows, page-locked."""
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).pin_memory()


@pytest.mark.parametrize("reduce", ["tiled", "ordered"])
@pytest.mark.parametrize("renumber", [True, False])
def test_packed_host_rows_match_the_x4_host_call(reduce, renumber):
    """EBB_MAP_HOST_XYZ: 12-byte (x, y, z) host rows for 4-float fields, widened
    and narrowed on the device, in the chunked form (tiled, many tiles) and
    the whole-field form (ordered): the outputs equal, bit for bit, those of
    the same call on 16-byte host elements, and match the oracle; the
    accumulating call adds; one field for u and w works too."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(12, "stvk", seed=53, permute=True)
    f, Kw, _ = oracle_maps(m, mu, lam, u, w, "stvk")
    red = {"tiled": abi.EBB_REDUCE_TILED, "ordered": abi.EBB_REDUCE_TILED_ORDERED}[reduce]
    with DeviceTetMesh(m.X, m.tets, mu, lam, renumber_verts=renumber) as dm:
        assert abi.ebb_relation_info(dm.ctx, dm.tets).ntiles >= 16
        for name in ("u", "w", "f", "k"):
            dm.vertex_field(name, torch.float32, x4=True)
        ur, wr = dm.rows(u), dm.rows(w)
        uh, wh = _host_xyz(ur), _host_xyz(wr)
        fh, kh = torch.full_like(uh, 7.0).pin_memory(), torch.full_like(uh, 7.0).pin_memory()
        o = abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F32, reduce=red,
                         flags=abi.EBB_MAP_ZERO_OUT | abi.EBB_MAP_HOST_XYZ)
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
        assert rel_err(dm.caller(fh.double().numpy()), f) < 1e-5
        assert rel_err(dm.caller(kh.double().numpy()), Kw) < 1e-5
        assert torch.equal(dm._tensors["f"][:, :3].cpu(), fh)       # the fields hold the same values
        # the same call on 16-byte host elements
        ux, wx = _host(ur, "x4"), _host(wr, "x4")
        fx, kx = torch.zeros_like(ux).pin_memory(), torch.zeros_like(ux).pin_memory()
        ox = abi.map_opts(abi.EBB_STVK, precision=abi.EBB_PREC_F32, reduce=red, flags=abi.EBB_MAP_ZERO_OUT)
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", ux, wx, fx, kx, ox)
        if reduce == "ordered":
            assert torch.equal(fx[:, :3], fh) and torch.equal(kx[:, :3], kh)
        else:
            assert rel_err(fx[:, :3].double().numpy(), fh.double().numpy()) < 1e-6
        # accumulation
        o.flags = abi.EBB_MAP_HOST_XYZ
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
        assert rel_err(dm.caller(fh.double().numpy()), 2 * f) < 1e-5
        assert rel_err(dm.caller(kh.double().numpy()), 2 * Kw) < 1e-5
        # one field for u and w
        o.flags = abi.EBB_MAP_ZERO_OUT | abi.EBB_MAP_HOST_XYZ
        abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "u", "f", "k", uh, uh, fh, kh, o)
        _, Ku, _ = oracle_maps(m, mu, lam, u, u, "stvk")
        assert rel_err(dm.caller(kh.double().numpy()), Ku) < 1e-5


def test_packed_host_rows_need_float4_fields():
    """EBB_MAP_HOST_XYZ on 3-plane or FP64 fields is refused before anything
    is copied: the host outputs and the device fields keep their values."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = problem(3, "stvk", seed=55)
    for dt in (torch.float32, torch.float64):
        with DeviceTetMesh(m.X, m.tets, mu, lam) as dm:
            for name in ("u", "w", "f", "k"):
                dm.vertex_field(name, dt)
            tu = dm._tensors["u"]
            tu.fill_(3.0)
            uh, wh = _host_xyz(u), _host_xyz(w)
            fh = torch.full_like(uh, 5.0).pin_memory()
            kh = torch.full_like(uh, 5.0).pin_memory()
            prec = abi.EBB_PREC_F64 if dt == torch.float64 else abi.EBB_PREC_F32
            o = abi.map_opts(abi.EBB_STVK, precision=prec, flags=abi.EBB_MAP_ZERO_OUT | abi.EBB_MAP_HOST_XYZ)
            with pytest.raises(abi.EbbError) as ei:
                abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
            assert ei.value.status == abi.EBB_ERR_ARG
            torch.cuda.synchronize()
            assert (fh == 5.0).all() and (kh == 5.0).all() and (tu == 3.0).all()
