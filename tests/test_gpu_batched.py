"""Batched implicit step (many independent meshes, per-mesh CG) against the
single-mesh step and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import fem, implicit
from _problems import rel_err

pytestmark = pytest.mark.gpu

G = (0.0, 0.0, -9.81)


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _batched(b, mu, lam, model, precision, max_iters, rtol, v0=None, steps=1, reduce=None):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    with DeviceTetMesh(b.X, b.tets, batch=b.batch) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64, value=np.zeros_like(b.X) if v0 is None else v0)
        dm.bind("pinned", torch.from_numpy(b.pinned.astype(np.uint8)).to(dm.device))
        prm = abi.step_params(abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN, 1e-3, 1000.0, mu, lam, G,
                              precision, max_iters=max_iters, rtol=rtol,
                              reduce=abi.EBB_REDUCE_AUTO if reduce is None else reduce)
        reps = []
        for _ in range(steps):
            reps.append(abi.ebb_cg_implicit_step_batched(dm.ctx, dm.tets, "u", "v", "pinned", "batch",
                                                         len(b.sides), prm))
        u = dm._tensors["u"].cpu().numpy().T.copy()
        v = dm._tensors["v"].cpu().numpy().T.copy()
    return u, v, reps


def _single(X, tets, pinned, mu, lam, model, precision, max_iters, rtol, v0, steps=1):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    with DeviceTetMesh(X, tets) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64, value=v0)
        dm.bind("pinned", torch.from_numpy(pinned.astype(np.uint8)).to(dm.device))
        prm = abi.step_params(abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN, 1e-3, 1000.0, mu, lam, G,
                              precision, max_iters=max_iters, rtol=rtol)
        reps = [abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm) for _ in range(steps)]
        return dm._tensors["u"].cpu().numpy().T.copy(), dm._tensors["v"].cpu().numpy().T.copy(), reps


@pytest.mark.parametrize("model", ["stvk", "nh"])
def test_batched_fp64_equals_single_mesh_steps(model):
    abi = _abi()
    b = meshgen.cube_grid_batch([2, 5, 3, 1, 4, 2, 6], jitter=0.01, seed=11)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    v0 = 0.05 * meshgen.random_field(b.X.shape[0], seed=5)
    v0[b.pinned] = 0.0
    ub, vb, reps = _batched(b, mu, lam, model, abi.EBB_PREC_F64, 400, 1e-14, v0, steps=2)
    iters = set()
    for m in range(len(b.sides)):
        X, tets, pinned = b.mesh(m)
        a, e = b.vert_off[m], b.vert_off[m + 1]
        us, vs, rs = _single(X, tets, pinned, mu, lam, model, abi.EBB_PREC_F64, 400, 1e-14, v0[a:e], steps=2)
        assert rel_err(vb[a:e], vs) < 1e-12, m
        assert rel_err(ub[a:e], us) < 1e-12, m
        for k in range(2):
            assert abs(reps[k][m].iters - rs[k].iters) <= 1
            assert reps[k][m].status == abi.EBB_OK
            iters.add(reps[k][m].iters)
    assert len(iters) > 1          # meshes really converge at different iterations


@pytest.mark.parametrize("reduce", ["auto", "gather", "ordered", "coop"])
def test_batched_mixed_matches_oracle_per_mesh(reduce):
    abi = _abi()
    b = meshgen.cube_grid_batch([3, 6, 4], jitter=0.01, seed=21)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    red = {"auto": abi.EBB_REDUCE_AUTO, "gather": abi.EBB_REDUCE_GATHER,
           "ordered": abi.EBB_REDUCE_TILED_ORDERED, "coop": abi.EBB_REDUCE_COOP}[reduce]
    ub, vb, reps = _batched(b, mu, lam, "nh", abi.EBB_PREC_F32, 1000, 1e-8, reduce=red)
    for m in range(len(b.sides)):
        X, tets, pinned = b.mesh(m)
        B, V = fem.rest_shape(X, tets)
        mass = fem.lumped_mass(V, tets, 1000.0, X.shape[0])
        uo, vo, info = implicit.implicit_step(X, np.zeros_like(X), np.zeros_like(X), tets, B, V, mass, mu, lam,
                                              fem.NEOHOOKEAN, 1e-3, np.array(G), pinned, 1000, 1e-8)
        a, e = b.vert_off[m], b.vert_off[m + 1]
        assert rel_err(vb[a:e], vo) < 1e-5, m
        assert rel_err(ub[a:e], uo) < 1e-5, m
        assert reps[0][m].rel_residual <= 1e-8


def test_batched_rejects_bad_batch_fields():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    b = meshgen.cube_grid_batch([2, 2], seed=1)
    # a tet joining two meshes is rejected at finalize
    tets = b.tets.copy()
    tets[0, 1] = b.vert_off[1]
    with pytest.raises(abi.EbbError) as ei:
        DeviceTetMesh(b.X, tets, batch=b.batch)
    assert ei.value.status == abi.EBB_ERR_KEY
    prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1e4, 1e4, G, abi.EBB_PREC_F64)
    with DeviceTetMesh(b.X, b.tets, batch=b.batch) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64)
        # ids must cover [0, nbatch)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step_batched(dm.ctx, dm.tets, "u", "v", None, "batch", 3, prm)
        assert ei.value.status == abi.EBB_ERR_ARG
        # ids must be non-decreasing along verts
        bad = torch.from_numpy(b.batch[::-1].copy()).to(dm.device)
        dm.bind("batch2", bad)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step_batched(dm.ctx, dm.tets, "u", "v", None, "batch2", 2, prm)
        assert ei.value.status == abi.EBB_ERR_ARG


def test_full_size_batch_sampled_meshes_match_oracle():
    """The benchmark's batch (256 cube grids, side log-uniform in [4, 24],
    3.4 M tets), one mixed step in one batched call; the smallest, a middle
    and the largest mesh are recomputed by the oracle on their own."""
    abi = _abi()
    sides = meshgen.batched_sizes(256, 4, 24, seed=4)
    b = meshgen.cube_grid_batch(sides, jitter=0.01, seed=400)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    ub, vb, reps = _batched(b, mu, lam, "nh", abi.EBB_PREC_F32, 1000, 1e-8)
    order = np.argsort(sides, kind="stable")
    for mi in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        X, tets, pinned = b.mesh(mi)
        B, V = fem.rest_shape(X, tets)
        mass = fem.lumped_mass(V, tets, 1000.0, X.shape[0])
        uo, vo, info = implicit.implicit_step(X, np.zeros_like(X), np.zeros_like(X), tets, B, V, mass, mu, lam,
                                              fem.NEOHOOKEAN, 1e-3, np.array(G), pinned, 1000, 1e-8)
        a, e = b.vert_off[mi], b.vert_off[mi + 1]
        assert rel_err(vb[a:e], vo) < 1e-5, mi
        assert rel_err(ub[a:e], uo) < 1e-5, mi
        assert reps[0][mi].rel_residual <= 1e-8
        assert abs(reps[0][mi].iters - info["iters"]) <= 2
