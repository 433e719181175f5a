"""The allocation-free implicit step against the regular one.

ebb_cg_implicit_step_noalloc serves callers that cannot allocate device
memory (a host framework that owns every device byte, a real-time loop that
must not touch the allocator): it keeps all of its working memory in one fixed
array inside the library.  Here it must reproduce ebb_cg_implicit_step on the
same mesh to the FP64 parity tolerance (1e-12 relative, max-norm), over two
calls in a row, so the second call also shows that state left in the shared
array by the first does not leak into the result.  This file is collected
last on purpose.
"""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

G = (0.0, 0.0, -9.81)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("model", ["stvk", "nh"])
def test_noalloc_step_matches_regular_step_twice(model):
    from paper_1506_07577_gb300 import abi
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh

    m = meshgen.cube_grid(6, jitter=0.01, seed=7)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=3)
    v0[m.pinned] = 0.0
    mdl = abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN
    prm = abi.step_params(mdl, 1e-3, 1000.0, mu, lam, G, abi.EBB_PREC_F64, max_iters=400, rtol=1e-14)
    dev = torch.device("cuda", 0)

    # regular entry point: relations, finalize, library-owned scratch
    ref = []
    with DeviceTetMesh(m.X, m.tets) as dm:
        u = dm.vertex_field("u", torch.float64)
        v = dm.vertex_field("v", torch.float64, value=v0)
        dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dev))
        for _ in range(2):
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
            ref.append((u.cpu().numpy().copy(), v.cpu().numpy().copy()))

    # allocation-free entry point: plain device arrays
    keys = torch.from_numpy(np.ascontiguousarray(m.tets.T)).to(dev)
    X = torch.from_numpy(np.ascontiguousarray(m.X.T)).to(dev)
    u = torch.zeros((3, m.n_verts), dtype=torch.float64, device=dev)
    v = torch.from_numpy(np.ascontiguousarray(v0.T)).to(dev)
    pin = torch.from_numpy(m.pinned.astype(np.uint8)).to(dev)
    torch.cuda.synchronize()
    for call in range(2):
        rep = abi.ebb_cg_implicit_step_noalloc(None, m.n_verts, m.n_tets, keys, X, u, v, pin, prm)
        assert rep.status == abi.EBB_OK and rep.iters > 0
        ur, vr = ref[call]
        assert _rel(v.cpu().numpy(), vr) < 1e-12, call
        assert _rel(u.cpu().numpy(), ur) < 1e-12, call


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1506_07577_gb300 import abi

    prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1e4, 1e4, G, abi.EBB_PREC_F64)
    dev = torch.device("cuda", 0)
    big = abi.EBB_NOALLOC_MAX_VERTS + 1
    X = torch.zeros((3, big), dtype=torch.float64, device=dev)
    with pytest.raises(abi.EbbError) as ei:
        abi.ebb_cg_implicit_step_noalloc(None, big, 0, None, X, X.clone(), X.clone(), None, prm)
    assert ei.value.status == abi.EBB_ERR_ARG
    keys = torch.zeros((4, abi.EBB_NOALLOC_MAX_TETS + 1), dtype=torch.int32, device=dev)
    with pytest.raises(abi.EbbError) as ei:
        abi.ebb_cg_implicit_step_noalloc(None, 4, abi.EBB_NOALLOC_MAX_TETS + 1, keys, X[:, :4].contiguous(),
                                         X[:, :4].contiguous(), X[:, :4].contiguous(), None, prm)
    assert ei.value.status == abi.EBB_ERR_ARG
    prm32 = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1e4, 1e4, G, abi.EBB_PREC_F32)
    with pytest.raises(abi.EbbError) as ei:
        abi.ebb_cg_implicit_step_noalloc(None, 4, 0, None, X[:, :4].contiguous(), X[:, :4].contiguous(),
                                         X[:, :4].contiguous(), None, prm32)
    assert ei.value.status == abi.EBB_ERR_ARG


def _noalloc_problem(n=3, seed=5):
    m = meshgen.cube_grid(n, jitter=0.01, seed=seed)
    dev = torch.device("cuda", 0)
    keys = torch.from_numpy(np.ascontiguousarray(m.tets.T)).to(dev)
    X = torch.from_numpy(np.ascontiguousarray(m.X.T)).to(dev)
    u = 0.001 * torch.from_numpy(np.ascontiguousarray(meshgen.random_field(m.n_verts, seed=seed).T)).to(dev)
    v = 0.05 * torch.from_numpy(np.ascontiguousarray(meshgen.random_field(m.n_verts, seed=seed + 1).T)).to(dev)
    return m, keys, X, u, v


def test_noalloc_bad_keys_and_inverted_rest_leave_state_untouched():
    """A key equal to n_verts, a key repeated inside one tet and an inverted
    rest tet are found before anything is written: the call fails and u, v
    keep their bits."""
    from paper_1506_07577_gb300 import abi

    m, keys, X, u, v = _noalloc_problem()
    prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, 1e4, 1e4, G, abi.EBB_PREC_F64, max_iters=50, rtol=1e-12)
    u0, v0 = u.clone(), v.clone()
    cases = []
    k = keys.clone()
    k[2, 7] = m.n_verts                        # out of range
    cases.append((k, abi.EBB_ERR_KEY))
    k = keys.clone()
    k[3, 4] = k[0, 4]                          # a vertex twice in one tet
    cases.append((k, abi.EBB_ERR_KEY))
    k = keys.clone()
    k[[2, 3], 5] = k[[3, 2], 5]                # two corners swapped: det(Dm) < 0
    cases.append((k, abi.EBB_ERR_INVERTED))
    for kk, want in cases:
        kk = kk.contiguous()
        torch.cuda.synchronize()
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step_noalloc(None, m.n_verts, m.n_tets, kk, X, u, v, None, prm)
        assert ei.value.status == want
        assert torch.equal(u, u0) and torch.equal(v, v0)


def test_noalloc_zero_iterations_moves_with_the_old_velocity():
    """max_iters = 0: no CG iteration, dv = 0, so v stays and u += dt v."""
    from paper_1506_07577_gb300 import abi

    m, keys, X, u, v = _noalloc_problem()
    dt = 1e-3
    prm = abi.step_params(abi.EBB_STVK, dt, 1000.0, 1e4, 1e4, G, abi.EBB_PREC_F64, max_iters=0, rtol=1e-12)
    u0, v0 = u.clone(), v.clone()
    torch.cuda.synchronize()
    rep = abi.ebb_cg_implicit_step_noalloc(None, m.n_verts, m.n_tets, keys, X, u, v, None, prm)
    assert rep.iters == 0 and rep.status == abi.EBB_OK
    assert torch.equal(v, v0)
    assert torch.allclose(u, u0 + dt * v0, rtol=0, atol=1e-18)
