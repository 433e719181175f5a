"""GPU adjoint of the implicit step (StVK, FP64): the step VJP against the
oracle's adjoint, the checkpointed autograd rollout against the oracle's
rollout gradient and against central finite differences of the GPU forward
rollout (h = 1e-6, FP64), and checkpoint-interval invariance."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import adjoint, fem
from _problems import rel_err

pytestmark = pytest.mark.gpu

G = (0.0, 0.0, -9.81)
DT = 5e-3


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _setup(n, seed):
    m = meshgen.cube_grid(n, jitter=0.02, seed=seed)
    mu, lam = meshgen.material_perturbed_lame(m.n_tets, 1e5, 0.45, 0.2, seed)
    return m, mu, lam


def _mesh(m, mu, lam):
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    dm = DeviceTetMesh(m.X, m.tets, mu, lam)
    dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dm.device))
    return dm


def _params(rtol=1e-14):
    abi = _abi()
    return abi.step_params(abi.EBB_STVK, DT, 1000.0, gravity=G, precision=abi.EBB_PREC_F64, max_iters=2000,
                           rtol=rtol)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda()


def test_step_vjp_matches_oracle_adjoint():
    abi = _abi()
    m, mu, lam = _setup(3, seed=2)
    u = 0.3 * meshgen.random_displacement(m.X, 3, amp=0.05, seed=2)
    u[m.pinned] = 0
    v = 0.2 * meshgen.random_field(m.n_verts, seed=3)
    v[m.pinned] = 0
    rng = np.random.default_rng(1)
    gu_out, gv_out = rng.normal(size=u.shape), rng.normal(size=v.shape)
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    gu, gv, gmu, glam, _ = adjoint.step_vjp(m.X, u, v, m.tets, B, V, mass, mu, lam, DT, np.array(G), m.pinned,
                                            gu_out, gv_out)
    with _mesh(m, mu, lam) as dm:
        dm.vertex_field("u", torch.float64, value=u)
        dm.vertex_field("v", torch.float64, value=v)
        tgu = dm.vertex_field("gu", torch.float64, value=gu_out)
        tgv = dm.vertex_field("gv", torch.float64, value=gv_out)
        tgmu = dm.bind_tets("gmu", torch.zeros(m.n_tets, dtype=torch.float64, device=dm.device))
        tglam = dm.bind_tets("glam", torch.zeros(m.n_tets, dtype=torch.float64, device=dm.device))
        rep = abi.ebb_cg_implicit_step_vjp(dm.ctx, dm.tets, "u", "v", "pinned", "gu", "gv", "gmu", "glam",
                                           _params())
        assert rep.status == abi.EBB_OK
        assert rel_err(tgu.cpu().numpy().T, gu) < 1e-8
        assert rel_err(tgv.cpu().numpy().T, gv) < 1e-8
        assert rel_err(tgmu.cpu().numpy(), gmu) < 1e-8
        assert rel_err(tglam.cpu().numpy(), glam) < 1e-8
        # the state fields are read only
        assert np.array_equal(dm._tensors["u"].cpu().numpy().T, u)


def _rollout_grad_gpu(m, mu, lam, steps, every, u0, v0):
    from paper_1506_07577_gb300.autograd import rollout
    with _mesh(m, mu, lam) as dm:
        tu0 = _dev(u0).requires_grad_(True)
        tv0 = _dev(v0).requires_grad_(True)
        tmu = torch.from_numpy(mu).cuda().requires_grad_(True)
        tlam = torch.from_numpy(lam).cuda().requires_grad_(True)
        uT, vT = rollout(dm, tu0, tv0, tmu, tlam, steps, _params(), checkpoint_every=every)
        loss = (uT ** 2).sum()
        loss.backward()
        return (float(loss.detach()), tu0.grad.cpu().numpy().T, tv0.grad.cpu().numpy().T, tmu.grad.cpu().numpy(),
                tlam.grad.cpu().numpy())


def test_rollout_gradient_matches_oracle_and_is_checkpoint_invariant():
    m, mu, lam = _setup(3, seed=4)
    steps = 6
    u0 = np.zeros_like(m.X)
    v0 = 0.1 * meshgen.random_field(m.n_verts, seed=1)
    v0[m.pinned] = 0
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
    states = adjoint.rollout(m.X, u0, v0, m.tets, B, V, mass, mu, lam, DT, np.array(G), m.pinned, steps)
    uT = states[-1][0]
    gu, gv, gmu, glam, _ = adjoint.rollout_grad(m.X, u0, v0, m.tets, B, V, mass, mu, lam, DT, np.array(G),
                                                m.pinned, steps, 2 * uT, np.zeros_like(uT))
    results = [_rollout_grad_gpu(m, mu, lam, steps, every, u0, v0) for every in (4, 1, 6)]
    loss, tgu, tgv, tgmu, tglam = results[0]
    assert abs(loss - np.sum(uT ** 2)) < 1e-10 * np.sum(uT ** 2)
    assert rel_err(tgu, gu) < 1e-7
    assert rel_err(tgv, gv) < 1e-7
    assert rel_err(tgmu, gmu) < 1e-7
    assert rel_err(tglam, glam) < 1e-7
    for other in results[1:]:
        for a, b in zip(other[1:], results[0][1:]):
            assert rel_err(a, b) < 1e-10


def test_rollout_gradient_matches_gpu_finite_differences():
    """Central differences (h = 1e-6, FP64) of the GPU forward rollout."""
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam = _setup(6, seed=7)
    steps, every = 10, 5
    u0 = np.zeros_like(m.X)
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=2)
    v0[m.pinned] = 0
    loss, gu, gv, gmu, glam = _rollout_grad_gpu(m, mu, lam, steps, every, u0, v0)

    def forward_loss(u0_, v0_, mu_, lam_):
        with _mesh(m, mu_, lam_) as dm:
            dm.vertex_field("u", torch.float64, value=u0_)
            dm.vertex_field("v", torch.float64, value=v0_)
            for _ in range(steps):
                abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", _params())
            return float((dm._tensors["u"] ** 2).sum())

    rng = np.random.default_rng(11)
    for trial in range(2):
        du = rng.normal(size=u0.shape) * 1e-3
        du[m.pinned] = 0
        dv = rng.normal(size=v0.shape) * 1e-2
        dv[m.pinned] = 0
        dmu = rng.normal(size=mu.shape) * 1e3
        dlam = rng.normal(size=lam.shape) * 1e3
        h = 1e-6
        fd = (forward_loss(u0 + h * du, v0 + h * dv, mu + h * dmu, lam + h * dlam)
              - forward_loss(u0 - h * du, v0 - h * dv, mu - h * dmu, lam - h * dlam)) / (2 * h)
        an = np.sum(gu * du) + np.sum(gv * dv) + np.sum(gmu * dmu) + np.sum(glam * dlam)
        assert abs(fd - an) < 1e-4 * abs(an), (trial, fd, an)


def test_full_size_rollout_gradient_matches_finite_differences():
    """The benchmark's differentiable workload at full size (32^3 StVK,
    per-tet Lame within 20%, 20 steps, checkpoints every 5, dt = 1e-3):
    the autograd gradient against central differences of the GPU forward
    rollout along one random direction in (u0, v0, mu, lambda)."""
    abi = _abi()
    from paper_1506_07577_gb300.autograd import rollout
    n, steps, every, dt = 32, 20, 5, 1e-3
    m = meshgen.cube_grid(n, jitter=0.01, seed=3)
    mu, lam = meshgen.material_perturbed_lame(m.n_tets, 1e5, 0.45, 0.2, seed=3)
    prm = abi.step_params(abi.EBB_STVK, dt, 1000.0, precision=abi.EBB_PREC_F64, max_iters=4000, rtol=1e-12)
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=3)
    v0[m.pinned] = 0.0

    def loss_of(mu_, lam_, u0_, v0_):
        with _mesh(m, mu_, lam_) as dm:
            dm.vertex_field("fu", torch.float64, value=u0_)
            dm.vertex_field("fv", torch.float64, value=v0_)
            for _ in range(steps):
                abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "fu", "fv", "pinned", prm)
            return float((dm._tensors["fu"] ** 2).sum())

    with _mesh(m, mu, lam) as dm:
        tu0 = torch.zeros((3, m.n_verts), dtype=torch.float64, device="cuda", requires_grad=True)
        tv0 = _dev(v0).requires_grad_(True)
        tmu = torch.from_numpy(mu).cuda().requires_grad_(True)
        tlam = torch.from_numpy(lam).cuda().requires_grad_(True)
        uT, _ = rollout(dm, tu0, tv0, tmu, tlam, steps, prm, checkpoint_every=every)
        (uT ** 2).sum().backward()
        gu, gv = tu0.grad.cpu().numpy().T, tv0.grad.cpu().numpy().T
        gmu, glam = tmu.grad.cpu().numpy(), tlam.grad.cpu().numpy()
    rng = np.random.default_rng(0)
    du = rng.normal(size=m.X.shape) * 1e-3
    du[m.pinned] = 0.0
    dv = rng.normal(size=m.X.shape) * 1e-2
    dv[m.pinned] = 0.0
    dmu = rng.normal(size=mu.shape) * 1e3
    dlam = rng.normal(size=lam.shape) * 1e3
    h = 1e-6
    u0 = np.zeros_like(m.X)
    fd = (loss_of(mu + h * dmu, lam + h * dlam, u0 + h * du, v0 + h * dv)
          - loss_of(mu - h * dmu, lam - h * dlam, u0 - h * du, v0 - h * dv)) / (2 * h)
    an = float(np.sum(gu * du) + np.sum(gv * dv) + np.sum(gmu * dmu) + np.sum(glam * dlam))
    assert abs(fd - an) < 1e-4 * abs(an), (fd, an)


def test_vjp_rejects_unsupported_forms():
    abi = _abi()
    m, mu, lam = _setup(2, seed=1)
    with _mesh(m, mu, lam) as dm:
        for name in ("u", "v", "gu", "gv"):
            dm.vertex_field(name, torch.float64)
        prm = abi.step_params(abi.EBB_NEOHOOKEAN, DT, 1000.0, precision=abi.EBB_PREC_F64)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step_vjp(dm.ctx, dm.tets, "u", "v", None, "gu", "gv", None, None, prm)
        assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step_vjp(dm.ctx, dm.tets, "u", "v", None, "gu", "gu", None, None, _params())
        assert ei.value.status == abi.EBB_ERR_PHASE


def test_vjp_at_equals_vjp_with_its_own_solve():
    """The VJP given the step's new velocity (from a forward step) equals the
    VJP that re-solves the step, to the forward solve's tolerance; and it
    refuses a v_next that is also an output."""
    abi = _abi()
    m, mu, lam = _setup(4, seed=5)
    u = 0.3 * meshgen.random_displacement(m.X, 4, amp=0.05, seed=5)
    u[m.pinned] = 0
    v = 0.2 * meshgen.random_field(m.n_verts, seed=6)
    v[m.pinned] = 0
    rng = np.random.default_rng(3)
    gu_out, gv_out = rng.normal(size=u.shape), rng.normal(size=v.shape)
    res = []
    with _mesh(m, mu, lam) as dm:
        for given in (False, True):
            dm.vertex_field("u", torch.float64, value=u)
            dm.vertex_field("v", torch.float64, value=v)
            tgu = dm.vertex_field("gu", torch.float64, value=gu_out)
            tgv = dm.vertex_field("gv", torch.float64, value=gv_out)
            tgmu = dm.bind_tets("gmu", torch.zeros(m.n_tets, dtype=torch.float64, device=dm.device))
            tglam = dm.bind_tets("glam", torch.zeros(m.n_tets, dtype=torch.float64, device=dm.device))
            if given:
                # the step's result from a forward step on copies of the state
                dm.vertex_field("u1", torch.float64, value=u)
                vn = dm.vertex_field("vn", torch.float64, value=v)
                abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u1", "vn", "pinned", _params())
                abi.ebb_cg_implicit_step_vjp_at(dm.ctx, dm.tets, "u", "v", "vn", "pinned", "gu", "gv", "gmu",
                                                "glam", _params())
                with pytest.raises(abi.EbbError) as ei:
                    abi.ebb_cg_implicit_step_vjp_at(dm.ctx, dm.tets, "u", "v", "gu", "pinned", "gu", "gv", None,
                                                    None, _params())
                assert ei.value.status == abi.EBB_ERR_PHASE
            else:
                abi.ebb_cg_implicit_step_vjp(dm.ctx, dm.tets, "u", "v", "pinned", "gu", "gv", "gmu", "glam",
                                             _params())
            res.append([t.cpu().numpy().copy() for t in (tgu, tgv, tgmu, tglam)])
    for a, b in zip(res[1], res[0]):
        assert rel_err(a, b) < 1e-12
